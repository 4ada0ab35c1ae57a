/*
 * oracle_dual.cpp -- the oracle (oracle.c, unchanged) compiled with dual numbers in place of double: every
 * function computes its value in .v and its directional derivative in .d. orc_rhs on a state with derivative
 * part delta returns RHS(u) and the Jacobian-vector product J(u) delta (forward-mode differentiation).
 *
 * TEST INFRASTRUCTURE, like oracle.c: only the tests call it; the library never links or calls it.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "dual.h"

typedef long double orc_ld_t;
#define ORC_LD_DEFINED 1
#define double dual
extern "C" {
#include "oracle.c"
}
#undef double
