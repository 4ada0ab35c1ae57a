"""Plain FP64 CPU oracle for entropy-stable flux-differencing LGL-DGSEM (arXiv:2112.10517).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` are the only callers. The library under ``paper_2112_10517_gb300`` never imports this
package and shares no code with it; this package never imports the library.

The arithmetic lives in ``oracle.c`` (plain C, IEEE double), compiled with gcc on first use into
``oracle/_build/liboracle.so``. This module only marshals numpy arrays. Every function cites the
paper's section or equation it follows; the C file states the formulas.

Array layouts (numpy, C order), N = p+1, Nd = N**ndims, nvar = ndims+2:
  u, du   [E, nvar, Nd]      conserved (rho, rho v_1..rho v_d, rho e); node index i1 fastest
  Ja      [E, ndims, ndims, Nd]  Ja[e, n, j] = (Ja^n)_j (reference direction n, Cartesian j)
  J       [E, Nd]
  xyz     [E, ndims, Nd]
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRC_GAUSS = os.path.join(_HERE, "gauss.c")
_SRC_DUAL = [os.path.join(_HERE, "oracle_dual.cpp"), os.path.join(_HERE, "dual.h")]
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_LIB_DUAL = os.path.join(_BUILD, "liboracle_dual.so")
_lock = threading.Lock()
_lib = None
_libd = None

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


def build(force: bool = False) -> str:
    """Compile oracle.c and gauss.c with gcc (plain -O2, no fast-math, portable flags) into oracle/_build, and the
    LGL source with dual numbers (oracle_dual.cpp, g++) for the JVP."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_LIB_PATH)) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(_SRC_GAUSS))
    if force or stale:
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, _SRC_GAUSS, "-lm"])
        os.replace(tmp, _LIB_PATH)
    deps = [_SRC] + _SRC_DUAL
    stale = (not os.path.exists(_LIB_DUAL)) or os.path.getmtime(_LIB_DUAL) < max(os.path.getmtime(d) for d in deps)
    if force or stale:
        tmp = _LIB_DUAL + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC_DUAL[0], "-lm"])
        os.replace(tmp, _LIB_DUAL)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB_PATH)
            lib.orc_logmean.restype = ctypes.c_double
            lib.orc_logmean.argtypes = [ctypes.c_double, ctypes.c_double]
            lib.orc_entropy_rate.restype = ctypes.c_double
            lib.orc_entropy.restype = ctypes.c_double
            _lib = lib
    return _lib


def _load_dual():
    global _libd
    _load()
    with _lock:
        if _libd is None:
            _libd = ctypes.CDLL(_LIB_DUAL)
    return _libd


class _Dual(ctypes.Structure):
    _fields_ = [("v", ctypes.c_double), ("d", ctypes.c_double)]


def _ptr(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ivec(v):
    arr = (ctypes.c_int * 3)(*(list(v) + [1] * (3 - len(v))))
    return arr


def _dvec(v):
    return (ctypes.c_double * 3)(*(list(v) + [0.0] * (3 - len(v))))


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle %s failed (rc=%d)" % (what, rc))


# --------------------------------------------------------------------------------------------
# Reference element (Sec. 2: LGL example, Def. derivative matrix)
# --------------------------------------------------------------------------------------------

def lgl(p: int):
    """LGL nodes and weights on [-1, 1] (Sec. 2, LGL-DGSEM example)."""
    lib = _load()
    x = np.zeros(p + 1)
    w = np.zeros(p + 1)
    _check(lib.orc_lgl(p, _ptr(x), _ptr(w)), "lgl")
    return x, w


def dmat(p: int) -> np.ndarray:
    """Nodal derivative matrix D, D[i, k] = l_k'(x_i) (Sec. 2, Def. derivative matrix)."""
    lib = _load()
    x, _ = lgl(p)
    D = np.zeros((p + 1, p + 1))
    _check(lib.orc_dmat(p, _ptr(x), _ptr(D)), "dmat")
    return D


# --------------------------------------------------------------------------------------------
# Pointwise physics (Sec. 3: Eq. Euler, Eq. logmean, Eq. flux_ranocha; Sec. 2 entropy pair)
# --------------------------------------------------------------------------------------------

def logmean(a, b) -> np.ndarray:
    """Logarithmic mean [[a]]/[[log a]] (Eq. logmean), via log1p."""
    lib = _load()
    a = _f64(a)
    b = _f64(np.broadcast_to(b, a.shape))
    out = np.zeros_like(a)
    lib.orc_logmean_batch(a.size, _ptr(a), _ptr(b), _ptr(out))
    return out


def euler_flux(u, j: int, ndims: int, gamma: float = 1.4) -> np.ndarray:
    """Physical flux f^j(u) for states u[..., nvar] (Eq. Euler)."""
    lib = _load()
    u = _f64(u)
    f = np.zeros_like(u)
    lib.orc_euler_flux_batch(u.size // (ndims + 2), _ptr(u), ndims, ctypes.c_double(gamma), j, _ptr(f))
    return f


FLUXES = {"ranocha": 0, "shima": 1}


def flux_dir(um, up, m, ndims: int, gamma: float = 1.4, flux: str = "ranocha") -> np.ndarray:
    """Directional two-point flux f(u-, u+, m) = sum_j m_j F_j (Eq. flux_ranocha or Eq. flux_shima_etal)."""
    lib = _load()
    um = _f64(um)
    up = _f64(np.broadcast_to(up, um.shape))
    n = um.size // (ndims + 2)
    m = _f64(np.broadcast_to(m, (n, ndims)))
    f = np.zeros_like(um)
    lib.orc_flux_dir_batch(FLUXES[flux], n, _ptr(um), _ptr(up), ndims, ctypes.c_double(gamma), _ptr(m), _ptr(f))
    return f


def flux_ranocha(um, up, m, ndims: int, gamma: float = 1.4) -> np.ndarray:
    """Directional Ranocha flux f(u-, u+, m) = sum_j m_j F_j (Eq. flux_ranocha; Sec. 2.3)."""
    return flux_dir(um, up, m, ndims, gamma, "ranocha")


def surface_flux(uin, uout, m, ndims: int, gamma: float = 1.4, llf: bool = True, flux: str = "ranocha") -> np.ndarray:
    """Surface flux: the two-point flux minus local Lax-Friedrichs dissipation when llf (Sec. 4.2)."""
    lib = _load()
    uin = _f64(uin)
    uout = _f64(np.broadcast_to(uout, uin.shape))
    n = uin.size // (ndims + 2)
    m = _f64(np.broadcast_to(m, (n, ndims)))
    f = np.zeros_like(uin)
    lib.orc_surface_flux_batch(FLUXES[flux], n, _ptr(uin), _ptr(uout), ndims, ctypes.c_double(gamma), _ptr(m),
                               int(bool(llf)), _ptr(f))
    return f


def entropy(u, ndims: int, gamma: float = 1.4):
    """Entropy U(u) and entropy variables w(u) = dU/du for states u[..., nvar] (Sec. 2)."""
    lib = _load()
    u = _f64(u)
    n = u.size // (ndims + 2)
    U = np.zeros(n)
    w = np.zeros_like(u)
    lib.orc_entropy_batch(n, _ptr(u), ndims, ctypes.c_double(gamma), _ptr(U), _ptr(w))
    return U.reshape(u.shape[:-1]), w


# --------------------------------------------------------------------------------------------
# Mesh, metrics (Sec. 2.3) and the semidiscretization (Eq. strong-form-SBP + Eq. fluxdiff-SBP)
# --------------------------------------------------------------------------------------------

def num_elements(ndims: int, nelem) -> int:
    return int(np.prod(list(nelem)[:ndims]))


def coords(ndims: int, nelem, lo, hi, p: int, mapping: int = 0, amp: float = 0.0) -> np.ndarray:
    """Node coordinates [E, ndims, Nd] of the periodic box mesh (affine or sine-perturbed mapping)."""
    lib = _load()
    E = num_elements(ndims, nelem)
    xyz = np.zeros((E, ndims, (p + 1) ** ndims))
    _check(lib.orc_coords(ndims, _ivec(nelem), _dvec(lo), _dvec(hi), p, mapping, ctypes.c_double(amp),
                          _ptr(xyz)), "coords")
    return xyz


def metrics(ndims: int, p: int, xyz, curl_form: bool = True):
    """Contravariant metric terms Ja [E, d, d, Nd] and Jacobian J [E, Nd] from node coordinates
    (Sec. 2.3; 3D conservative curl form unless curl_form=False, the cross-product negative control)."""
    lib = _load()
    xyz = _f64(xyz)
    E = xyz.shape[0]
    Nd = (p + 1) ** ndims
    Ja = np.zeros((E, ndims, ndims, Nd))
    J = np.zeros((E, Nd))
    _check(lib.orc_metrics(ndims, p, E, _ptr(xyz), int(bool(curl_form)), _ptr(Ja), _ptr(J)), "metrics")
    return Ja, J


def rhs(ndims: int, p: int, nelem, Ja, J, u, gamma: float = 1.4, llf: bool = True,
        elem_range=None, scale: bool = False, flux: str = "ranocha") -> np.ndarray:
    """du/dt of the flux-differencing LGL-DGSEM (Eq. strong-form-SBP with Eq. fluxdiff-SBP,
    curvilinear via Eq. curvilinear-rewrite). elem_range=(b, e) computes only elements [b, e) and returns
    that slice [e-b, nvar, Nd]. scale=True returns instead (1/J) x the sum of |terms| of that sum, the
    magnitude that the rounding of any evaluation of it scales with."""
    lib = _load()
    Ja = _f64(Ja)
    J = _f64(J)
    u = _f64(u)
    E = num_elements(ndims, nelem)
    assert u.shape == (E, ndims + 2, (p + 1) ** ndims), u.shape
    b, e = (0, E) if elem_range is None else elem_range
    assert 0 <= b <= e <= E
    du = np.zeros((e - b,) + u.shape[1:])
    _check(lib.orc_rhs(ndims, p, _ivec(nelem), _ptr(Ja), _ptr(J), _ptr(u), ctypes.c_double(gamma),
                       FLUXES[flux], int(bool(llf)), int(b), int(e), int(bool(scale)), _ptr(du)), "rhs")
    return du


def integrate(ndims: int, p: int, J, q):
    """(sum J W q_c, sum |J W q_c|) per field c of q [E, nvar, Nd] (LGL quadrature)."""
    lib = _load()
    J = _f64(J)
    q = _f64(q)
    nv = ndims + 2
    out = np.zeros(nv)
    ab = np.zeros(nv)
    lib.orc_integrate(ndims, p, q.shape[0], _ptr(J), _ptr(q), _ptr(out), _ptr(ab))
    return out, ab


def entropy_rate(ndims: int, p: int, J, u, du, gamma: float = 1.4):
    """(dS/dt, scale) with dS/dt = sum J W w(u).du and scale = sum |J W w(u).du| (Sec. 2)."""
    lib = _load()
    J = _f64(J)
    u = _f64(u)
    du = _f64(du)
    ab = ctypes.c_double(0.0)
    s = lib.orc_entropy_rate(ndims, p, u.shape[0], _ptr(J), _ptr(u), _ptr(du), ctypes.c_double(gamma),
                             ctypes.byref(ab))
    return float(s), float(ab.value)


RK4_CLASSIC = 0
LSRK45_CK = 1


def ck45_coefficients():
    """A, B of the 2N-storage five-stage fourth-order method of Carpenter and Kennedy (Sec. 4.1)."""
    lib = _load()
    A = np.zeros(5)
    B = np.zeros(5)
    lib.orc_ck45_coeffs(_ptr(A), _ptr(B))
    return A, B


def rk_step(scheme: int, ndims: int, p: int, nelem, Ja, J, u, dt: float, gamma: float = 1.4,
            llf: bool = True, flux: str = "ranocha") -> np.ndarray:
    """One time step (Sec. 4.1): scheme 0 classical RK4, scheme 1 Carpenter-Kennedy 5-stage 2N."""
    lib = _load()
    u = _f64(u).copy()
    _check(lib.orc_rk_step(scheme, ndims, p, _ivec(nelem), _ptr(_f64(Ja)), _ptr(_f64(J)),
                           ctypes.c_double(gamma), FLUXES[flux], int(bool(llf)), ctypes.c_double(dt), _ptr(u)),
           "rk_step")
    return u


def logmean_grad(a, b):
    """(dL/da, dL/db) of the oracle's logarithmic mean, by its dual-number evaluation."""
    lib = _load_dual()
    lib.orc_logmean.restype = _Dual
    lib.orc_logmean.argtypes = [_Dual, _Dual]
    a = np.atleast_1d(_f64(a))
    b = np.atleast_1d(_f64(np.broadcast_to(b, a.shape)))
    ga = np.array([lib.orc_logmean(_Dual(x, 1.0), _Dual(y, 0.0)).d for x, y in zip(a, b)])
    gb = np.array([lib.orc_logmean(_Dual(x, 0.0), _Dual(y, 1.0)).d for x, y in zip(a, b)])
    return ga, gb


def jvp(ndims: int, p: int, nelem, Ja, J, u, delta, gamma: float = 1.4, llf: bool = True, flux: str = "ranocha"):
    """(RHS(u), J(u) delta): the oracle's RHS evaluated in dual numbers (oracle_dual.cpp compiles oracle.c with
    `double` taken as a dual number), i.e. forward-mode differentiation, exact up to rounding."""
    lib = _load_dual()
    u = _f64(u)
    delta = _f64(np.broadcast_to(delta, u.shape))
    E = num_elements(ndims, nelem)
    assert u.shape == (E, ndims + 2, (p + 1) ** ndims), u.shape

    def dual_of(v, d=None):
        out = np.zeros(np.shape(v) + (2,))
        out[..., 0] = v
        if d is not None:
            out[..., 1] = d
        return out

    Jad = dual_of(_f64(Ja))
    Jd = dual_of(_f64(J))
    ud = dual_of(u, delta)
    dud = np.zeros_like(ud)
    _check(lib.orc_rhs(ndims, p, _ivec(nelem), _ptr(Jad), _ptr(Jd), _ptr(ud), _Dual(gamma, 0.0),
                       FLUXES[flux], int(bool(llf)), 0, E, 0, _ptr(dud)), "rhs (dual)")
    return dud[..., 0].copy(), dud[..., 1].copy()


# --------------------------------------------------------------------------------------------
# Legendre-Gauss collocation with entropy projection (Sec. 6, gauss.c), affine periodic boxes
# --------------------------------------------------------------------------------------------

def gauss(p: int):
    """Legendre-Gauss nodes and weights with p + 1 points (Sec. 6)."""
    lib = _load()
    x = np.zeros(p + 1)
    w = np.zeros(p + 1)
    _check(lib.org_gauss(p, _ptr(x), _ptr(w)), "org_gauss")
    return x, w


def lagrange_at(p: int, x, s: float) -> np.ndarray:
    """Lagrange basis of the nodes x at the point s (the rows of the face restriction R)."""
    lib = _load()
    x = _f64(x)
    out = np.zeros(p + 1)
    lib.org_lagrange_at(p, _ptr(x), ctypes.c_double(s), _ptr(out))
    return out


def cons_from_entropy(w, ndims: int, gamma: float = 1.4) -> np.ndarray:
    """u(w), the inverse of the entropy-variable map (Sec. 2), for states w[..., nvar]."""
    lib = _load()
    w = _f64(w)
    u = np.zeros_like(w)
    lib.org_cons_from_entropy_batch(w.size // (ndims + 2), _ptr(w), ndims, ctypes.c_double(gamma), _ptr(u))
    return u


def gauss_coords(ndims: int, nelem, lo, hi, p: int) -> np.ndarray:
    """Node coordinates [E, ndims, Nd] of the Gauss collocation mesh of the box [lo, hi]."""
    lib = _load()
    E = num_elements(ndims, nelem)
    xyz = np.zeros((E, ndims, (p + 1) ** ndims))
    _check(lib.org_gauss_coords(ndims, _ivec(nelem), _dvec(lo), _dvec(hi), p, _ptr(xyz)), "org_gauss_coords")
    return xyz


def gauss_rhs(ndims: int, p: int, nelem, lo, hi, u, gamma: float = 1.4, llf: bool = False) -> np.ndarray:
    """du/dt of the Legendre-Gauss collocation scheme with entropy projection (Sec. 6, Eq. fluxdiff-GSBP-opDsplit
    and Eq. hybridized_gauss_formulation), Ranocha's flux in the volume and at the surface, optional LLF."""
    lib = _load()
    u = _f64(u)
    du = np.zeros_like(u)
    _check(lib.org_gauss_rhs(ndims, p, _ivec(nelem), _dvec(lo), _dvec(hi), _ptr(u), ctypes.c_double(gamma),
                             int(llf), _ptr(du)), "org_gauss_rhs")
    return du


def dmat_nodes(p: int, x) -> np.ndarray:
    """Nodal derivative matrix of arbitrary distinct nodes x (barycentric form, as dmat)."""
    lib = _load()
    x = _f64(x)
    D = np.zeros((p + 1, p + 1))
    _check(lib.orc_dmat(p, _ptr(x), _ptr(D)), "orc_dmat")
    return D


def gauss_project(ndims: int, p: int, u, gamma: float = 1.4) -> np.ndarray:
    """The entropy projection (Sec. 6): face states u(R w(u)) [E, 2 ndims (p+1)^(ndims-1), nvar], face node
    f = (n*2 + s)*NL + t (direction n, side s = 0 at xi_n = -1, t over the other directions)."""
    lib = _load()
    u = _f64(u)
    E = u.shape[0]
    NL = (p + 1) ** (ndims - 1)
    out = np.zeros((E, 2 * ndims * NL, ndims + 2))
    _check(lib.org_gauss_project(ndims, p, E, _ptr(u), ctypes.c_double(gamma), _ptr(out)), "org_gauss_project")
    return out
