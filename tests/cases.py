"""Shared set-up for tests: seeded scenarios evaluated by the oracle (CPU) and, in GPU tests, by the library.

Only the tests import this module. It builds oracle references; it never feeds a library result to the oracle.
"""
import math

import numpy as np

import oracle as orc
from paper_2112_10517_gb300 import inputs

PI = math.pi


def twisted_coords(nd, nelem, p, amp=0.1):
    """Affine nodes on [-pi, pi]^d moved by a smooth periodic map with a different perturbation per component."""
    xyz = orc.coords(nd, nelem, [-PI] * nd, [PI] * nd, p)
    X = [xyz[:, m].copy() for m in range(nd)]
    out = np.empty_like(xyz)
    for m in range(nd):
        a, b = X[(m + 1) % nd], X[(m + 2) % nd] if nd == 3 else X[m]
        out[:, m] = X[m] + amp * np.sin(a) * np.cos(b + 0.3 * m)
    return out


class Scenario:
    """A mesh + state, with the oracle's metrics and (lazily) its RHS."""

    def __init__(self, nd, nelem, p, mapping="sine", amp=0.1, box=None, ic="smooth", llf=True, seed=0,
                 flux="ranocha", state_fp32=False, **dg_extra):
        self.nd, self.nelem, self.p = nd, list(nelem), p
        self.mapping, self.amp, self.llf, self.flux = mapping, amp, llf, flux
        self.dg_extra = dg_extra  # library-only options (log-mean variants); the oracle has one definition
        self.lo, self.hi = box if box is not None else ([-PI] * nd, [PI] * nd)
        if mapping == "twisted":
            self.xyz = twisted_coords(nd, nelem, p, amp)
        elif mapping == "affine_nodes":  # affine coordinates handed over as nodes: the general (curved) code path
            self.xyz = orc.coords(nd, nelem, self.lo, self.hi, p, mapping=0, amp=0.0)
        else:
            self.xyz = orc.coords(nd, nelem, self.lo, self.hi, p, mapping=1 if mapping == "sine" else 0,
                                  amp=amp if mapping == "sine" else 0.0)
        self.Ja, self.J = orc.metrics(nd, p, self.xyz)
        L = [h - l for l, h in zip(self.lo, self.hi)]
        if ic == "smooth":
            self.u = inputs.smooth_random(self.xyz, seed=seed, lengths=L)
        elif ic == "rough":
            self.u = inputs.smooth_random(self.xyz, seed=seed, lengths=L) + 0.05 * inputs.random_state(self.xyz, seed + 1)
        elif ic == "random":
            self.u = inputs.random_state(self.xyz, seed=seed)
        elif ic == "tgv":
            self.u = inputs.taylor_green(self.xyz)
        elif ic == "noisy_sine":
            self.u = inputs.noisy_sine_2d(self.xyz, seed=seed)
        elif ic == "vortex":
            self.u = inputs.isentropic_vortex(self.xyz, eps=20.0)
        elif ic == "sine_paper":
            self.u = inputs.sine_paper(self.xyz)
        elif ic == "free_stream":
            self.u = inputs.free_stream(self.xyz)
        elif ic == "pressure_eq":
            self.u = inputs.pressure_equilibrium(self.xyz, seed=seed)
        else:
            raise ValueError(ic)
        if state_fp32:
            # float-representable state: the FP32 mode's rounding of the state is then exact, and differences of
            # the state at rounding level of FP64 (interface nodes whose coordinates differ in the last bit) are
            # the same on both sides
            self.u = self.u.astype(np.float32).astype(np.float64)
        self._du = None

    @property
    def E(self):
        return self.u.shape[0]

    def du_ref(self):
        if self._du is None:
            self._du = orc.rhs(self.nd, self.p, self.nelem, self.Ja, self.J, self.u, llf=self.llf, flux=self.flux)
        return self._du

    def du_scale(self):
        """(1/J) sum |terms| of the RHS sum at each node (oracle scale mode)."""
        if getattr(self, "_scale", None) is None:
            self._scale = orc.rhs(self.nd, self.p, self.nelem, self.Ja, self.J, self.u, llf=self.llf, scale=True,
                                  flux=self.flux)
        return self._scale

    def dg_kwargs(self):
        kw = dict(ndims=self.nd, nelem=self.nelem, polydeg=self.p, lo=self.lo, hi=self.hi,
                  surface="llf" if self.llf else "ec", flux=self.flux, **self.dg_extra)
        if self.mapping in ("twisted", "affine_nodes"):
            kw.update(mapping="nodes", node_xyz=self.xyz)
        elif self.mapping == "sine":
            kw.update(mapping="sine", amp=self.amp)
        else:
            kw.update(mapping="affine")
        return kw


def rel_err_per_var(got, ref):
    """max_i |got - ref| / max_i |ref| for each variable (normwise, per variable)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    nv = ref.shape[1]
    out = []
    for c in range(nv):
        scale = np.max(np.abs(ref[:, c]))
        out.append(np.max(np.abs(got[:, c] - ref[:, c])) / (scale if scale > 0 else 1.0))
    return np.array(out)


def parity_errors(got, ref, scale):
    """Per variable: (plain, term) errors. plain = max|got - ref| / max|ref|; term = max|got - ref| / max scale,
    with scale = (1/J) sum |terms| of the RHS sum (oracle scale mode): the magnitude that the rounding of any
    FP64 evaluation of the sum is proportional to. The two coincide up to the cancellation factor
    kappa = max scale / max|ref| of the data."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    plain, term = [], []
    for c in range(ref.shape[1]):
        d = np.max(np.abs(got[:, c] - ref[:, c]))
        r = np.max(np.abs(ref[:, c]))
        t = np.max(scale[:, c])
        plain.append(d / (r if r > 0 else 1.0))
        term.append(d / (t if t > 0 else 1.0))  # a variable whose terms all vanish (v = 0): absolute error
    return np.array(plain), np.array(term)


# FP64 parity bars (see test_parity_gpu.py): term-relative for every case; plain normwise relative wherever the data
# are well conditioned, i.e. for each variable whose cancellation factor kappa = max scale / max|du| is at most
# KAPPA_MAX. The plain error of two correct FP64 evaluations is about kappa times their term-relative difference:
# the plain bar is max(PLAIN64, PLAIN64_PER_KAPPA * kappa), which is 1e-12 for kappa <= 10 and a term-relative bar ten
# times stricter than TOL64 above (measured on the GPU: up to 8.8e-12 plain at kappa = 185, p = 7, i.e. 4.8e-14
# term-relative; the rough, random, vortex and smooth states have kappa = 3 .. 330). The Mach 0.1 Taylor-Green vortex
# sums pressure terms 1e3 .. 3e4 times larger than its RHS: the plain difference of two correct FP64 evaluations is
# ~1e-8 there and only the term-relative bar applies.
TOL64 = 1e-12
PLAIN64 = 1e-12
PLAIN64_PER_KAPPA = 1e-13
KAPPA_MAX = 1e3


def conditioning(ref, scale):
    """kappa per variable: max scale / max|ref| (inf where the RHS of a variable vanishes)."""
    out = []
    for c in range(ref.shape[1]):
        r = np.max(np.abs(ref[:, c]))
        out.append(np.max(scale[:, c]) / r if r > 0 else np.inf)
    return np.array(out)


def assert_parity(got, sc_or_ref, tol=TOL64, plain_tol="auto", scale=None):
    """Per-variable parity of `got` with the oracle: term-relative error <= tol, and, for FP64 bars (tol <= TOL64),
    plain normwise relative error <= max(plain_tol, PLAIN64_PER_KAPPA * kappa) for every variable with
    kappa <= KAPPA_MAX. sc_or_ref is a Scenario, or the oracle's RHS with `scale` given. Returns (plain, term,
    kappa)."""
    if scale is None:
        ref, scale = sc_or_ref.du_ref(), sc_or_ref.du_scale()
    else:
        ref = sc_or_ref
    plain, term = parity_errors(got, ref, scale)
    kappa = conditioning(np.asarray(ref), scale)
    if plain_tol == "auto":
        plain_tol = PLAIN64 if tol <= TOL64 else None
    print("parity plain %s | term %s | kappa %s" % (" ".join("%.1e" % x for x in plain),
                                                    " ".join("%.1e" % x for x in term),
                                                    " ".join("%.1e" % x for x in kappa)))
    assert np.all(term <= tol), (term, plain)
    if plain_tol is not None:
        mask = kappa <= KAPPA_MAX
        bar = np.maximum(plain_tol, PLAIN64_PER_KAPPA * kappa)
        assert np.all(plain[mask] <= bar[mask]), (plain, kappa)
    return plain, term, kappa
