"""The log-mean variants of the volume terms (Sec. 3.1, Algorithms 2 and 3, the polynomial 1/log form; Sec. 7.2,
logarithms precomputed once per node) against the oracle, on the three initial conditions of the paper's
ablation (isentropic vortex with eps = 20, the sinusoidal state rho = 2 + prod sin(pi x_m / 5), p = rho^gamma,
and a random state), in 2D and 3D and at every polynomial degree the kernels are compiled for.

All variants compute the same means up to rounding, so the bounds are those of the default path
(cases.assert_parity): FP64 1e-12 of the term magnitude (the oracle's scale mode) and a plain relative bar max(1e-12,
1e-13 kappa) for every variable with kappa <= 1e3, FP32 4e-6 of the term magnitude.
"""
import numpy as np
import pytest

import oracle as orc
from cases import TOL64, Scenario, assert_parity, parity_errors, rel_err_per_var

pytestmark = pytest.mark.gpu

TOL32 = 4e-6
BOX5 = {2: ([-5.0] * 2, [5.0] * 2), 3: ([-5.0] * 3, [5.0] * 3)}
VARIANTS = [dict(logmean="rcp", precompute_logs=True), dict(logmean="alg"), dict(logmean="alg_poly")]


@pytest.fixture(scope="module")
def dgmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10517_gb300 import build
    build.build()
    from paper_2112_10517_gb300 import dg
    return dg


def gpu_rhs(dgmod, sc, precision="fp64"):
    import torch
    ctx = dgmod.DG(precision=precision, **sc.dg_kwargs())
    du = ctx.rhs(torch.from_numpy(sc.u).cuda())
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    return du.cpu().numpy()


def scenario(nd, nelem, p, ic, seed=0, mapping="sine", **extra):
    return Scenario(nd, nelem, p, mapping=mapping, box=BOX5[nd], ic=ic, llf=True, seed=seed, **extra)


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
@pytest.mark.parametrize("p,nelem", [(1, [3, 4, 3]), (2, [3, 3, 3]), (3, [4, 3, 4]), (4, [2, 3, 3]),
                                     (5, [2, 2, 3]), (6, [2, 1, 3]), (7, [2, 2, 1])])
def test_variants_3d_every_degree(dgmod, variant, p, nelem):
    for ic in ("random", "sine_paper"):
        sc = scenario(3, nelem, p, ic, seed=60 + p, **VARIANTS[variant])
        assert_parity(gpu_rhs(dgmod, sc), sc, TOL64)


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
def test_variants_2d_every_degree(dgmod, variant, p):
    for ic in ("random", "sine_paper"):
        sc = scenario(2, [3, 4], p, ic, seed=70 + p, **VARIANTS[variant])
        assert_parity(gpu_rhs(dgmod, sc), sc, TOL64)


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
def test_variants_isentropic_vortex(dgmod, variant):
    # eps = 20 vortex on [-5, 5]^3, 8^3 elements, p = 3: constant far field (series branch) and a strong core
    sc = scenario(3, [8, 8, 8], 3, "vortex", **VARIANTS[variant])
    assert_parity(gpu_rhs(dgmod, sc), sc, TOL64)


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
def test_variants_agree_with_default(dgmod, variant):
    # the variants against the default path on identical data: both within rounding of the same sums
    base = scenario(3, [3, 3, 2], 4, "random", seed=80)
    var = scenario(3, [3, 3, 2], 4, "random", seed=80, **VARIANTS[variant])
    _, term = parity_errors(gpu_rhs(dgmod, var), gpu_rhs(dgmod, base), base.du_scale())
    assert np.all(term <= TOL64), term


@pytest.mark.parametrize("variant", range(len(VARIANTS)))
@pytest.mark.parametrize("nd,nelem,p", [(3, [3, 2, 3], 3), (2, [4, 5], 5), (3, [2, 2, 1], 7)])
def test_variants_fp32(dgmod, variant, nd, nelem, p):
    # float-representable states: the sinusoidal state has v = 0, so its density and energy rates are only the LLF
    # terms of FP64 rounding-level jumps at interfaces, which the FP32 rounding of the state would otherwise erase
    for ic in ("random", "sine_paper"):
        sc = scenario(nd, nelem, p, ic, seed=90, state_fp32=True, **VARIANTS[variant])
        assert_parity(gpu_rhs(dgmod, sc, precision="fp32"), sc, TOL32)


def test_precomputed_logs_cartesian(dgmod):
    for nd, nelem, p in ((3, [3, 4, 2], 3), (2, [5, 3], 6)):
        for precision, tol in (("fp64", TOL64), ("fp32", TOL32)):
            sc = scenario(nd, nelem, p, "random", seed=95, mapping="affine", precompute_logs=True)
            assert_parity(gpu_rhs(dgmod, sc, precision=precision), sc, tol)


def test_precomputed_logs_entropy_conservation(dgmod):
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="random", llf=False, seed=11, precompute_logs=True)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    du = ctx.rhs(u)
    s, ab = ctx.entropy_rate(u, du)
    assert abs(s) <= 1e-13 * ab, (s, ab)


@pytest.mark.parametrize("scheme", [0, 1])
def test_precomputed_logs_dg_step(dgmod, scheme):
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", box=BOX5[3], ic="sine_paper", llf=True, precompute_logs=True)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    dt = 0.01
    ref = sc.u
    for _ in range(3):
        ctx.step(u, dt, scheme=scheme)
        ref = orc.rk_step(scheme, 3, 3, sc.nelem, sc.Ja, sc.J, ref, dt, llf=True)
    err = rel_err_per_var(u.cpu().numpy() - sc.u, ref - sc.u)
    assert np.all(err <= 1e-11), err


def test_variant_restrictions(dgmod):
    import torch
    sc = scenario(3, [2, 2, 2], 3, "sine_paper", logmean="alg")
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    with pytest.raises(dgmod.DGError) as ei:  # the algorithm variants are dg_rhs only
        ctx.step(u, 0.01)
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    sc = scenario(3, [2, 2, 2], 3, "sine_paper", precompute_logs=True)
    ctx = dgmod.DG(**sc.dg_kwargs())
    with pytest.raises(dgmod.DGError) as ei:
        ctx.vjp(u, u.clone())
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    alg = dgmod.DG(**scenario(3, [2, 2, 2], 3, "sine_paper", logmean="alg").dg_kwargs())
    with pytest.raises(dgmod.DGError) as ei:  # batches run the default or the precomputed-logarithm kernels
        dgmod.DGBatch([alg], [u], [torch.empty_like(u)])
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    kw = scenario(3, [2, 2, 2], 3, "sine_paper").dg_kwargs()
    kw.update(flux="shima", precompute_logs=True)  # the Shima flux has no logarithmic means
    with pytest.raises(dgmod.DGError) as ei:
        dgmod.DG(**kw)
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
