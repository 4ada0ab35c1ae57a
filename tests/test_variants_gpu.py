"""Parity of the library's variants with the oracle: the kinetic-energy- and pressure-equilibrium-preserving
flux of Shima et al. (Sec. 2.2; the second two-point flux the paper evaluates), and the Cartesian
specialisation that an affine mesh runs (constant metric terms Ja^i_i = J / (h_i / 2) and 1/J, no per-node
metric loads).

Same measure and bounds as the Ranocha-flux parity tests (cases.assert_parity): FP64 1e-12 of the term magnitude
(the oracle's scale mode) and a plain relative bar max(1e-12, 1e-13 kappa) for every variable with kappa <= 1e3
(all but the Mach 0.1 Taylor-Green vortex), FP32 4e-6 of the term magnitude.
"""
import numpy as np
import pytest

import oracle as orc
from cases import TOL64, Scenario, assert_parity, parity_errors, rel_err_per_var

pytestmark = pytest.mark.gpu

TOL32 = 4e-6


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
    return ctx, du.cpu().numpy()


# ------------------------------------------------------------------------------------------------
# Shima et al. flux, curvilinear meshes
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("p,nelem", [(1, [3, 4, 5]), (2, [3, 3, 3]), (3, [3, 2, 5]), (4, [2, 3, 3]),
                                     (5, [2, 2, 3]), (7, [2, 2, 1])])
@pytest.mark.parametrize("llf", [False, True])
def test_shima_3d_curved(dgmod, p, nelem, llf):
    sc = Scenario(3, nelem, p, mapping="sine", ic="rough", llf=llf, seed=30 + p, flux="shima")
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc, TOL64)


@pytest.mark.parametrize("p", [1, 3, 6])
def test_shima_2d_curved_and_twisted(dgmod, p):
    for mapping in ("sine", "twisted"):
        sc = Scenario(2, [3, 4], p, mapping=mapping, ic="rough", llf=True, seed=40 + p, flux="shima")
        _, du = gpu_rhs(dgmod, sc)
        assert_parity(du, sc, TOL64)


def test_shima_tgv_16cubed_p3(dgmod):
    sc = Scenario(3, [16, 16, 16], 3, mapping="sine", ic="tgv", llf=True, flux="shima")
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc, TOL64)


@pytest.mark.parametrize("nd,nelem,p", [(3, [3, 2, 3], 4), (2, [4, 5], 3)])
def test_shima_fp32(dgmod, nd, nelem, p):
    sc = Scenario(nd, nelem, p, mapping="sine", ic="rough", llf=True, seed=45, flux="shima")
    _, du = gpu_rhs(dgmod, sc, precision="fp32")
    assert_parity(du, sc, TOL32)


def test_shima_conservation_and_free_stream(dgmod):
    sc = Scenario(3, [3, 3, 2], 4, mapping="twisted", ic="rough", llf=True, seed=46, flux="shima")
    _, du = gpu_rhs(dgmod, sc)
    tot, ab = orc.integrate(3, 4, sc.J, du)
    assert np.all(np.abs(tot) <= 1e-13 * ab)
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="free_stream", llf=True, flux="shima")
    _, du = gpu_rhs(dgmod, sc)
    scale = sc.du_scale()
    for c in range(5):
        assert np.max(np.abs(du[:, c])) <= 1e-13 * np.max(scale[:, c]), c


def test_shima_pressure_equilibrium(dgmod):
    # uniform velocity and pressure: momentum and energy rates follow the density rate exactly (the flux's
    # pressure-equilibrium property, Sec. 2.2)
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="pressure_eq", llf=True, seed=13, flux="shima")
    _, du = gpu_rhs(dgmod, sc)
    v = [0.1, -0.2, 0.3]
    scale = np.max(np.abs(du[:, 0]))
    for j in range(3):
        np.testing.assert_allclose(du[:, 1 + j], v[j] * du[:, 0], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(du[:, 4], 0.5 * np.dot(v, v) * du[:, 0], rtol=0, atol=1e-12 * scale)


def test_shima_is_not_entropy_conservative(dgmod):
    # negative control for the entropy test of the Ranocha flux: the same rough state with central surface
    # fluxes produces an entropy rate far above rounding under the Shima flux
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="random", llf=False, seed=11, flux="shima")
    ctx, du = gpu_rhs(dgmod, sc)
    s, ab = ctx.entropy_rate(torch.from_numpy(sc.u).cuda(), torch.from_numpy(du).cuda())
    assert abs(s) > 1e-8 * ab, (s, ab)
    s_ref, ab_ref = orc.entropy_rate(3, 3, sc.J, sc.u, du)
    assert abs(s - s_ref) <= 1e-13 * ab_ref


@pytest.mark.parametrize("scheme", [0, 1])
def test_shima_dg_step(dgmod, scheme):
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="smooth", llf=True, seed=47, flux="shima")
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    dt = 0.01
    ref = sc.u
    for _ in range(3):
        ctx.step(u, dt, scheme=scheme)
        ref = orc.rk_step(scheme, 3, 3, sc.nelem, sc.Ja, sc.J, ref, dt, llf=True, flux="shima")
    err = rel_err_per_var(u.cpu().numpy() - sc.u, ref - sc.u)
    assert np.all(err <= 1e-11), err


def test_shima_rejected_by_adjoint_and_batch(dgmod):
    import torch
    sc = Scenario(3, [2, 2, 2], 3, mapping="sine", ic="smooth", llf=True, seed=48, flux="shima")
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    with pytest.raises(dgmod.DGError) as ei:
        ctx.vjp(u, u.clone())
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    with pytest.raises(dgmod.DGError) as ei:
        dgmod.DGBatch([ctx], [u], [torch.empty_like(u)])
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED


# ------------------------------------------------------------------------------------------------
# Cartesian specialisation: an affine mesh (constant metrics) against the oracle and against the general
# curvilinear path on the same mesh (affine coordinates handed over as nodes)
# ------------------------------------------------------------------------------------------------

CART_CASES = [
    # 2D Euler, [-1,1]^2, 8x8 quads, p = 3, noisy sine density wave
    dict(nd=2, nelem=[8, 8], p=3, box=([-1.0, -1.0], [1.0, 1.0]), ic="noisy_sine"),
    # anisotropic boxes and element counts: h differs per direction
    dict(nd=2, nelem=[5, 3], p=5, box=([-1.0, 0.0], [2.0, 0.5]), ic="rough"),
    dict(nd=3, nelem=[3, 4, 2], p=3, box=([-1.0, -2.0, 0.0], [1.0, 2.0, 3.0]), ic="rough"),
    dict(nd=3, nelem=[2, 3, 3], p=4, box=([0.0, 0.0, 0.0], [1.0, 3.0, 0.7]), ic="random"),
    dict(nd=3, nelem=[4, 4, 4], p=7, box=None, ic="tgv"),
]


@pytest.mark.parametrize("case", range(len(CART_CASES)))
@pytest.mark.parametrize("flux", ["ranocha", "shima"])
def test_cartesian_fp64(dgmod, case, flux):
    c = CART_CASES[case]
    for llf in (False, True):
        sc = Scenario(c["nd"], c["nelem"], c["p"], mapping="affine", box=c["box"], ic=c["ic"], llf=llf, seed=50,
                      flux=flux)
        ctx, du = gpu_rhs(dgmod, sc)
        assert_parity(du, sc, TOL64)
        gen = Scenario(c["nd"], c["nelem"], c["p"], mapping="affine_nodes", box=c["box"], ic=c["ic"], llf=llf,
                       seed=50, flux=flux)
        _, du_gen = gpu_rhs(dgmod, gen)
        _, term = parity_errors(du, du_gen, sc.du_scale())
        assert np.all(term <= TOL64), term


@pytest.mark.parametrize("case", [0, 2, 4])
@pytest.mark.parametrize("flux", ["ranocha", "shima"])
def test_cartesian_fp32(dgmod, case, flux):
    c = CART_CASES[case]
    sc = Scenario(c["nd"], c["nelem"], c["p"], mapping="affine", box=c["box"], ic=c["ic"], llf=True, seed=51,
                  flux=flux)
    _, du = gpu_rhs(dgmod, sc, precision="fp32")
    assert_parity(du, sc, TOL32)


def test_cartesian_entropy_and_conservation(dgmod):
    import torch
    c = CART_CASES[2]
    sc = Scenario(c["nd"], c["nelem"], c["p"], mapping="affine", box=c["box"], ic="random", llf=False, seed=52)
    ctx, du = gpu_rhs(dgmod, sc)
    s, ab = ctx.entropy_rate(torch.from_numpy(sc.u).cuda(), torch.from_numpy(du).cuda())
    assert abs(s) <= 1e-13 * ab, (s, ab)
    tot, ab = orc.integrate(3, c["p"], sc.J, du)
    assert np.all(np.abs(tot) <= 1e-13 * ab)


@pytest.mark.parametrize("scheme", [0, 1])
def test_cartesian_dg_step(dgmod, scheme):
    import torch
    c = CART_CASES[2]
    sc = Scenario(c["nd"], c["nelem"], c["p"], mapping="affine", box=c["box"], ic="smooth", llf=True, seed=53)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    dt = 0.005
    ref = sc.u
    for _ in range(3):
        ctx.step(u, dt, scheme=scheme)
        ref = orc.rk_step(scheme, 3, c["p"], sc.nelem, sc.Ja, sc.J, ref, dt, llf=True)
    err = rel_err_per_var(u.cpu().numpy() - sc.u, ref - sc.u)
    assert np.all(err <= 1e-11), err
