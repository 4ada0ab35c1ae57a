"""Parity of the CUDA RHS (through the C ABI) with the CPU oracle, element by element, plus the properties
the paper fixes, measured on the GPU result.

The oracle evaluates the strong form with all ordered pairs and Cartesian fluxes; the library evaluates
the flux-differencing operator Dt with each pair once and directional fluxes (Sec. 2.1-2.3). The two are
algebraically identical, so they agree to round-off.

FP64 tolerances, per variable, normwise (cases.assert_parity):
- 1e-12 relative to the magnitude of the terms the RHS sums, max_i (1/J_i) sum |terms_i| (the oracle's scale
  mode), in every case. Rounding of any FP64 evaluation is proportional to that magnitude.
- plain relative, max|du_gpu - du_ref| / max|du_ref| <= max(1e-12, 1e-13 kappa), for every variable whose
  cancellation factor kappa = max scale / max|du_ref| is at most 1e3 (every state here but the Taylor-Green
  vortex): 1e-12 where kappa <= 10, else a term-relative bar ten times stricter than the first. The Mach 0.1
  Taylor-Green vortex sums pressure terms 1e3 .. 3e4 times larger than its RHS, so the plain relative difference of
  two correct FP64 evaluations is ~1e-8 there (the FP64 oracle is 3e-8 from a long-double build of itself at
  16^3); those variables are held to the term-relative bar.
"""
import math

import numpy as np
import pytest

import oracle as orc
from cases import TOL64, Scenario, assert_parity, parity_errors, rel_err_per_var

pytestmark = pytest.mark.gpu


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
    u = torch.from_numpy(sc.u).cuda()
    du = ctx.rhs(u)
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    return ctx, du.cpu().numpy()


# ------------------------------------------------------------------------------------------------
# Geometry parity: the library's node coordinates and metric terms against the oracle's
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd,nelem,p,mapping", [(2, [3, 4], 3, "sine"), (3, [2, 3, 2], 4, "sine"),
                                                 (3, [2, 2, 2], 3, "twisted"), (2, [8, 8], 3, "affine")])
def test_geometry_matches_oracle(dgmod, nd, nelem, p, mapping):
    sc = Scenario(nd, nelem, p, mapping=mapping)
    ctx = dgmod.DG(**sc.dg_kwargs())
    np.testing.assert_allclose(ctx.node_coords(), sc.xyz, rtol=0, atol=1e-14)
    Ja, J = ctx.metrics()
    np.testing.assert_allclose(Ja, sc.Ja, rtol=0, atol=1e-13 * np.max(np.abs(sc.Ja)))
    np.testing.assert_allclose(J, sc.J, rtol=1e-13)


# ------------------------------------------------------------------------------------------------
# RHS parity, FP64
# ------------------------------------------------------------------------------------------------

def test_rhs_2d_cartesian_noisy_sine_8x8_p3(dgmod):
    # 2D Euler, [-1,1]^2, 8x8 affine quads, p = 3, rho = 1 + 0.1 sin(pi x) sin(pi y), v = (0.1, 0.2), p = 1
    # plus seeded uniform(-1e-2, 1e-2) noise on the primitives; Ranocha volume flux, Ranocha + LLF surface
    sc = Scenario(2, [8, 8], 3, mapping="affine", box=([-1.0, -1.0], [1.0, 1.0]), ic="noisy_sine", llf=True)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc, plain_tol=1e-12)  # both bars (kappa 9 .. 64)


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("llf", [False, True])
def test_rhs_2d_curved_every_degree(dgmod, p, llf):
    sc = Scenario(2, [5, 3], p, mapping="sine", ic="rough", llf=llf, seed=p)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc)


@pytest.mark.parametrize("p,nelem", [(1, [3, 4, 5]), (2, [3, 3, 3]), (3, [3, 2, 5]), (4, [2, 3, 3]),
                                     (5, [2, 2, 3]), (6, [2, 1, 3]), (7, [2, 2, 1])])
@pytest.mark.parametrize("llf", [False, True])
def test_rhs_3d_curved_every_degree(dgmod, p, nelem, llf):
    # element counts are not multiples of the elements per CTA: ragged last block
    sc = Scenario(3, nelem, p, mapping="sine", ic="rough", llf=llf, seed=10 + p)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc)


@pytest.mark.parametrize("nd,nelem,p", [(3, [3, 2, 3], 3), (2, [4, 5], 4)])
def test_rhs_twisted_mesh_from_node_coordinates(dgmod, nd, nelem, p):
    sc = Scenario(nd, nelem, p, mapping="twisted", ic="rough", llf=True, seed=3)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc)


def test_rhs_random_states_take_the_log_branch(dgmod):
    # independent random nodal states: nearly every pair takes the log branch of Algorithms 2 and 3
    sc = Scenario(3, [2, 3, 2], 3, mapping="sine", ic="random", llf=True, seed=7)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc)


def test_rhs_isentropic_vortex_paper_workload(dgmod):
    # Sec. 4.1: isentropic vortex with eps = 20 on [-5,5]^3, 8 elements per direction, p = 3
    sc = Scenario(3, [8, 8, 8], 3, mapping="affine", box=([-5.0] * 3, [5.0] * 3), ic="vortex", llf=True)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc)


@pytest.mark.parametrize("nd,nelem", [(3, [1, 1, 1]), (2, [1, 1]), (3, [1, 4, 1]), (2, [1, 7])])
def test_rhs_single_element_periodic_self_coupling(dgmod, nd, nelem):
    # an element that is its own neighbour in one or more directions
    sc = Scenario(nd, nelem, 3, mapping="sine", ic="rough", llf=True, seed=5)
    _, du = gpu_rhs(dgmod, sc)
    assert_parity(du, sc)


def test_rhs_tgv_16cubed_p3_full_size(dgmod):
    # the 3D curvilinear Taylor-Green workload at full size: 16^3 elements, p = 3, 262,144 DOF, Mach 0.1
    # (kappa 1e3 .. 3e4: the term-relative bar; assert_parity skips the plain bar for those variables)
    sc = Scenario(3, [16, 16, 16], 3, mapping="sine", ic="tgv", llf=True)
    _, du = gpu_rhs(dgmod, sc)
    _, _, kappa = assert_parity(du, sc)
    assert np.all(kappa > 1e3)  # the reason the plain bar does not apply here


def test_rhs_64cubed_p3_sampled_elements(dgmod):
    # 64^3 elements, p = 3 (16.8M DOF): the oracle computes a seeded sample of elements
    import torch
    nelem = [64, 64, 64]
    p = 3
    xyz = orc.coords(3, nelem, [-math.pi] * 3, [math.pi] * 3, p, mapping=1, amp=0.1)
    from paper_2112_10517_gb300 import inputs
    u = inputs.taylor_green(xyz)
    Ja, J = orc.metrics(3, p, xyz)
    ctx = dgmod.DG(3, nelem, p, lo=[-math.pi] * 3, hi=[math.pi] * 3, mapping="sine", amp=0.1, surface="llf")
    du = ctx.rhs(torch.from_numpy(u).cuda()).cpu().numpy()
    rng = np.random.Generator(np.random.PCG64(0))
    sample = np.unique(np.concatenate([[0, 1, 63, 64 * 64 - 1, u.shape[0] - 1], rng.integers(0, u.shape[0], 60)]))
    ref = np.zeros((len(sample),) + u.shape[1:])
    scale = np.zeros_like(ref)
    for s, e in enumerate(sample):
        ref[s] = orc.rhs(3, p, nelem, Ja, J, u, llf=True, elem_range=(int(e), int(e) + 1))[0]
        scale[s] = orc.rhs(3, p, nelem, Ja, J, u, llf=True, elem_range=(int(e), int(e) + 1), scale=True)[0]
    assert_parity(du[sample], ref, scale=scale)  # low Mach: kappa > 1e3, the term-relative bar


# ------------------------------------------------------------------------------------------------
# Properties of the GPU result that the paper fixes
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd,nelem,p", [(3, [3, 2, 3], 3), (2, [4, 3], 5)])
def test_free_stream_preserved_on_gpu(dgmod, nd, nelem, p):
    # curl-form metrics satisfy the discrete metric identities (Sec. 2.3): a constant state stays constant up
    # to rounding of the terms (pressure times metric) that cancel
    for mapping in ("sine", "twisted"):
        sc = Scenario(nd, nelem, p, mapping=mapping, ic="free_stream", llf=True)
        _, du = gpu_rhs(dgmod, sc)
        scale = sc.du_scale()
        for c in range(nd + 2):
            assert np.max(np.abs(du[:, c])) <= 1e-13 * np.max(scale[:, c]), c



@pytest.mark.parametrize("nd,nelem,p", [(3, [3, 2, 3], 3), (2, [4, 3], 4)])
def test_entropy_conservation_on_gpu(dgmod, nd, nelem, p):
    import torch
    sc = Scenario(nd, nelem, p, mapping="sine", ic="random", llf=False, seed=11)
    ctx, du = gpu_rhs(dgmod, sc)
    s_gpu, ab = ctx.entropy_rate(torch.from_numpy(sc.u).cuda(), torch.from_numpy(du).cuda())
    s_ref, ab_ref = orc.entropy_rate(nd, p, sc.J, sc.u, du)
    assert abs(s_gpu) <= 1e-13 * ab, (s_gpu, ab)
    assert abs(s_gpu - s_ref) <= 1e-13 * ab_ref
    assert abs(ab - ab_ref) <= 1e-12 * ab_ref
    # with LLF the scheme dissipates entropy
    sc = Scenario(nd, nelem, p, mapping="sine", ic="random", llf=True, seed=11)
    ctx, du = gpu_rhs(dgmod, sc)
    s_gpu, ab = ctx.entropy_rate(torch.from_numpy(sc.u).cuda(), torch.from_numpy(du).cuda())
    assert s_gpu < -1e-6 * ab


def test_conservation_on_gpu(dgmod):
    sc = Scenario(3, [3, 3, 2], 4, mapping="twisted", ic="rough", llf=True, seed=12)
    _, du = gpu_rhs(dgmod, sc)
    tot, ab = orc.integrate(3, 4, sc.J, du)
    assert np.all(np.abs(tot) <= 1e-13 * ab)


def test_pressure_equilibrium_on_gpu(dgmod):
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="pressure_eq", llf=True, seed=13)
    _, du = gpu_rhs(dgmod, sc)
    v = [0.1, -0.2, 0.3]
    scale = np.max(np.abs(du[:, 0]))
    for j in range(3):
        np.testing.assert_allclose(du[:, 1 + j], v[j] * du[:, 0], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(du[:, 4], 0.5 * np.dot(v, v) * du[:, 0], rtol=0, atol=1e-12 * scale)


# ------------------------------------------------------------------------------------------------
# Time stepping (dg_step) against the oracle's time steps
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("scheme", [0, 1])
def test_dg_step_matches_oracle(dgmod, scheme):
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="smooth", llf=True, seed=14)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    dt = 0.01
    for _ in range(3):
        ctx.step(u, dt, scheme=scheme)
    ref = sc.u
    for _ in range(3):
        ref = orc.rk_step(scheme, 3, 3, sc.nelem, sc.Ja, sc.J, ref, dt, llf=True)
    got = u.cpu().numpy()
    # the step changes u by O(dt du); compare the increments
    err = rel_err_per_var(got - sc.u, ref - sc.u)
    assert np.all(err <= 1e-11), err


# ------------------------------------------------------------------------------------------------
# Errors: argument errors and the non-physical flag (host-detected or flagged by the kernel; no fault)
# ------------------------------------------------------------------------------------------------

def test_nonphysical_state_is_flagged(dgmod):
    import torch
    sc = Scenario(3, [2, 2, 2], 2, mapping="sine", ic="smooth", llf=True)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    assert ctx.check_status() == dgmod.DG_OK
    bad = u.clone()
    bad[1, 0, 5] = -1.0  # negative density at one node
    ctx.rhs(bad)
    assert ctx.check_status() == dgmod.DG_ERR_NONPHYSICAL
    assert ctx.check_status() == dgmod.DG_OK  # the flag was cleared
    ctx.rhs(u)
    assert ctx.check_status() == dgmod.DG_OK


def test_argument_errors_on_gpu(dgmod):
    import ctypes
    import torch
    sc = Scenario(2, [2, 2], 2, mapping="affine", ic="smooth")
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    p = ctypes.c_void_p(u.data_ptr())
    assert dgmod.dg_rhs(ctx.ctx, p, p, 0.0, None) == dgmod.DG_ERR_ARG  # aliasing u and du
    assert dgmod.dg_rhs(ctx.ctx, p, None, 0.0, None) == dgmod.DG_ERR_ARG
    assert dgmod.dg_step(ctx.ctx, p, p, 0.0, 0.1, 7, None) == dgmod.DG_ERR_ARG  # unknown scheme
    with pytest.raises(ValueError):
        ctx.rhs(u[:, :, :3].contiguous())


# ------------------------------------------------------------------------------------------------
# FP32 flux mode: per-field error against the FP64 oracle. FP32 fluxes and line sums round at 2^-24
# relative to the terms they sum: the bound is 4e-6 of the term magnitude (about 60 ulp), per variable.
# ------------------------------------------------------------------------------------------------
TOL32 = 4e-6


@pytest.mark.parametrize("p,nelem", [(1, [3, 4, 5]), (2, [3, 3, 3]), (3, [3, 2, 5]), (4, [2, 3, 3]),
                                     (5, [2, 2, 3]), (6, [2, 1, 3]), (7, [2, 2, 1])])
def test_rhs_fp32_mode_3d_every_degree(dgmod, p, nelem):
    sc = Scenario(3, nelem, p, mapping="sine", ic="rough", llf=True, seed=20 + p)
    _, du = gpu_rhs(dgmod, sc, precision="fp32")
    assert_parity(du, sc, tol=TOL32)


def test_rhs_fp32_mode_2d(dgmod):
    sc = Scenario(2, [8, 8], 3, mapping="affine", box=([-1.0, -1.0], [1.0, 1.0]), ic="noisy_sine", llf=True)
    _, du = gpu_rhs(dgmod, sc, precision="fp32")
    assert_parity(du, sc, tol=TOL32)


@pytest.mark.parametrize("nelem,p", [([16, 16, 16], 3), ([4, 4, 4], 7)])
def test_rhs_fp32_mode_tgv(dgmod, nelem, p):
    sc = Scenario(3, nelem, p, mapping="sine", ic="tgv", llf=True)
    _, du = gpu_rhs(dgmod, sc, precision="fp32")
    assert_parity(du, sc, tol=TOL32)


def test_rhs_fp32_mode_random_states_log_branch(dgmod):
    sc = Scenario(3, [2, 3, 2], 3, mapping="sine", ic="random", llf=True, seed=7)
    _, du = gpu_rhs(dgmod, sc, precision="fp32")
    assert_parity(du, sc, tol=TOL32)
