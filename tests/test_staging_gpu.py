"""The two ways the volume kernel stages an element tile (dg_opts.staging): asynchronous copies into shared memory
that overlap the computation of a persistent CTA's tiles (DG_STAGING_PIPELINED: bulk copies for even node counts
per line, per-thread cp.async for odd ones), and direct loads by one CTA per tile (DG_STAGING_DIRECT);
DG_STAGING_AUTO picks the first on meshes with enough tiles per CTA. The pipelined kernel evaluates the same terms
(the lifted surface term starts its line sums, where the direct kernel adds it after them), so it must meet the
FP32 parity bound against the oracle (4e-6 of the term magnitude) and agree with the direct kernel to rounding; the cases cover ragged last tiles, lower-neighbour faces that wrap around the periodic mesh (copied
element by element), tiles that are smaller than the grid and grids that loop over a tile count several times
(both stage buffers reused twice), 2D and 3D, Cartesian and curvilinear meshes, both two-point fluxes, the fused
RK4 and CK45 stage updates, and state arrays that are only 8-byte aligned (the launcher then falls back to direct
loads).
"""
import numpy as np
import pytest

import oracle as orc
from cases import Scenario, assert_parity, parity_errors, rel_err_per_var

pytestmark = pytest.mark.gpu

TOL32 = 4e-6
TOL64 = 1e-12


@pytest.fixture(scope="module")
def dgmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10517_gb300 import build
    build.build()
    from paper_2112_10517_gb300 import dg
    return dg


def rhs_with(dgmod, sc, staging, u=None, precision="fp32"):
    import torch
    ctx = dgmod.DG(precision=precision, staging=staging, **sc.dg_kwargs())
    if u is None:
        u = torch.from_numpy(sc.u).cuda()
    du = ctx.rhs(u)
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    return du.cpu().numpy()


CASES = [
    # nd, nelem, p, mapping, flux, ic
    (3, [3, 3, 3], 1, "sine", "ranocha", "rough"),   # 8 elements per tile: 27 = 3 x 8 + 3, ragged last tile
    (3, [3, 2, 5], 3, "sine", "ranocha", "rough"),   # 2 per tile, n1 = 3: x-neighbours wrap inside tiles
    (3, [2, 2, 3], 5, "sine", "shima", "rough"),     # 1 per tile
    (3, [2, 2, 1], 7, "affine", "ranocha", "rough"),  # Cartesian: no metric copies
    (3, [3, 2, 3], 3, "affine", "shima", "random"),
    (2, [5, 3], 1, "affine", "ranocha", "random"),
    (2, [4, 3], 3, "sine", "shima", "rough"),
    (2, [3, 3], 5, "sine", "ranocha", "rough"),
    (2, [2, 3], 7, "sine", "ranocha", "rough"),
    (3, [1, 3, 2], 1, "sine", "ranocha", "rough"),   # one element along x: every x-neighbour is the element itself
    (3, [3, 1, 1], 3, "affine", "ranocha", "rough"),  # one element along y and z
    (2, [1, 5], 3, "affine", "shima", "random"),
    (3, [1, 1, 1], 5, "sine", "ranocha", "rough"),    # a single element, its own neighbour in every direction
    # odd node counts (even p): per-thread cp.async copies instead of bulk copies
    (3, [3, 3, 2], 2, "sine", "ranocha", "rough"),
    (3, [2, 3, 2], 4, "sine", "shima", "rough"),
    (3, [2, 1, 2], 6, "affine", "ranocha", "rough"),
    (2, [4, 3], 2, "sine", "ranocha", "rough"),
    (2, [3, 2], 4, "affine", "ranocha", "random"),
    (2, [2, 3], 6, "sine", "shima", "rough"),
]


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("nd,nelem,p,mapping,flux,ic", CASES)
def test_both_stagings_match_oracle(dgmod, precision, nd, nelem, p, mapping, flux, ic):
    sc = Scenario(nd, nelem, p, mapping=mapping, ic=ic, llf=True, seed=600 + 10 * nd + p, flux=flux)
    ref, scale = sc.du_ref(), sc.du_scale()
    tol = TOL32 if precision == "fp32" else TOL64
    got = {}
    for staging in ("pipelined", "direct"):
        got[staging] = rhs_with(dgmod, sc, staging, precision=precision)
        print(staging)
        assert_parity(got[staging], ref, tol=tol, scale=scale)  # FP64: also the plain bar (rough, random states)
    _, term = parity_errors(got["pipelined"], got["direct"], scale)
    print("pipelined vs direct term", " ".join("%.1e" % x for x in term))
    assert np.all(term <= tol), term


@pytest.mark.parametrize("nelem,p", [([32, 32, 32], 1), ([16, 16, 16], 3), ([8, 8, 8], 5), ([16, 16, 16], 2),
                                     ([8, 8, 8], 4)])
def test_stagings_agree_on_many_tiles_per_cta(dgmod, nelem, p):
    # thousands of tiles: each persistent CTA loops several times, both stage buffers change parity twice or more
    # (the 16^3 case is also checked against the oracle, element by element, by the FP32 Taylor-Green parity test)
    # (the two kernels add the surface term at different points of the sums: they agree to FP32 rounding of the
    # summed terms, the measure of the parity tests)
    sc = Scenario(3, nelem, p, mapping="sine", ic="tgv", llf=True)
    a = rhs_with(dgmod, sc, "pipelined")
    d = rhs_with(dgmod, sc, "direct")
    _, term = parity_errors(a, d, sc.du_scale())
    print("pipelined vs direct, term-relative per variable", term)
    assert np.all(term <= TOL32), term


@pytest.mark.parametrize("nelem,p", [([16, 16, 16], 3), ([16, 16, 16], 1), ([12, 12, 12], 2)])
def test_fp64_stagings_agree_on_many_tiles_per_cta(dgmod, nelem, p):
    sc = Scenario(3, nelem, p, mapping="sine", ic="tgv", llf=True)
    a = rhs_with(dgmod, sc, "pipelined", precision="fp64")
    d = rhs_with(dgmod, sc, "direct", precision="fp64")
    _, term = parity_errors(a, d, sc.du_scale())
    print("pipelined vs direct (FP64), term-relative per variable", term)
    assert np.all(term <= TOL64), term


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_step_both_stagings(dgmod, scheme, precision):
    # dg_step fuses the stage update into the volume kernel: RK4 stage 0 and every CK45 stage read u as the stage
    # input (the staged input doubles as the update operand), the later RK4 stages stage u and acc separately
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="smooth", llf=True, seed=640, state_fp32=True)
    dt = 0.005
    ref = sc.u
    for _ in range(3):
        ref = orc.rk_step(scheme, 3, 3, sc.nelem, sc.Ja, sc.J, ref, dt, llf=True)
    res = {}
    tol = 2e-5 if precision == "fp32" else 1e-11
    for staging in ("pipelined", "direct"):
        ctx = dgmod.DG(precision=precision, staging=staging, **sc.dg_kwargs())
        u = torch.from_numpy(sc.u).cuda()
        for _ in range(3):
            ctx.step(u, dt, scheme=scheme)
        torch.cuda.synchronize()
        assert ctx.check_status() == dgmod.DG_OK
        res[staging] = u.cpu().numpy()
        err = rel_err_per_var(res[staging] - sc.u, ref - sc.u)
        print(staging, "increment error vs oracle", err)
        assert np.all(err <= tol), (staging, err)
    err = rel_err_per_var(res["pipelined"] - sc.u, res["direct"] - sc.u)
    print("pipelined vs direct increments", err)
    assert np.all(err <= tol), err


def test_eight_byte_aligned_state_falls_back(dgmod):
    # a state at an 8-byte offset cannot be bulk-copied: the launcher takes the direct-load kernel instead
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="rough", llf=True, seed=650)
    n = sc.u.size
    buf = torch.empty(n + 1, dtype=torch.float64, device="cuda")
    u_off = buf[1:].view(sc.u.shape)
    u_off.copy_(torch.from_numpy(sc.u))
    assert u_off.data_ptr() % 16 == 8
    off = rhs_with(dgmod, sc, "pipelined", u=u_off)
    plain, term = parity_errors(off, sc.du_ref(), sc.du_scale())
    assert np.all(term <= TOL32), (term, plain)
    direct = rhs_with(dgmod, sc, "direct")
    assert np.array_equal(off, direct)


def test_auto_selects_by_tiles_per_cta(dgmod):
    # DG_STAGING_AUTO runs the pipelined kernel only with at least 4 tiles per resident CTA: a small mesh gets the
    # per-tile kernel, the 32^3 p = 3 mesh (16,384 tiles of 2 elements) the pipelined one; both bit for bit
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="rough", llf=True, seed=660)
    assert np.array_equal(rhs_with(dgmod, sc, "auto"), rhs_with(dgmod, sc, "direct"))
    sc = Scenario(3, [32, 32, 32], 3, mapping="sine", ic="tgv", llf=True)
    auto, pipe = rhs_with(dgmod, sc, "auto"), rhs_with(dgmod, sc, "pipelined")
    assert np.array_equal(auto, pipe)
    # FP32 at p = 2 stays on the per-tile kernel (measured faster there) even with many tiles; FP64 does not
    sc = Scenario(3, [24, 24, 24], 2, mapping="sine", ic="tgv", llf=True)
    assert np.array_equal(rhs_with(dgmod, sc, "auto"), rhs_with(dgmod, sc, "direct"))
    assert np.array_equal(rhs_with(dgmod, sc, "auto", precision="fp64"),
                          rhs_with(dgmod, sc, "pipelined", precision="fp64"))


def test_device_wait_timeout_is_reported_and_the_context_recovers(dgmod):
    # the pipelined kernel's waits on its own copies are bounded; a wait that runs out raises the timeout flag.
    # The self-test waits, with the same bounded wait, on an mbarrier nothing completes (no fault, no hang)
    import time
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="rough", llf=True, seed=670)
    ctx = dgmod.DG(precision="fp32", staging="pipelined", **sc.dg_kwargs())
    t0 = time.time()
    assert dgmod.dg_selftest_wait_timeout(ctx.ctx, None) == dgmod.DG_OK
    assert ctx.check_status() == dgmod.DG_ERR_TIMEOUT
    elapsed = time.time() - t0
    assert 0.1 < elapsed < 30.0, elapsed
    assert ctx.check_status() == dgmod.DG_OK  # read and cleared
    du = ctx.rhs(torch.from_numpy(sc.u).cuda())
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    _, term = parity_errors(du.cpu().numpy(), sc.du_ref(), sc.du_scale())
    assert np.all(term <= TOL32), term
