"""Parity of the library's Legendre-Gauss collocation scheme with entropy projection (Sec. 6; dg_opts.nodes =
DG_NODES_GAUSS) with the oracle's dense hybridized formulation (oracle/gauss.c), element by element, plus the
properties the scheme is built for, measured on the GPU result.

The library evaluates the hybridized operators line by line (each pair of a line once, each node-face-point pair
once); the oracle builds the dense multi-dimensional operators. Both are exact rewrites of the same sums, so they
agree to rounding: 1e-12 of max |du| per variable on the smooth-plus-noise states used here (their RHS has no
large cancellation: the terms are within a factor ~10 of the result).
"""
import math

import numpy as np
import pytest

import oracle as orc
from cases import rel_err_per_var
from paper_2112_10517_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def dgmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10517_gb300 import build
    build.build()
    from paper_2112_10517_gb300 import dg
    return dg


def make(dgmod, nd, nelem, p, box=None, llf=False, ic="rough", seed=0):
    lo, hi = box if box is not None else ([-1.0] * nd, [1.0] * nd)
    ctx = dgmod.DG(nd, nelem, p, lo=lo, hi=hi, mapping="affine", surface="llf" if llf else "ec", nodes="gauss")
    xyz = orc.gauss_coords(nd, nelem, lo, hi, p)
    L = [h - l for l, h in zip(lo, hi)]
    if ic == "rough":
        u = inputs.smooth_random(xyz, seed=seed, lengths=L) + 0.05 * inputs.random_state(xyz, seed + 1)
    elif ic == "smooth":
        u = inputs.smooth_random(xyz, seed=seed, lengths=L)
    elif ic == "free_stream":
        u = inputs.free_stream(xyz)
    elif ic == "vortex":
        u = inputs.isentropic_vortex(xyz, eps=5.0)
    else:
        raise ValueError(ic)
    return ctx, lo, hi, xyz, u


def gpu_rhs(dgmod, ctx, u):
    import torch
    du = ctx.rhs(torch.from_numpy(u).cuda())
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    return du.cpu().numpy()


def test_gauss_node_coordinates(dgmod):
    for nd, nelem, p in ((2, [3, 4], 3), (3, [2, 3, 2], 5)):
        lo, hi = [-1.0, 0.0, 2.0][:nd], [1.0, 3.0, 2.5][:nd]
        ctx = dgmod.DG(nd, nelem, p, lo=lo, hi=hi, mapping="affine", nodes="gauss")
        np.testing.assert_allclose(ctx.node_coords(), orc.gauss_coords(nd, nelem, lo, hi, p), rtol=0, atol=1e-14)


@pytest.mark.parametrize("p,nelem", [(1, [3, 4, 3]), (2, [3, 3, 3]), (3, [4, 3, 2]), (4, [2, 3, 3]),
                                     (5, [2, 2, 3]), (6, [2, 1, 3]), (7, [2, 2, 1])])
@pytest.mark.parametrize("llf", [False, True])
def test_gauss_rhs_3d_every_degree(dgmod, p, nelem, llf):
    ctx, lo, hi, xyz, u = make(dgmod, 3, nelem, p, llf=llf, seed=10 + p)
    du = gpu_rhs(dgmod, ctx, u)
    ref = orc.gauss_rhs(3, p, nelem, lo, hi, u, llf=llf)
    err = rel_err_per_var(du, ref)
    print("gauss 3d p=%d llf=%d err %s" % (p, llf, " ".join("%.1e" % e for e in err)))
    assert np.all(err <= TOL), err


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("llf", [False, True])
def test_gauss_rhs_2d_every_degree(dgmod, p, llf):
    ctx, lo, hi, xyz, u = make(dgmod, 2, [3, 4], p, llf=llf, seed=20 + p)
    du = gpu_rhs(dgmod, ctx, u)
    ref = orc.gauss_rhs(2, p, [3, 4], lo, hi, u, llf=llf)
    err = rel_err_per_var(du, ref)
    assert np.all(err <= TOL), err


def test_gauss_rhs_anisotropic_box_and_vortex(dgmod):
    box = ([-5.0, -4.0, -3.0], [5.0, 6.0, 3.0])
    ctx, lo, hi, xyz, u = make(dgmod, 3, [4, 3, 5], 3, box=box, llf=True, ic="vortex")
    du = gpu_rhs(dgmod, ctx, u)
    ref = orc.gauss_rhs(3, 3, [4, 3, 5], lo, hi, u, llf=True)
    assert np.all(rel_err_per_var(du, ref) <= TOL)


def test_gauss_free_stream_conservation_entropy(dgmod):
    import torch
    ctx, lo, hi, xyz, u = make(dgmod, 3, [3, 2, 3], 3, ic="free_stream")
    assert np.abs(gpu_rhs(dgmod, ctx, u)).max() <= 1e-13
    _, wg = orc.gauss(3)
    W = wg.copy()
    for _ in range(2):
        W = np.kron(wg, W)
    for llf in (False, True):
        ctx, lo, hi, xyz, u = make(dgmod, 3, [3, 2, 3], 3, llf=llf, seed=31)
        du = gpu_rhs(dgmod, ctx, u)
        tot = np.einsum("evi,i->v", du, W)
        ab = np.einsum("evi,i->v", np.abs(du), W)
        assert np.all(np.abs(tot) <= 1e-13 * ab)
        s, sab = ctx.entropy_rate(torch.from_numpy(u).cuda(), torch.from_numpy(du).cuda())
        if llf:
            assert s < -1e-6 * sab
        else:
            assert abs(s) <= 1e-13 * sab, (s, sab)


@pytest.mark.parametrize("scheme", [0, 1])
def test_gauss_dg_step(dgmod, scheme):
    # the library's fused stage updates against the same Runge-Kutta schemes applied to the oracle's RHS
    import torch
    nd, nelem, p = 3, [3, 2, 3], 3
    ctx, lo, hi, xyz, u0 = make(dgmod, nd, nelem, p, llf=True, ic="smooth", seed=41)
    u = torch.from_numpy(u0).cuda()
    dt = 0.002
    f = lambda v: orc.gauss_rhs(nd, p, nelem, lo, hi, v, llf=True)
    ref = u0.copy()
    A, B = orc.ck45_coefficients()
    for _ in range(3):
        ctx.step(u, dt, scheme=scheme)
        if scheme == 0:
            k1 = f(ref)
            k2 = f(ref + 0.5 * dt * k1)
            k3 = f(ref + 0.5 * dt * k2)
            k4 = f(ref + dt * k3)
            ref = ref + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
        else:
            K = np.zeros_like(ref)
            for s in range(5):
                K = A[s] * K + dt * f(ref)
                ref = ref + B[s] * K
    assert ctx.check_status() == dgmod.DG_OK
    err = rel_err_per_var(u.cpu().numpy() - u0, ref - u0)
    assert np.all(err <= 1e-11), err


def test_gauss_unsupported_combinations(dgmod):
    for kw in (dict(mapping="sine", amp=0.1), dict(precision="fp32"), dict(flux="shima"),
               dict(precompute_logs=True)):
        args = dict(mapping="affine")
        args.update(kw)
        with pytest.raises(dgmod.DGError) as ei:
            dgmod.DG(3, [2, 2, 2], 3, nodes="gauss", **args)
        assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED, kw
    import torch
    ctx, lo, hi, xyz, u = make(dgmod, 3, [2, 2, 2], 3)
    ut = torch.from_numpy(u).cuda()
    with pytest.raises(dgmod.DGError) as ei:
        ctx.vjp(ut, ut.clone())
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    with pytest.raises(dgmod.DGError) as ei:
        dgmod.DGBatch([ctx], [ut], [torch.empty_like(ut)])
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED


def test_gauss_inadmissible_face_state_is_flagged(dgmod):
    # independent random nodal states: interpolating w(u) to the faces overshoots (|l_k(+-1)| > 1) and rho/p < 0
    # can result; the projection flags the state instead of producing a face state
    import torch
    nd, nelem, p = 3, [2, 2, 2], 3
    ctx = dgmod.DG(nd, nelem, p, mapping="affine", nodes="gauss")
    xyz = orc.gauss_coords(nd, nelem, [-1.0] * 3, [1.0] * 3, p)
    rng = np.random.Generator(np.random.PCG64(3))
    rho = rng.uniform(0.05, 3.0, xyz[:, 0].shape)
    pr = rng.uniform(0.05, 3.0, xyz[:, 0].shape)
    u = inputs.prim_to_cons(rho, [0.0 * rho] * 3, pr)
    _, w = orc.entropy(np.ascontiguousarray(np.moveaxis(u, 1, 2)), nd)
    x, _ = orc.gauss(p)
    lp = orc.lagrange_at(p, x, 1.0)
    # the test state is chosen so that some face value of -w_E = rho/p is negative
    wE = np.moveaxis(w, 2, 1)[:, 4].reshape(-1, 4, 4, 4)  # [E, i3, i2, i1]
    assert np.any(np.einsum("k,eabk->eab", lp, wE) > 0)
    ctx.rhs(torch.from_numpy(u).cuda())
    assert ctx.check_status() == dgmod.DG_ERR_NONPHYSICAL
