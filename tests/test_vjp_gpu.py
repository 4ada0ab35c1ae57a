"""dg_vjp, the hand-written adjoint of the RHS: ubar = J(u)^T gbar with J = d RHS/du.

Checked against the oracle's forward-mode JVP (oracle.c compiled with dual numbers) by the dot-product identity
<gbar, J delta> = <J^T gbar, delta>, against central finite differences of the GPU forward RHS (eps = 1e-6) on
seeded directions, and entrywise against the full Jacobian on a tiny mesh.
"""
import numpy as np
import pytest

import oracle as orc
from cases import Scenario
from paper_2112_10517_gb300 import inputs

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


def vjp(dgmod, sc, gbar):
    import torch
    ctx = dgmod.DG(**sc.dg_kwargs())
    ub = ctx.vjp(torch.from_numpy(sc.u).cuda(), torch.from_numpy(gbar).cuda()).cpu().numpy()
    assert ctx.check_status() == dgmod.DG_OK
    return ctx, ub


def dot_test(dgmod, sc, seed):
    gbar = inputs.perturbation(sc.u.shape, seed)
    delta = inputs.perturbation(sc.u.shape, seed + 1) * np.abs(sc.u)
    _, ub = vjp(dgmod, sc, gbar)
    _, jd = orc.jvp(sc.nd, sc.p, sc.nelem, sc.Ja, sc.J, sc.u, delta, llf=sc.llf)
    lhs = np.sum(gbar * jd)
    rhs = np.sum(ub * delta)
    scale = np.sum(np.abs(gbar * jd))
    return abs(lhs - rhs) / scale


@pytest.mark.parametrize("nd,nelem,p", [(3, [8, 8, 8], 4)])
def test_vjp_dot_product_8cubed_p4(dgmod, nd, nelem, p):
    # the differentiation workload: 3D curvilinear 8^3 elements, polydeg 4, FP64, seeded smooth random state
    sc = Scenario(nd, nelem, p, mapping="sine", ic="smooth", llf=True, seed=40)
    assert dot_test(dgmod, sc, seed=41) <= 1e-12


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("llf", [False, True])
def test_vjp_dot_product_every_degree(dgmod, p, llf):
    for nd, nelem in ((3, [2, 3, 2]), (2, [3, 4])):
        sc = Scenario(nd, nelem, p, mapping="sine", ic="rough", llf=llf, seed=50 + p)
        assert dot_test(dgmod, sc, seed=60 + p) <= 1e-12, nd


def test_vjp_dot_product_log_branch_and_twisted_mesh(dgmod):
    sc = Scenario(3, [2, 2, 3], 3, mapping="twisted", ic="random", llf=True, seed=70)
    assert dot_test(dgmod, sc, seed=71) <= 1e-12
    sc = Scenario(3, [4, 4, 4], 3, mapping="sine", ic="tgv", llf=True)
    assert dot_test(dgmod, sc, seed=72) <= 1e-12


def test_vjp_central_finite_differences(dgmod):
    # central differences of the GPU forward RHS, eps = 1e-6, 8 seeded directions, 8^3 p = 4
    import torch
    sc = Scenario(3, [8, 8, 8], 4, mapping="sine", ic="smooth", llf=True, seed=80)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    for k in range(8):
        gbar = torch.from_numpy(inputs.perturbation(sc.u.shape, 100 + k)).cuda()
        delta = torch.from_numpy(inputs.perturbation(sc.u.shape, 200 + k) * np.abs(sc.u)).cuda()
        ub = ctx.vjp(u, gbar)
        eps = 1e-6
        fd = (ctx.rhs(u + eps * delta) - ctx.rhs(u - eps * delta)) / (2 * eps)
        lhs = float(torch.sum(gbar * fd))
        rhs = float(torch.sum(ub * delta))
        scale = float(torch.sum(torch.abs(gbar * fd)))
        assert abs(lhs - rhs) <= 1e-7 * scale, (k, lhs, rhs)


def test_vjp_full_jacobian_2cubed_p2(dgmod):
    # every column of J by dual numbers (oracle), every row of J^T by dg_vjp, compared entrywise
    import torch
    sc = Scenario(3, [2, 2, 2], 2, mapping="sine", ic="rough", llf=True, seed=90)
    ctx = dgmod.DG(**sc.dg_kwargs())
    n = sc.u.size
    Jref = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        _, jd = orc.jvp(sc.nd, sc.p, sc.nelem, sc.Ja, sc.J, sc.u, e.reshape(sc.u.shape), llf=True)
        Jref[:, j] = jd.ravel()
    u = torch.from_numpy(sc.u).cuda()
    Jrows = np.zeros((n, n))  # row i of J = J^T e_i from dg_vjp
    g = torch.zeros(n, dtype=torch.float64, device="cuda")
    for i in range(n):
        g.zero_()
        g[i] = 1.0
        Jrows[i] = ctx.vjp(u, g.view(sc.u.shape)).cpu().numpy().ravel()
    np.testing.assert_allclose(Jrows, Jref, rtol=0, atol=1e-12 * np.max(np.abs(Jref)))


def test_autograd_function(dgmod):
    import torch
    sc = Scenario(3, [2, 3, 2], 3, mapping="sine", ic="smooth", llf=True, seed=95)
    ctx = dgmod.DG(**sc.dg_kwargs())
    DGRhs = dgmod.rhs_function()
    u = torch.from_numpy(sc.u).cuda().requires_grad_(True)
    w = torch.from_numpy(inputs.perturbation(sc.u.shape, 96)).cuda()
    loss = torch.sum(DGRhs.apply(ctx, u) * w)
    loss.backward()
    ref = ctx.vjp(u.detach(), w)
    torch.testing.assert_close(u.grad, ref, rtol=0, atol=0)


def test_vjp_rejects_fp32_and_aliasing(dgmod):
    import ctypes
    import torch
    sc = Scenario(3, [2, 2, 2], 3, mapping="sine", ic="smooth", llf=True, seed=97)
    ctx32 = dgmod.DG(precision="fp32", **sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    with pytest.raises(dgmod.DGError) as ei:
        ctx32.vjp(u, u.clone())
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    ctx = dgmod.DG(**sc.dg_kwargs())
    g = u.clone()
    assert dgmod.dg_vjp(ctx.ctx, ctypes.c_void_p(u.data_ptr()), ctypes.c_void_p(g.data_ptr()),
                        ctypes.c_void_p(g.data_ptr()), None) == dgmod.DG_ERR_ARG
