"""The FP64 pipelined volume kernel's counter schedule. Where every resident CTA has at least two full tiles and the
launcher predicts an earlier end for it, the CTAs take their tiles after the first from a per-context counter, the
mesh's last round in half tiles, and the last CTA to finish resets the counter for the next launch. The RHS must meet
the oracle's parity bound, agree with the direct (one CTA per tile) kernel to rounding, and stay the same bit for bit
over repeated calls, fused stage updates and graph replays: a counter left non-zero would make the next launch skip
tiles. The p = 3 sizes are ones for which the launcher takes the counter on a GPU with 152 SMs and two resident
CTAs per SM (16 x 16 x 17: 1,088 tiles, at most 8 per SM round-robin against 14.3 half tiles per SM; 17^3: an
element count that is odd, so the last half tile holds one element; a partition of 12 element layers); the 16^3
mesh, where round-robin is kept, and the FP32 kernel, which always takes round-robin, check that those paths are
unchanged; p = 2 (odd node count) copies per thread."""

import numpy as np
import pytest

from cases import Scenario, assert_parity, parity_errors

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


CASES = [
    # precision, nelem, p
    ("fp64", [16, 16, 17], 3),
    ("fp64", [17, 17, 17], 3),
    ("fp64", [16, 16, 16], 3),
    ("fp32", [16, 16, 16], 3),
    ("fp64", [24, 24, 24], 2),
]


@pytest.mark.parametrize("precision,nelem,p", CASES)
def test_dynamic_tiles_match_oracle_and_direct_kernel_and_repeat(dgmod, precision, nelem, p):
    import torch
    sc = Scenario(3, nelem, p, mapping="sine", ic="smooth", llf=True, seed=90 + p)
    pipe = dgmod.DG(precision=precision, staging="pipelined", **sc.dg_kwargs())
    direct = dgmod.DG(precision=precision, staging="direct", **sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    first = pipe.rhs(u).cpu().numpy()
    for _ in range(3):  # consecutive launches on one stream, each needing the counter reset by the one before
        again = pipe.rhs(u).cpu().numpy()
        np.testing.assert_array_equal(again, first)
    assert pipe.check_status() == dgmod.DG_OK
    ref, scale = sc.du_ref(), sc.du_scale()
    tol = TOL32 if precision == "fp32" else TOL64
    assert_parity(first, ref, tol=tol, scale=scale)
    other = direct.rhs(u).cpu().numpy()
    _, term = parity_errors(first, other, scale)  # the surface term enters the sums at different points
    assert np.all(term <= tol), term


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_dynamic_tiles_in_steps_and_graph_replays(dgmod, precision):
    import torch
    sc = Scenario(3, [16, 16, 17], 3, mapping="sine", ic="smooth", llf=True, seed=95)
    ctx = dgmod.DG(precision=precision, staging="pipelined", **sc.dg_kwargs())
    u0 = torch.from_numpy(sc.u).cuda()
    scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device="cuda")
    dt = 1e-3
    # eager: rhs, two steps, rhs (the volume kernel with and without the fused update, alternating)
    u = u0.clone()
    du_a = ctx.rhs(u).clone()
    for _ in range(2):
        ctx.step(u, dt, scheme=0, scratch=scratch)
    du_b = ctx.rhs(u).clone()
    torch.cuda.synchronize()
    eager = (du_a.cpu().numpy(), u.cpu().numpy(), du_b.cpu().numpy())
    # the same sequence captured once and replayed twice
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    ug = u0.clone()
    da, db = torch.empty_like(u0), torch.empty_like(u0)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        ctx.rhs(ug, da, stream=side)
        for _ in range(2):
            ctx.step(ug, dt, scheme=0, scratch=scratch, stream=side)
        ctx.rhs(ug, db, stream=side)
    for _ in range(2):
        ug.copy_(u0)
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(da.cpu().numpy(), eager[0])
        np.testing.assert_array_equal(ug.cpu().numpy(), eager[1])
        np.testing.assert_array_equal(db.cpu().numpy(), eager[2])
    assert ctx.check_status() == dgmod.DG_OK


def test_dynamic_tiles_on_a_partition_equal_whole_mesh(dgmod):
    import torch
    from paper_2112_10517_gb300 import partition
    sc = Scenario(3, [16, 16, 24], 3, mapping="sine", ic="smooth", llf=True, seed=96)
    whole = dgmod.DG(staging="pipelined", **sc.dg_kwargs())
    ref = whole.rhs(torch.from_numpy(sc.u).cuda()).cpu().numpy()
    layer = 16 * 16
    slabs = []
    for b, e in partition.slab_plan(24, 2):  # 12 layers each: 3,072 elements from the ghost layer on
        ctx = dgmod.DG(staging="pipelined", part=(b, e), **sc.dg_kwargs())
        u = torch.full(ctx.shape, float("nan"), dtype=torch.float64, device="cuda")
        u[layer:] = torch.from_numpy(sc.u[b * layer:e * layer]).cuda()
        slabs.append((ctx, u, ctx.halo_buffers(), (b, e)))
    for ctx, u, bufs, _ in slabs:
        ctx.pack(u, bufs[0], bufs[1])
    partition.exchange_local([s[2] for s in slabs])
    for ctx, u, bufs, _ in slabs:
        ctx.unpack(u, bufs[2], bufs[3])
    for ctx, u, _, (b, e) in slabs:
        for _ in range(2):
            du = torch.full_like(u, float("nan"))
            ctx.rhs(u, du)
            got = du.cpu().numpy()
            np.testing.assert_array_equal(got[layer:], ref[b * layer:e * layer])
            assert np.all(np.isnan(got[:layer]))
        assert ctx.check_status() == dgmod.DG_OK
