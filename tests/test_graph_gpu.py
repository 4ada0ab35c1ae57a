"""dg_rhs and dg_step inside CUDA graphs: the library neither allocates nor synchronizes in these calls, so a
captured sequence replays the same kernels; replays must equal eager execution bit for bit (LGL FP64 and FP32 with
both Runge-Kutta schemes, Gauss collocation), and the non-physical flag still reaches dg_check_status."""
import math

import numpy as np
import pytest

from cases import Scenario

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


def context(dgmod, precision="fp64", nodes="lgl"):
    from paper_2112_10517_gb300 import inputs
    mapping = dict(mapping="affine") if nodes == "gauss" else dict(mapping="sine", amp=0.1)
    ctx = dgmod.DG(3, [4, 3, 5], 3, lo=[-math.pi] * 3, hi=[math.pi] * 3, surface="llf", precision=precision,
                   nodes=nodes, **mapping)
    return ctx, inputs.taylor_green(ctx.node_coords(), mach=0.3)


@pytest.mark.parametrize("precision,nodes", [("fp64", "lgl"), ("fp32", "lgl"), ("fp64", "gauss")])
@pytest.mark.parametrize("scheme", [0, 1])
def test_step_graph_replay_equals_eager(dgmod, precision, nodes, scheme):
    import torch
    ctx, u0 = context(dgmod, precision, nodes)
    u = torch.from_numpy(u0).cuda()
    scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device="cuda")
    dt, steps = 0.002, 3
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    ctx.step(u, dt, scheme=scheme, scratch=scratch)  # first calls outside the capture
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        for _ in range(steps):
            ctx.step(u, dt, scheme=scheme, scratch=scratch, stream=side)
    u.copy_(torch.from_numpy(u0))
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    replayed = u.cpu().numpy()
    u.copy_(torch.from_numpy(u0))
    for _ in range(2 * steps):
        ctx.step(u, dt, scheme=scheme, scratch=scratch)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(replayed, u.cpu().numpy())
    assert ctx.check_status() == dgmod.DG_OK


def test_rhs_graph_replay_and_flag(dgmod):
    import torch
    ctx, u0 = context(dgmod)
    u = torch.from_numpy(u0).cuda()
    du = torch.empty_like(u)
    ref = ctx.rhs(u).clone()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        ctx.rhs(u, du, stream=side)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(du, ref)
    u[1, 0, 3] = -1.0  # a negative density: the replayed kernels raise the flag
    graph.replay()
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_ERR_NONPHYSICAL
    assert ctx.check_status() == dgmod.DG_OK


def test_profiling_counts_the_selected_kernels_only(dgmod):
    # dg_profile_enable times every kernel; dg_profile_enable_kernels only those of its mask (the bench's timed
    # region carries events around the volume kernel alone); every launch is counted either way
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="smooth", llf=True, seed=710)
    ctx = dgmod.DG(**sc.dg_kwargs())
    u = torch.from_numpy(sc.u).cuda()
    du = torch.empty_like(u)
    n0 = ctx.launch_count()
    ctx.profile(True)
    for _ in range(3):
        ctx.rhs(u, du)
    assert ctx.profile_read(dgmod.KERNEL_VOLUME)[1] == 3 and ctx.profile_read(dgmod.KERNEL_INTERFACE)[1] == 3
    ctx.profile(True, kernels=[dgmod.KERNEL_VOLUME])
    for _ in range(2):
        ctx.rhs(u, du)
    vol_ms, vol_n = ctx.profile_read(dgmod.KERNEL_VOLUME)
    assert vol_n == 2 and vol_ms > 0.0
    assert ctx.profile_read(dgmod.KERNEL_INTERFACE)[1] == 0
    ctx.profile(True, kernels=[dgmod.KERNEL_VOLUME], every=3)  # launches 0, 3, 6 of the volume kernel
    for _ in range(7):
        ctx.rhs(u, du)
    assert ctx.profile_read(dgmod.KERNEL_VOLUME)[1] == 3
    ctx.profile(False)
    ctx.rhs(u, du)
    assert ctx.profile_read(dgmod.KERNEL_VOLUME)[1] == 0
    assert ctx.launch_count() - n0 == 26


def test_host_buffer_entry_points_match_device_calls(dgmod):
    # dg_rhs_host / dg_step_host: the same kernels on device copies of a host state, bit for bit; pinned host
    # memory (asynchronous copies) and pageable memory (synchronous copies)
    import torch
    sc = Scenario(3, [3, 2, 3], 3, mapping="sine", ic="smooth", llf=True, seed=720)
    ctx = dgmod.DG(**sc.dg_kwargs())
    du_dev = ctx.rhs(torch.from_numpy(sc.u).cuda()).cpu()
    uh = torch.from_numpy(sc.u.copy()).pin_memory()
    duh = torch.empty_like(uh).pin_memory()
    ctx.rhs_host(uh, duh)
    torch.cuda.synchronize()
    assert torch.equal(duh, du_dev)
    up, dup = torch.from_numpy(sc.u.copy()), torch.empty(uh.shape, dtype=torch.float64)
    ctx.rhs_host(up, dup)
    torch.cuda.synchronize()
    assert torch.equal(dup, du_dev)
    ud = torch.from_numpy(sc.u).cuda()
    for _ in range(2):
        ctx.step(ud, 1e-3)
        ctx.step_host(uh, 1e-3)
    torch.cuda.synchronize()
    assert torch.equal(uh, ud.cpu())
    assert ctx.check_status() == dgmod.DG_OK
    with pytest.raises(TypeError):
        ctx.rhs_host(ud, duh)  # a device tensor is not a host state


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("precision,nelem,staging", [("fp64", [16, 16, 16], "auto"), ("fp32", [16, 16, 16], "auto"),
                                                     ("fp64", [3, 4, 3], "direct")])
def test_host_step_writes_the_result_into_pinned_memory(dgmod, scheme, precision, nelem, staging):
    # a pinned result buffer receives the last stage's state from the volume kernel itself (through its device
    # address); a pageable one by a copy: both equal dg_step on the device bit for bit, both schemes, both kernels
    import torch
    sc = Scenario(3, nelem, 3, mapping="sine", ic="tgv", llf=True)
    ctx = dgmod.DG(precision=precision, staging=staging, **sc.dg_kwargs())
    ud = torch.from_numpy(sc.u).cuda()
    pinned = torch.from_numpy(sc.u.copy()).pin_memory()
    pageable = torch.from_numpy(sc.u.copy())
    for _ in range(2):
        ctx.step(ud, 1e-3, scheme)
        ctx.step_host(pinned, 1e-3, scheme)
        ctx.step_host(pageable, 1e-3, scheme)
        torch.cuda.synchronize()
    ref = ud.cpu()
    assert torch.equal(pinned, ref) and torch.equal(pageable, ref)
    assert ctx.check_status() == dgmod.DG_OK


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("staging,p,nelem", [("pipelined", 3, [16, 16, 16]), ("direct", 3, [4, 3, 5]),
                                             ("pipelined", 2, [9, 8, 10])])
def test_overlapped_launches_equal_serial_launches(dgmod, precision, staging, p, nelem):
    # DG_LAUNCH_OVERLAP schedules each interface and pipelined volume kernel ahead, as a programmatic dependent of
    # the kernel before it; reads of the state, the fluxes and the RK operands wait for that kernel's writes.
    # Back-to-back dg_rhs calls on different
    # states (the second interface kernel rewrites the flux buffer the first volume kernel reads) and RK steps
    # (each stage reads what the previous one wrote) must equal ordinary launches bit for bit.
    import torch
    from paper_2112_10517_gb300 import inputs
    res = {}
    for launch in ("overlap", "serial"):
        ctx = dgmod.DG(3, nelem, p, lo=[-math.pi] * 3, hi=[math.pi] * 3, mapping="sine", amp=0.1, surface="llf",
                       precision=precision, staging=staging, launch=launch)
        u0 = inputs.taylor_green(ctx.node_coords(), mach=0.3)
        ua = torch.from_numpy(u0).cuda()
        ub = (ua * 1.01).contiguous()
        torch.cuda.synchronize()
        dus = [torch.empty_like(ua) for _ in range(4)]
        for k in range(4):
            ctx.rhs(ua if k % 2 == 0 else ub, du=dus[k])
        u = ua.clone()
        scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device="cuda")
        for scheme in (0, 1, 0):
            ctx.step(u, 0.002, scheme=scheme, scratch=scratch)
        torch.cuda.synchronize()
        assert ctx.check_status() == dgmod.DG_OK
        res[launch] = [d.cpu().numpy() for d in dus] + [u.cpu().numpy()]
    for a, b in zip(res["overlap"], res["serial"]):
        np.testing.assert_array_equal(a, b)
    np.testing.assert_array_equal(res["overlap"][0], res["overlap"][2])
    np.testing.assert_array_equal(res["overlap"][1], res["overlap"][3])


@pytest.mark.parametrize("nd,nelem,chunked,extra", [(3, [4, 3, 9], True, {}), (3, [3, 2, 4], True, {}),
                                                   (2, [5, 11], True, {}), (3, [2, 3, 3], False, {}),
                                                   (3, [3, 2, 8], True, {"precision": "fp32"}),
                                                   (3, [2, 2, 8], False, {"nodes": "gauss", "mapping": "affine"})])
def test_host_entry_points_upload_the_state_in_chunks(dgmod, nd, nelem, chunked, extra):
    # with at least 4 element layers along the last direction the host state arrives in 2 chunks of layers on a
    # copy stream, and the first interface fluxes are computed per chunk as it arrives (2 interface launches
    # instead of 1): bit for bit the device calls' results, for uneven chunks (9 layers), two layers per chunk
    # (4), 2D, FP32, and one copy for 3 layers and for Gauss collocation; pinned and pageable host memory
    import torch
    extra = dict(extra)
    sc = Scenario(nd, nelem, 3, mapping=extra.pop("mapping", "sine"), ic="smooth", llf=True, seed=730)
    ctx = dgmod.DG(**sc.dg_kwargs(), **extra)
    ud = torch.from_numpy(sc.u).cuda()
    n0 = ctx.launch_count()
    du_dev = ctx.rhs(ud).cpu()
    base = ctx.launch_count() - n0  # the device call's kernels; chunked: one interface launch more
    for pin in (True, False):
        uh = torch.from_numpy(sc.u.copy())
        duh = torch.empty_like(uh)
        if pin:
            uh, duh = uh.pin_memory(), duh.pin_memory()
        n0 = ctx.launch_count()
        ctx.rhs_host(uh, duh)
        torch.cuda.synchronize()
        assert ctx.launch_count() - n0 == base + (1 if chunked else 0)
        assert torch.equal(duh, du_dev)
    for scheme in (0, 1):
        ud = torch.from_numpy(sc.u).cuda()
        uh = torch.from_numpy(sc.u.copy()).pin_memory()
        for _ in range(2):
            ctx.step(ud, 1e-3, scheme)
            ctx.step_host(uh, 1e-3, scheme)
        torch.cuda.synchronize()
        assert torch.equal(uh, ud.cpu()), scheme
    assert ctx.check_status() == dgmod.DG_OK
