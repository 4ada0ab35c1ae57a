"""Host logic of the slab partition (paper_2112_10517_gb300/partition.py) on CPU: the slab plan, the periodic
neighbours, the halo exchange between gloo ranks (world sizes 2 and 3, where with two ranks both neighbours are
the same rank and the two planes must not be confused), the all-reduce of diagnostics, and the order in which a
slab exchanges halos around the Runge-Kutta stages. The face-plane layout the exchange moves is the one include/dg.h
documents for dg_part_pack / dg_part_unpack: [layer][nvar][N^(d-1)], plane i_last = 0 of the first own layer going
down, plane i_last = p of the last own layer going up."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2112_10517_gb300 import partition  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_slab_plan_covers_the_cut_with_balanced_slabs():
    for n in range(1, 21):
        for world in range(1, n + 1):
            plan = partition.slab_plan(n, world)
            assert plan[0][0] == 0 and plan[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(plan, plan[1:]))
            sizes = [e - b for b, e in plan]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        partition.slab_plan(3, 4)


def test_neighbours_are_periodic():
    assert partition.neighbors(0, 1) == (0, 0)
    assert partition.neighbors(0, 2) == (1, 1)
    assert partition.neighbors(0, 4) == (3, 1) and partition.neighbors(3, 4) == (2, 0)


def global_state(nd, nelem, p, seed=0):
    rng = np.random.Generator(np.random.PCG64(seed))
    E = int(np.prod(nelem))
    return rng.standard_normal((E, nd + 2, (p + 1) ** nd))


def plane(u_elems, k, nl):
    """Node plane i_last = k of each element: [elements][nvar][nl]."""
    return u_elems[:, :, k * nl:(k + 1) * nl]


def _worker(rank, world, port, nd, nelem, p, out):
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        # tagged scalars first: which rank's buffer arrives where
        L = 6
        send_lo = torch.full((L,), rank * 10 + 1.0, dtype=torch.float64)
        send_hi = torch.full((L,), rank * 10 + 2.0, dtype=torch.float64)
        recv_lo, recv_hi = torch.zeros(L, dtype=torch.float64), torch.zeros(L, dtype=torch.float64)
        partition.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world)
        lower, upper = partition.neighbors(rank, world)
        ok_tags = bool(torch.all(recv_lo == lower * 10 + 2.0)) and bool(torch.all(recv_hi == upper * 10 + 1.0))
        # the real planes: this rank's slab of a global state, ghost layer in front (only its two planes are set)
        N, nl = p + 1, (p + 1) ** (nd - 1)
        layer = int(np.prod(nelem[:-1]))
        u = global_state(nd, nelem, p)
        b, e = partition.slab_plan(nelem[-1], world)[rank]
        ext = np.full((layer * (e - b + 1),) + u.shape[1:], np.nan)
        ext[layer:] = u[b * layer:e * layer]
        s_lo = torch.from_numpy(np.ascontiguousarray(plane(ext[layer:2 * layer], 0, nl)).ravel())
        s_hi = torch.from_numpy(np.ascontiguousarray(plane(ext[-layer:], N - 1, nl)).ravel())
        r_lo, r_hi = torch.zeros_like(s_lo), torch.zeros_like(s_hi)
        partition.exchange(s_lo, s_hi, r_lo, r_hi, rank, world)
        ext[:layer, :, (N - 1) * nl:N * nl] = r_lo.numpy().reshape(layer, nd + 2, nl)
        ext[:layer, :, 0:nl] = r_hi.numpy().reshape(layer, nd + 2, nl)
        nlast = nelem[-1]
        below = u[((b - 1) % nlast) * layer:((b - 1) % nlast + 1) * layer]
        above = u[(e % nlast) * layer:(e % nlast + 1) * layer]
        ok_planes = (np.array_equal(plane(ext[:layer], N - 1, nl), plane(below, N - 1, nl)) and
                     np.array_equal(plane(ext[:layer], 0, nl), plane(above, 0, nl)) and
                     bool(np.all(np.isnan(ext[:layer, :, nl:(N - 1) * nl]))))
        tot = partition.allreduce_sum([1.0, rank], torch.device("cpu"))
        out[rank] = (ok_tags, ok_planes, tot.tolist())
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,nd,nelem,p", [(2, 3, [2, 3, 4], 3), (3, 3, [2, 2, 5], 2), (2, 2, [3, 4], 4)])
def test_gloo_halo_exchange_delivers_the_neighbour_planes(world, nd, nelem, p):
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, nd, nelem, p, out), nprocs=world, join=True)
    for r in range(world):
        ok_tags, ok_planes, tot = out[r]
        assert ok_tags and ok_planes, r
        assert tot == [float(world), float(sum(range(world)))]


def test_single_rank_is_its_own_neighbour():
    a, b = torch.arange(4.0), torch.arange(4.0) + 10
    c, d = torch.zeros(4), torch.zeros(4)
    partition.exchange(a, b, c, d, 0, 1)
    assert torch.equal(c, b) and torch.equal(d, a)
    bufs = [[torch.full((3,), 10.0 * r + 1), torch.full((3,), 10.0 * r + 2), torch.zeros(3), torch.zeros(3)]
            for r in range(3)]
    partition.exchange_local(bufs)
    for r in range(3):
        assert torch.all(bufs[r][2] == 10.0 * ((r - 1) % 3) + 2) and torch.all(bufs[r][3] == 10.0 * ((r + 1) % 3) + 1)


class FakeSlabContext:
    """Records the calls a Slab makes (no device)."""

    def __init__(self):
        self.part = object()
        self.calls = []

    def halo_buffers(self):
        return [torch.zeros(2) for _ in range(4)]

    def pack(self, state, a, b, stream=None):
        self.calls.append(("pack", id(state)))

    def unpack(self, state, a, b, stream=None):
        self.calls.append(("unpack", id(state)))

    def stage_interface(self, u, scratch, scheme, st, region):
        self.calls.append(("iface", st, region))

    def stage_volume(self, u, scratch, dt, scheme, st):
        self.calls.append(("stage", st))

    def rhs(self, u, du=None):
        self.calls.append(("rhs", id(u)))


def test_slab_exchanges_each_stage_input_before_the_stage(monkeypatch):
    # RK4 reads u at stage 0 and the stage state scratch[0] at stages 1-3; CK(5,4) reads u at every stage
    import types
    import sys
    fake_dg = types.SimpleNamespace(DG_RK4_CLASSIC=0, DG_REGION_INTERIOR=0, DG_REGION_BOUNDARY=1,
                                    DG=types.SimpleNamespace(stage_input=lambda scheme, st: 1 if scheme == 0 and st > 0
                                                             else 0))
    monkeypatch.setitem(sys.modules, "paper_2112_10517_gb300.dg", fake_dg)
    monkeypatch.setattr(sys.modules["paper_2112_10517_gb300"], "dg", fake_dg, raising=False)
    ctx = FakeSlabContext()
    moved = []

    class Pending:  # a transfer in flight: its wait is recorded among the context's calls
        def wait(self):
            ctx.calls.append(("finish",))

    def transport(*bufs):
        moved.append(len(bufs))
        ctx.calls.append(("start",))
        return [Pending()]
    slab = partition.Slab(ctx, exchange_fn=transport)
    u, scratch = torch.zeros(3), torch.zeros(2, 3)
    slab.step(u, scratch, 0.1, 0)
    y = id(scratch[0])
    kinds = [c[0] for c in ctx.calls]
    # per stage: the interior faces between the start and the finish of the transfers, the boundary faces after
    # the unpack, then the volume kernel
    assert kinds == ["pack", "start", "iface", "finish", "unpack", "iface", "stage"] * 4 and moved == [4] * 4
    assert [c[2] for c in ctx.calls if c[0] == "iface"] == [0, 1] * 4
    assert [c[1] for c in ctx.calls if c[0] == "stage"] == [0, 1, 2, 3]
    packs = [c[1] for c in ctx.calls if c[0] == "pack"]
    assert packs[0] == id(u) and packs[1] != id(u)
    ctx.calls.clear()
    slab.step(u, scratch[:1], 0.1, 1)
    assert [c[1] for c in ctx.calls if c[0] == "pack"] == [id(u)] * 5
    ctx.calls.clear()
    slab.rhs(u)
    assert [c[0] for c in ctx.calls] == ["pack", "start", "finish", "unpack", "rhs"]
    del y
