"""Slab partition of one periodic mesh over ranks, and the halo exchange of a flux-differencing RHS.

Sec. 2.4: the volume terms are element-local and each interface flux needs only the two adjacent elements' face
states. So a mesh cut into slabs of element layers along its last direction needs, per RHS evaluation (per
Runge-Kutta stage), one plane of face states from each neighbouring slab and nothing else; the conservation and
entropy diagnostics need one all-reduce of nvar + 2 scalars. The library's partitioned contexts (dg_init_part,
include/dg.h) hold a ghost layer for those planes and pack / unpack them on the device; this module plans the slabs,
moves the planes between ranks (torch.distributed point-to-point: NCCL for CUDA tensors, gloo for CPU tensors) and
drives a slab's RHS and time step. A single rank is its own neighbour (the mesh is periodic).
"""
from __future__ import annotations


def slab_plan(n_last: int, world: int):
    """Balanced contiguous element-layer ranges [begin, end) for `world` slabs of a mesh with n_last layers along
    its last direction (the first n_last % world slabs get one layer more)."""
    if world < 1 or n_last < world:
        raise ValueError("need 1 <= world <= layers along the cut (%d slabs of %d layers)" % (world, n_last))
    base, extra = divmod(n_last, world)
    out, b = [], 0
    for r in range(world):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def neighbors(rank: int, world: int):
    """(lower, upper) neighbour ranks of a slab along the periodic cut direction."""
    return (rank - 1) % world, (rank + 1) % world


# message tags (gloo matches on them; NCCL matches in posting order, which the list below keeps the same on every
# rank): the lower-face plane travels down, the upper-face plane up
TAG_DOWN, TAG_UP = 7, 8


def exchange_start(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """Queues send_lo -> the lower neighbour's recv_hi and send_hi -> the upper neighbour's recv_lo, and returns the
    requests that exchange_finish waits for. NCCL runs the transfers on its own stream after the work queued so far
    on the current stream (the pack), so that work queued on the current stream before exchange_finish overlaps
    them. One rank: local copies on the current stream, no requests."""
    if world == 1:
        recv_lo.copy_(send_hi)
        recv_hi.copy_(send_lo)
        return []
    import torch.distributed as dist
    lower, upper = neighbors(rank, world)
    ops = [dist.P2POp(dist.isend, send_lo, lower, group, TAG_DOWN),
           dist.P2POp(dist.irecv, recv_hi, upper, group, TAG_DOWN),
           dist.P2POp(dist.isend, send_hi, upper, group, TAG_UP),
           dist.P2POp(dist.irecv, recv_lo, lower, group, TAG_UP)]
    return dist.batch_isend_irecv(ops)


def exchange_finish(pending):
    """Waits for exchange_start's requests (NCCL: the current stream waits for the transfers; gloo: the host)."""
    for req in pending or ():
        req.wait()


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, group=None):
    """exchange_start and exchange_finish: the receives are complete on the current stream (NCCL) or on the host
    (gloo) when it returns."""
    exchange_finish(exchange_start(send_lo, send_hi, recv_lo, recv_hi, rank, world, group))


def exchange_local(bufs):
    """The same exchange among slabs held by one process (bufs[r] = (send_lo, send_hi, recv_lo, recv_hi) of slab r,
    slabs in order along the cut): recv_lo[r] <- send_hi[r - 1], recv_hi[r] <- send_lo[r + 1], periodic."""
    w = len(bufs)
    for r in range(w):
        bufs[r][2].copy_(bufs[(r - 1) % w][1])
        bufs[r][3].copy_(bufs[(r + 1) % w][0])


def allreduce_sum(values, device, group=None):
    """Sum a small vector of diagnostics (conserved totals, entropy rate) over all ranks (FP64)."""
    import numpy as np
    import torch
    import torch.distributed as dist
    t = torch.tensor(np.asarray(values, dtype=np.float64), dtype=torch.float64, device=device)
    if dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


class Slab:
    """One rank's slab: a partitioned context (dg.DG with part=...) and its four halo buffers. rhs() runs pack ->
    exchange -> unpack -> RHS; step() runs, per stage, pack -> exchange start -> the interior faces' fluxes (which
    read no ghost-layer data, so they overlap the transfers) -> exchange finish -> unpack -> the boundary faces'
    fluxes -> volume and update. `exchange_fn(send_lo, send_hi, recv_lo, recv_hi)` queues the plane transfers and
    returns what exchange_finish waits for (default: exchange_start over torch.distributed with this rank's
    neighbours; a blocking transport may return None)."""

    def __init__(self, ctx, rank: int = 0, world: int = 1, group=None, exchange_fn=None):
        if ctx.part is None:
            raise ValueError("Slab needs a partitioned context (dg.DG(..., part=(begin, end)))")
        self.ctx, self.rank, self.world, self.group = ctx, rank, world, group
        self.bufs = ctx.halo_buffers()
        self.exchange_fn = exchange_fn or (lambda a, b, c, d: exchange_start(a, b, c, d, rank, world, group))

    def halo(self, state, stream=None):
        send_lo, send_hi, recv_lo, recv_hi = self.bufs
        self.ctx.pack(state, send_lo, send_hi, stream=stream)
        exchange_finish(self.exchange_fn(send_lo, send_hi, recv_lo, recv_hi))
        self.ctx.unpack(state, recv_lo, recv_hi, stream=stream)

    def rhs(self, u, du=None):
        self.halo(u)
        return self.ctx.rhs(u, du)

    def step(self, u, scratch, dt: float, scheme: int):
        from . import dg
        stages = 4 if scheme == dg.DG_RK4_CLASSIC else 5
        send_lo, send_hi, recv_lo, recv_hi = self.bufs
        for st in range(stages):
            state = u if dg.DG.stage_input(scheme, st) == 0 else scratch[0]
            self.ctx.pack(state, send_lo, send_hi)
            pending = self.exchange_fn(send_lo, send_hi, recv_lo, recv_hi)
            self.ctx.stage_interface(u, scratch, scheme, st, dg.DG_REGION_INTERIOR)  # overlaps the transfers
            exchange_finish(pending)
            self.ctx.unpack(state, recv_lo, recv_hi)
            self.ctx.stage_interface(u, scratch, scheme, st, dg.DG_REGION_BOUNDARY)
            self.ctx.stage_volume(u, scratch, dt, scheme, st)
        return u
