"""Partitioned contexts (dg_init_part): one periodic mesh cut into slabs of element layers along its last
direction, each slab a context with a ghost layer, halo planes packed, moved and unpacked between them (Sec. 2.4:
volume terms are element-local, each interface flux needs the two adjacent elements' face states).

Several slabs run in one process on one GPU; exchange_local moves the planes as a transport between ranks would.
The slabs' RHS and Runge-Kutta steps must equal the whole mesh's, bit for bit (the same arithmetic on the same
inputs: the slabs' node coordinates and metric terms are those of the whole mesh, and every interface flux is
computed from the same two states and the lower element's metric terms), with both volume-kernel stagings, FP64 and
FP32, both fluxes, EC and LLF surfaces, and a slab that is its own neighbour. The diagnostics summed over the slabs
equal the whole mesh's to rounding; the oracle confirms the assembled RHS."""
import math

import numpy as np
import pytest

import oracle as orc
from cases import Scenario, assert_parity

pytestmark = pytest.mark.gpu

PI = math.pi


@pytest.fixture(scope="module")
def dgmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10517_gb300 import build
    build.build()
    from paper_2112_10517_gb300 import dg
    return dg


def make_slabs(dgmod, sc, nslabs, **kw):
    import torch
    from paper_2112_10517_gb300 import partition
    whole = dgmod.DG(**sc.dg_kwargs(), **kw)
    layer = int(np.prod(sc.nelem[:-1]))
    slabs = []
    for b, e in partition.slab_plan(sc.nelem[-1], nslabs):
        ctx = dgmod.DG(**sc.dg_kwargs(), part=(b, e), **kw)
        assert ctx.ghost_elems == layer and ctx.nelem_total == layer * (e - b + 1)
        assert ctx.ndofs == layer * (e - b) * ctx.nodes_per_elem
        # geometry: the slab's elements (ghost layer = layer b - 1, periodic) are those of the whole mesh
        g = np.concatenate([np.arange(((b - 1) % sc.nelem[-1]) * layer, ((b - 1) % sc.nelem[-1] + 1) * layer),
                            np.arange(b * layer, e * layer)])
        np.testing.assert_array_equal(ctx.node_coords(), whole.node_coords()[g])
        np.testing.assert_array_equal(ctx.metrics()[0], whole.metrics()[0][g])
        u = torch.full(ctx.shape, float("nan"), dtype=torch.float64, device="cuda")  # ghost: only two planes read
        u[layer:] = torch.from_numpy(sc.u[b * layer:e * layer]).cuda()
        slabs.append((ctx, u, ctx.halo_buffers(), (b, e)))
    return whole, slabs, layer


def halo_all(slabs, states):
    from paper_2112_10517_gb300 import partition
    for (ctx, _, bufs, _), st in zip(slabs, states):
        ctx.pack(st, bufs[0], bufs[1])
    partition.exchange_local([s[2] for s in slabs])
    for (ctx, _, bufs, _), st in zip(slabs, states):
        ctx.unpack(st, bufs[2], bufs[3])


CASES = [(3, [3, 2, 6], 3, 2), (3, [2, 3, 5], 3, 3), (3, [3, 2, 4], 4, 1), (3, [2, 2, 7], 2, 4), (2, [4, 6], 3, 3),
         (2, [3, 5], 5, 2)]


@pytest.mark.parametrize("staging", ["direct", "pipelined"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nd,nelem,p,nslabs", CASES)
def test_slab_rhs_equals_whole_mesh_bit_for_bit(dgmod, nd, nelem, p, nslabs, precision, staging):
    import torch
    sc = Scenario(nd, nelem, p, mapping="sine", ic="rough", llf=True, seed=70 + p)
    whole, slabs, layer = make_slabs(dgmod, sc, nslabs, precision=precision, staging=staging)
    ref = whole.rhs(torch.from_numpy(sc.u).cuda()).cpu().numpy()
    halo_all(slabs, [s[1] for s in slabs])
    for ctx, u, _, (b, e) in slabs:
        du = torch.full_like(u, float("nan"))
        ctx.rhs(u, du)
        assert ctx.check_status() == dgmod.DG_OK
        got = du.cpu().numpy()
        np.testing.assert_array_equal(got[layer:], ref[b * layer:e * layer])
        assert np.all(np.isnan(got[:layer]))  # the ghost layer of du is not written
    if precision == "fp64" and staging == "direct":  # the assembled RHS against the oracle
        assembled = np.concatenate([s[0].rhs(s[1]).cpu().numpy()[layer:] for s in slabs])
        assert_parity(assembled, sc)


@pytest.mark.parametrize("flux,surface,p_ref", [("ranocha", "ec", 0.0), ("shima", "llf", 0.0),
                                                ("ranocha", "llf", 0.9)])
def test_slab_variants_equal_whole_mesh(dgmod, flux, surface, p_ref):
    import torch
    sc = Scenario(3, [3, 3, 5], 3, mapping="sine", ic="rough", llf=surface == "llf", seed=80, flux=flux)
    for precision in ("fp64", "fp32"):
        whole, slabs, layer = make_slabs(dgmod, sc, 2, precision=precision, p_ref=p_ref)
        ref = whole.rhs(torch.from_numpy(sc.u).cuda()).cpu().numpy()
        halo_all(slabs, [s[1] for s in slabs])
        for ctx, u, _, (b, e) in slabs:
            np.testing.assert_array_equal(ctx.rhs(u).cpu().numpy()[layer:], ref[b * layer:e * layer])


def test_slab_cartesian_mesh_equals_whole_mesh(dgmod):
    import torch
    sc = Scenario(3, [4, 3, 6], 3, mapping="affine", ic="rough", llf=True, seed=81)
    whole, slabs, layer = make_slabs(dgmod, sc, 3)
    ref = whole.rhs(torch.from_numpy(sc.u).cuda()).cpu().numpy()
    halo_all(slabs, [s[1] for s in slabs])
    for ctx, u, _, (b, e) in slabs:
        np.testing.assert_array_equal(ctx.rhs(u).cpu().numpy()[layer:], ref[b * layer:e * layer])


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_slab_time_steps_equal_whole_mesh(dgmod, scheme, precision):
    # per stage: pack the stage's input state on every slab, exchange, unpack, run the stage
    import torch
    sc = Scenario(3, [3, 2, 6], 3, mapping="sine", ic="smooth", llf=True, seed=82)
    whole, slabs, layer = make_slabs(dgmod, sc, 3, precision=precision)
    uw = torch.from_numpy(sc.u).cuda()
    nreg = 2 if scheme == 0 else 1
    dt = 0.01
    scr = [torch.full((nreg,) + s[0].shape, float("nan"), dtype=torch.float64, device="cuda") for s in slabs]
    stages = 4 if scheme == 0 else 5
    for _ in range(3):
        whole.step(uw, dt, scheme)
        for st in range(stages):
            ins = [s[1] if dgmod.DG.stage_input(scheme, st) == 0 else scr[k][0] for k, s in enumerate(slabs)]
            halo_all(slabs, ins)
            for k, s in enumerate(slabs):
                s[0].step_stage(s[1], scr[k], dt, scheme, st)
    ref = uw.cpu().numpy()
    for ctx, u, _, (b, e) in slabs:
        assert ctx.check_status() == dgmod.DG_OK
        np.testing.assert_array_equal(u.cpu().numpy()[layer:], ref[b * layer:e * layer])
    # a partitioned context cannot run dg_step (no halo exchange between its stages)
    with pytest.raises(dgmod.DGError) as ei:
        slabs[0][0].step(slabs[0][1], dt, scheme)
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED


def test_slab_diagnostics_sum_to_whole_mesh(dgmod):
    # conserved totals and the entropy rate of the slabs' own elements add up to the whole mesh's (one all-reduce
    # of nvar + 2 scalars in a multi-rank run); both are sums in a different order, so to rounding
    import torch
    sc = Scenario(3, [3, 2, 5], 3, mapping="sine", ic="random", llf=False, seed=83)
    whole, slabs, layer = make_slabs(dgmod, sc, 2)
    uw = torch.from_numpy(sc.u).cuda()
    duw = whole.rhs(uw)
    tot_w = whole.conserved_totals(uw)
    s_w, ab_w = whole.entropy_rate(uw, duw)
    ref_tot, _ = orc.integrate(3, 3, sc.J, sc.u)
    np.testing.assert_allclose(tot_w, ref_tot, rtol=1e-13)
    halo_all(slabs, [s[1] for s in slabs])
    tot, s_sum, ab_sum = np.zeros(5), 0.0, 0.0
    for ctx, u, _, _ in slabs:
        du = ctx.rhs(u)
        tot += ctx.conserved_totals(u)
        s, ab = ctx.entropy_rate(u, du)
        s_sum += s
        ab_sum += ab
    np.testing.assert_allclose(tot, tot_w, rtol=1e-13)
    assert abs(ab_sum - ab_w) <= 1e-13 * ab_w
    assert abs(s_sum - s_w) <= 1e-13 * ab_w and abs(s_sum) <= 1e-13 * ab_sum  # EC surface flux: entropy conserved


def test_partition_arguments(dgmod):
    sc = Scenario(3, [2, 2, 4], 3, mapping="sine", ic="smooth")
    for part in ((2, 2), (-1, 2), (0, 5), (3, 1)):
        with pytest.raises(dgmod.DGError) as ei:
            dgmod.DG(**sc.dg_kwargs(), part=part)
        assert ei.value.status == dgmod.DG_ERR_ARG
    node_sc = Scenario(3, [2, 2, 4], 3, mapping="twisted", ic="smooth")
    with pytest.raises(dgmod.DGError) as ei:  # node coordinates cannot give the ghost layer's geometry
        dgmod.DG(**node_sc.dg_kwargs(), part=(0, 2))
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED
    whole = dgmod.DG(**sc.dg_kwargs())
    import ctypes
    info = dgmod.DgPartInfo()
    assert dgmod.dg_part_get_info(whole.ctx, ctypes.byref(info)) == dgmod.DG_ERR_ARG


@pytest.mark.parametrize("scheme", [0, 1])
@pytest.mark.parametrize("precision,nelem,nslabs", [("fp64", [3, 2, 6], 3), ("fp32", [3, 2, 6], 2),
                                                   ("fp64", [2, 3, 4], 4)])
def test_slab_stages_overlapping_the_exchange_equal_whole_mesh(dgmod, scheme, precision, nelem, nslabs):
    # per stage: pack, the interior faces' fluxes (no ghost-layer data: they may overlap the transfers), exchange,
    # unpack, the boundary faces' fluxes, volume; slabs of 2 own layers and of 1 (no interior faces); bit for bit
    # the whole mesh's steps; then the same through partition.Slab on a single slab (its own neighbour)
    import torch
    from paper_2112_10517_gb300 import partition
    sc = Scenario(3, nelem, 3, mapping="sine", ic="smooth", llf=True, seed=84)
    whole, slabs, layer = make_slabs(dgmod, sc, nslabs, precision=precision)
    uw = torch.from_numpy(sc.u).cuda()
    nreg = 2 if scheme == 0 else 1
    dt = 0.01
    scr = [torch.full((nreg,) + s[0].shape, float("nan"), dtype=torch.float64, device="cuda") for s in slabs]
    stages = 4 if scheme == 0 else 5
    for _ in range(2):
        whole.step(uw, dt, scheme)
        for st in range(stages):
            ins = [s[1] if dgmod.DG.stage_input(scheme, st) == 0 else scr[k][0] for k, s in enumerate(slabs)]
            for (ctx, _, bufs, _), state in zip(slabs, ins):
                ctx.pack(state, bufs[0], bufs[1])
            for k, s in enumerate(slabs):
                s[0].stage_interface(s[1], scr[k], scheme, st, dgmod.DG_REGION_INTERIOR)
            partition.exchange_local([s[2] for s in slabs])
            for (ctx, _, bufs, _), state in zip(slabs, ins):
                ctx.unpack(state, bufs[2], bufs[3])
            for k, s in enumerate(slabs):
                s[0].stage_interface(s[1], scr[k], scheme, st, dgmod.DG_REGION_BOUNDARY)
                s[0].stage_volume(s[1], scr[k], dt, scheme, st)
    ref = uw.cpu().numpy()
    for ctx, u, _, (b, e) in slabs:
        assert ctx.check_status() == dgmod.DG_OK
        np.testing.assert_array_equal(u.cpu().numpy()[layer:], ref[b * layer:e * layer])
    # one slab of the whole mesh through partition.Slab (default transport: local copies)
    one = dgmod.DG(**sc.dg_kwargs(), part=(0, nelem[-1]), precision=precision)
    u1 = torch.full(one.shape, float("nan"), dtype=torch.float64, device="cuda")
    u1[layer:] = torch.from_numpy(sc.u).cuda()
    s1 = torch.full((nreg,) + one.shape, float("nan"), dtype=torch.float64, device="cuda")
    slab = partition.Slab(one)
    for _ in range(2):
        slab.step(u1, s1, dt, scheme)
    np.testing.assert_array_equal(u1.cpu().numpy()[layer:], ref)
    # an ordinary context has no regions; an unknown region is an argument error
    with pytest.raises(dgmod.DGError) as ei:
        whole.stage_interface(uw, torch.zeros((nreg,) + whole.shape, dtype=torch.float64, device="cuda"), scheme, 0,
                              dgmod.DG_REGION_INTERIOR)
    assert ei.value.status == dgmod.DG_ERR_ARG
    with pytest.raises(dgmod.DGError) as ei:
        one.stage_interface(u1, s1, scheme, 0, 2)
    assert ei.value.status == dgmod.DG_ERR_ARG
