"""The 3D curvilinear Taylor-Green workload run in time: 16^3 elements, p = 3, Mach 0.1, 100 steps of the
four-stage low-storage RK4 (dg_step). At every step the entropy rate (dg_entropy_rate) is checked: zero to
rounding with the EC surface flux, non-positive with LLF (Sec. 2: EC/ED semidiscretizations). Conserved totals
stay constant (discrete conservation; RK preserves linear invariants), and a free stream stays constant on the
curved mesh (curl-form metrics, Sec. 2.3)."""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2112_10517_gb300 import inputs

pytestmark = pytest.mark.gpu

NELEM = [16, 16, 16]
P = 3


@pytest.fixture(scope="module")
def dgmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10517_gb300 import build
    build.build()
    from paper_2112_10517_gb300 import dg
    return dg


def totals(ctx, u):
    J = ctx.metrics()[1]
    return orc.integrate(3, P, J, u.cpu().numpy())


@pytest.mark.parametrize("surface", ["ec", "llf"])
def test_tgv_100_steps_entropy_and_conservation(dgmod, surface):
    import torch
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    ctx = dgmod.DG(3, NELEM, P, lo=lo, hi=hi, mapping="sine", amp=0.1, surface=surface)
    u = torch.from_numpy(inputs.taylor_green(ctx.node_coords(), mach=0.1)).cuda()
    dt = 0.5 * (2 * math.pi / NELEM[0]) / (P + 1) ** 2 / (1.0 + 1.0 / 0.1)
    tot0, ab0 = totals(ctx, u)
    du = torch.empty_like(u)
    rates = []
    for step in range(100):
        ctx.rhs(u, du)
        s, scale = ctx.entropy_rate(u, du)
        rates.append((s, scale))
        ctx.step(u, dt)
    assert ctx.check_status() == dgmod.DG_OK
    for s, scale in rates:
        if surface == "ec":
            assert abs(s) <= 1e-13 * scale, (s, scale)
        else:
            assert s <= 1e-13 * scale, (s, scale)
    if surface == "llf":
        assert sum(s for s, _ in rates) < 0.0
    tot1, _ = totals(ctx, u)
    # momentum components share one scale (the Taylor-Green z-momentum is zero initially)
    scale = np.array([ab0[0]] + [ab0[1:4].max()] * 3 + [ab0[4]])
    assert np.all(np.abs(tot1 - tot0) <= 1e-13 * scale), (tot1 - tot0, scale)


def test_free_stream_100_steps_curved(dgmod):
    import torch
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    ctx = dgmod.DG(3, NELEM, P, lo=lo, hi=hi, mapping="sine", amp=0.1, surface="llf")
    u0 = inputs.free_stream(ctx.node_coords(), v=[0.1, 0.2, 0.3])
    u = torch.from_numpy(u0).cuda()
    dt = 0.5 * (2 * math.pi / NELEM[0]) / (P + 1) ** 2 / 2.0
    for _ in range(100):
        ctx.step(u, dt)
    # 400 stages of rounding: the drift stays at 1e-13 of the state's magnitude
    dev = np.max(np.abs(u.cpu().numpy() - u0), axis=(0, 2))
    assert np.all(dev <= 1e-12 * np.max(np.abs(u0))), dev
