"""The step bench.py times, at its full sizes and in its launch configuration, against the oracle: one classical
RK4 step (dg_step: four RHS evaluations with the stage updates fused into the volume kernel) of the curvilinear
Taylor-Green vortex, p = 3, Mach 0.1, sine mapping of amplitude 0.1 on [-pi, pi]^3, at 16^3 elements (262,144 DOF,
the headline) and 32^3 elements (2,097,152 DOF, inputs larger than L2), in FP64 and in the FP32 flux mode, with the
library's default options (automatic staging, which takes the pipelined volume kernel at these sizes, and
programmatic dependent launches) and the bench's time step (CFL 0.5 on the smallest node spacing). Every DOF is
compared.

Bound: the step's increment is dt times the RK4 combination of four RHS evaluations (weights summing to 1), each
within the parity bound of the RHS (term-relative: FP64 1e-12, FP32 4e-6 of the largest RHS term magnitude), plus
what an error of one stage carries into the later stages' states (dt times the RHS's Lipschitz constant, below
1 at CFL 0.5). So |increment - oracle increment| <= 2 tol dt max(terms), tested per variable; the FP64 state
update itself rounds at eps |u|, far below that."""
import functools
import math

import numpy as np
import pytest

import oracle as orc
from cases import Scenario, parity_errors

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 4e-6}
POLYDEG = 3
MACH = 0.1


@pytest.fixture(scope="module")
def dgmod():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_10517_gb300 import build
    build.build()
    from paper_2112_10517_gb300 import dg
    return dg


def bench_dt(ne):
    # the bench's step: CFL 0.5 on the smallest node spacing, |v| + c <= 1 + 1/M for the Taylor-Green state
    return 0.5 * (2 * math.pi / ne) / (POLYDEG + 1) ** 2 / (1.0 + 1.0 / MACH)


@functools.lru_cache(maxsize=None)
def oracle_step(ne):
    """The scenario, the oracle's RK4 step from its state and the RHS term magnitudes at that state."""
    sc = Scenario(3, [ne] * 3, POLYDEG, mapping="sine", amp=0.1, ic="tgv", llf=True)
    ref = orc.rk_step(0, 3, POLYDEG, sc.nelem, sc.Ja, sc.J, sc.u, bench_dt(ne), llf=True)
    return sc, ref, sc.du_scale()


@pytest.mark.parametrize("ne", [16, 32])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_bench_step_matches_oracle_at_full_size(dgmod, precision, ne):
    import torch
    sc, ref, scale = oracle_step(ne)
    ctx = dgmod.DG(precision=precision, **sc.dg_kwargs())
    assert ctx.ndofs == ne ** 3 * (POLYDEG + 1) ** 3
    u = torch.from_numpy(sc.u).cuda()
    scratch = torch.empty((2,) + ctx.shape, dtype=torch.float64, device="cuda")
    dt = bench_dt(ne)
    ctx.step(u, dt, dgmod.DG_RK4_CLASSIC, scratch=scratch)
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    got = u.cpu().numpy()
    _, term = parity_errors((got - sc.u) / dt, (ref - sc.u) / dt, scale)
    print(precision, ne, "increment error / (dt max terms) per variable:", " ".join("%.1e" % x for x in term))
    assert np.all(term <= 2 * TOL[precision]), term
