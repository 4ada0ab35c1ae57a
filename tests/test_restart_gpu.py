"""Checkpoint and resume: the state of a run is (u, t, step count, Runge-Kutta scheme), and the mesh and options that
made the context. A run stopped after some steps, its state saved to host memory, its context freed and a new one
made from the same mesh and options, must continue bit for bit as the run that never stopped: the stage kernels
sum in a fixed order and a context keeps nothing between steps but its geometry, which dg_init recomputes the
same way (LGL FP64 and FP32, both schemes, and a mesh large enough for the FP64 volume kernel's counter
schedule)."""
import math

import numpy as np
import pytest

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


def make(dgmod, nelem, precision):
    return dgmod.DG(3, nelem, 3, lo=[-math.pi] * 3, hi=[math.pi] * 3, mapping="sine", amp=0.1, surface="llf",
                    precision=precision)


@pytest.mark.parametrize("nelem", [[4, 3, 5], [16, 16, 17]])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("scheme", [0, 1])
def test_resumed_run_equals_uninterrupted_run(dgmod, nelem, precision, scheme, tmp_path):
    import torch
    from paper_2112_10517_gb300 import inputs
    ctx = make(dgmod, nelem, precision)
    u0 = inputs.taylor_green(ctx.node_coords(), mach=0.1)
    dt, steps, half = 1e-3, 6, 3
    u = torch.from_numpy(u0).cuda()
    for _ in range(steps):
        ctx.step(u, dt, scheme=scheme)
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    straight = u.cpu().numpy()
    # the same run stopped after `half` steps: state to a file, context freed, a new context, the rest
    u = torch.from_numpy(u0).cuda()
    for _ in range(half):
        ctx.step(u, dt, scheme=scheme)
    torch.cuda.synchronize()
    path = tmp_path / "checkpoint.npz"
    np.savez(path, u=u.cpu().numpy(), t=half * dt, step=half, scheme=scheme)
    del ctx, u
    torch.cuda.synchronize()
    saved = np.load(path)
    ctx = make(dgmod, nelem, precision)
    u = torch.from_numpy(saved["u"]).cuda()
    for _ in range(steps - int(saved["step"])):
        ctx.step(u, dt, scheme=int(saved["scheme"]))
    torch.cuda.synchronize()
    assert ctx.check_status() == dgmod.DG_OK
    np.testing.assert_array_equal(u.cpu().numpy(), straight)
