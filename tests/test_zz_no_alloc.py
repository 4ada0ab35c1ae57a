"""dg_rhs_noalloc: the RHS for callers that cannot allocate device memory (for example an application whose
memory manager owns all device memory, or a latency-critical path where an allocation could synchronize the
device). It keeps the interface fluxes in one fixed device array inside the library instead of a per-context
workspace, so it must give the same du as dg_rhs, on repeated calls that reuse that array.

Collected last on purpose: a run that stops at the first failure has run every other test before this one.
"""
import ctypes

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


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_dg_rhs_on_two_calls_in_a_row(dgmod, precision):
    import torch
    # two different states on the same mesh, evaluated back to back through the shared array
    sc1 = Scenario(3, [4, 3, 5], 3, mapping="sine", ic="rough", llf=True, seed=31)
    sc2 = Scenario(3, [4, 3, 5], 3, mapping="sine", ic="tgv", llf=True)
    ctx = dgmod.DG(precision=precision, **sc1.dg_kwargs())
    Ja_h, J_h = ctx.metrics()
    Ja = torch.from_numpy(Ja_h.astype(np.float32 if precision == "fp32" else np.float64)).cuda()
    invJ = torch.from_numpy(1.0 / J_h).cuda()
    nelem = (ctypes.c_int * 3)(*sc1.nelem)
    prec = dgmod.DG_FP32 if precision == "fp32" else dgmod.DG_FP64
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for sc in (sc1, sc2):
        u = torch.from_numpy(sc.u).cuda()
        ref = ctx.rhs(u).cpu().numpy()
        du = torch.full_like(u, float("nan"))
        st = dgmod.dg_rhs_noalloc(3, nelem, 3, prec, dgmod.DG_SURF_EC_LLF, 1.4, _ptr(u), _ptr(Ja), _ptr(invJ),
                                  _ptr(du), _ptr(flag), stream)
        assert st == dgmod.DG_OK, dgmod.dg_status_string(st)
        torch.cuda.synchronize()
        got = du.cpu().numpy()
        assert int(flag.item()) == 0
        # same tolerance as the FP64 parity tests, per variable against the magnitude of the RHS
        for c in range(5):
            scale = np.max(np.abs(ref[:, c]))
            assert np.max(np.abs(got[:, c] - ref[:, c])) <= 1e-12 * scale, c


def test_noalloc_flags_nonphysical_states_and_rejects_bad_sizes(dgmod):
    import torch
    sc = Scenario(2, [3, 2], 4, mapping="sine", ic="smooth", llf=True, seed=32)
    ctx = dgmod.DG(**sc.dg_kwargs())
    Ja_h, J_h = ctx.metrics()
    Ja = torch.from_numpy(Ja_h).cuda()
    invJ = torch.from_numpy(1.0 / J_h).cuda()
    u = torch.from_numpy(sc.u).cuda()
    u[0, 0, 3] = -1.0
    du = torch.empty_like(u)
    flag = torch.zeros(1, dtype=torch.int32, device="cuda")
    nelem = (ctypes.c_int * 3)(3, 2, 1)
    st = dgmod.dg_rhs_noalloc(2, nelem, 4, dgmod.DG_FP64, dgmod.DG_SURF_EC_LLF, 1.4, _ptr(u), _ptr(Ja), _ptr(invJ),
                              _ptr(du), _ptr(flag), None)
    assert st == dgmod.DG_OK
    torch.cuda.synchronize()
    assert int(flag.item()) != 0
    # interface fluxes of 64^3 elements at p = 3 (FP64) exceed the fixed array: rejected before any work
    big = (ctypes.c_int * 3)(64, 64, 64)
    st = dgmod.dg_rhs_noalloc(3, big, 3, dgmod.DG_FP64, dgmod.DG_SURF_EC_LLF, 1.4, _ptr(u), _ptr(Ja), _ptr(invJ),
                              _ptr(du), None, None)
    assert st == dgmod.DG_ERR_UNSUPPORTED
    st = dgmod.dg_rhs_noalloc(3, nelem, 3, dgmod.DG_FP64, dgmod.DG_SURF_EC_LLF, 1.4, _ptr(u), _ptr(Ja), _ptr(invJ),
                              _ptr(u), None, None)
    assert st == dgmod.DG_ERR_ARG  # u and du are the same array
