"""Batched RHS (dg_batch_*): many meshes of uneven size and degree, one persistent volume launch per degree. Each
instance's
du must match dg_rhs on its own context (the same formulas; the compiler may contract multiply-adds differently
in the two kernels, so agreement is to rounding, measured like the parity tests) and the oracle; the autotuner's
choices must not change results beyond rounding."""
import numpy as np
import pytest

from cases import Scenario, parity_errors

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


def make_batch(dgmod, precision, specs, seed0=100, ic="smooth", **extra):
    import torch
    scs, ctxs, us, dus = [], [], [], []
    for k, (nelem, p) in enumerate(specs):
        sc = Scenario(3, nelem, p, mapping="sine", ic=ic, llf=True, seed=seed0 + k, **extra)
        ctx = dgmod.DG(precision=precision, **sc.dg_kwargs())
        scs.append(sc)
        ctxs.append(ctx)
        us.append(torch.from_numpy(sc.u).cuda())
        dus.append(torch.full_like(us[-1], float("nan")))
    return scs, ctxs, us, dus


SPECS = [([2, 3, 2], 2), ([3, 3, 3], 3), ([1, 2, 2], 5), ([4, 2, 3], 4), ([2, 2, 2], 1), ([5, 1, 3], 2),
         ([2, 2, 3], 5), ([3, 4, 2], 3)]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_matches_single_context_rhs_and_oracle(dgmod, precision):
    import torch
    scs, ctxs, us, dus = make_batch(dgmod, precision, SPECS)
    batch = dgmod.DGBatch(ctxs, us, dus)
    refs = [c.rhs(u).cpu().numpy() for c, u in zip(ctxs, us)]
    tol = 1e-12 if precision == "fp64" else 4e-6
    scales = [sc.du_scale() for sc in scs]
    for threads in (128, 192, 256):
        for cps in (0, 1):
            for d in dus:
                d.fill_(float("nan"))
            batch.set_tuning(threads, cps)
            batch.rhs()
            torch.cuda.synchronize()
            for sc, ref, d, sca in zip(scs, refs, dus, scales):
                plain, term = parity_errors(d.cpu().numpy(), ref, sca)
                assert np.all(term <= tol), (threads, cps, sc.p, term)
    for sc, d in zip(scs, dus):
        plain, term = parity_errors(d.cpu().numpy(), sc.du_ref(), sc.du_scale())
        assert np.all(term <= tol), (sc.p, term)
    for c in ctxs:
        assert c.check_status() == dgmod.DG_OK


def test_batch_autotune_and_cache(dgmod, tmp_path):
    import torch
    scs, ctxs, us, dus = make_batch(dgmod, "fp64", SPECS[:5], seed0=200)
    batch = dgmod.DGBatch(ctxs, us, dus)
    cache = str(tmp_path / "tune.txt")
    th, cps = batch.autotune(cache)
    assert th in (128, 192, 256) and cps >= 1
    text = open(cache).read()
    assert text.count("\n") == 1 and ("\t%d\t%d" % (th, cps)) in text
    # a second plan with the same signature reads the cache instead of timing
    batch2 = dgmod.DGBatch(ctxs, us, dus)
    assert batch2.autotune(cache) == (th, cps)
    assert open(cache).read() == text
    batch.rhs()
    torch.cuda.synchronize()
    for sc, c, u, d in zip(scs, ctxs, us, dus):
        plain, term = parity_errors(d.cpu().numpy(), c.rhs(u).cpu().numpy(), sc.du_scale())
        assert np.all(term <= 1e-12), term


def test_batch_rejects_mixed_precision_and_high_degree(dgmod):
    import ctypes
    import torch
    _, c64, u64, d64 = make_batch(dgmod, "fp64", SPECS[:1])
    _, c32, u32, d32 = make_batch(dgmod, "fp32", SPECS[:1])
    with pytest.raises(dgmod.DGError) as ei:
        dgmod.DGBatch(c64 + c32, u64 + u32, d64 + d32)
    assert ei.value.status == dgmod.DG_ERR_ARG
    _, c7, u7, d7 = make_batch(dgmod, "fp64", [([1, 1, 2], 6)])
    with pytest.raises(dgmod.DGError) as ei:
        dgmod.DGBatch(c7, u7, d7)
    assert ei.value.status == dgmod.DG_ERR_UNSUPPORTED


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_with_precomputed_logarithms(dgmod, precision):
    # contexts with precompute_logs: the batch runs the per-node-logarithm kernels (Sec. 7.2); rough states take the
    # log branches
    import torch
    scs, ctxs, us, dus = make_batch(dgmod, precision, SPECS, seed0=300, ic="rough", precompute_logs=True)
    batch = dgmod.DGBatch(ctxs, us, dus)
    tol = 1e-12 if precision == "fp64" else 4e-6
    for threads in (128, 256):
        batch.set_tuning(threads, 0)
        batch.rhs()
        torch.cuda.synchronize()
        for sc, c, u, d in zip(scs, ctxs, us, dus):
            _, term = parity_errors(d.cpu().numpy(), c.rhs(u).cpu().numpy(), sc.du_scale())
            assert np.all(term <= tol), (threads, sc.p, term)
            _, term = parity_errors(d.cpu().numpy(), sc.du_ref(), sc.du_scale())
            assert np.all(term <= tol), (threads, sc.p, term)
    # contexts must agree on the log-mean variant
    _, c1, u1, d1 = make_batch(dgmod, precision, SPECS[:1], seed0=400)
    with pytest.raises(dgmod.DGError) as ei:
        dgmod.DGBatch(ctxs[:1] + c1, us[:1] + u1, dus[:1] + d1)
    assert ei.value.status == dgmod.DG_ERR_ARG


def test_batch_rhs_in_a_cuda_graph(dgmod):
    # dg_batch_rhs issues launches only (no allocation, no synchronization, no attribute calls after the first
    # call), so a captured batch RHS replays the same kernels: bitwise equal to the eager call
    import torch
    scs, ctxs, us, dus = make_batch(dgmod, "fp64", SPECS, seed0=500)
    batch = dgmod.DGBatch(ctxs, us, dus)
    batch.set_tuning(192, 0)
    batch.rhs()
    torch.cuda.synchronize()
    eager = [d.clone() for d in dus]
    for d in dus:
        d.fill_(float("nan"))
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        batch.rhs(stream=side)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(eager, dus):
        assert torch.equal(a, b)
