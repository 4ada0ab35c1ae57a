"""Pins of the Legendre-Gauss collocation oracle (oracle/gauss.c; Sec. 6) to what the paper and the mathematics fix:
closed-form Gauss rules, quadrature exactness, the generalized SBP property of (M, D, R, B), the inverse entropy
map, and, for the RHS with entropy projection, free-stream preservation, conservation, entropy conservation with
entropy-conservative fluxes (the property the entropy projection exists for), entropy dissipation with LLF, and
convergence to the exact -div f of a travelling density wave.
"""
import math

import numpy as np
import pytest

import oracle as orc
from paper_2112_10517_gb300 import inputs


def tensor_weights(wg, nd):
    W = wg.copy()
    for _ in range(nd - 1):
        W = np.kron(wg, W)  # node index i1 fastest
    return W


@pytest.mark.parametrize("p,xref,wref", [
    (1, [-1 / math.sqrt(3), 1 / math.sqrt(3)], [1.0, 1.0]),
    (2, [-math.sqrt(0.6), 0.0, math.sqrt(0.6)], [5 / 9, 8 / 9, 5 / 9]),
    (3, [-math.sqrt(3 / 7 + 2 / 7 * math.sqrt(1.2)), -math.sqrt(3 / 7 - 2 / 7 * math.sqrt(1.2)),
         math.sqrt(3 / 7 - 2 / 7 * math.sqrt(1.2)), math.sqrt(3 / 7 + 2 / 7 * math.sqrt(1.2))],
     [(18 - math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36, (18 + math.sqrt(30)) / 36, (18 - math.sqrt(30)) / 36]),
])
def test_gauss_closed_forms(p, xref, wref):
    x, w = orc.gauss(p)
    np.testing.assert_allclose(x, xref, rtol=0, atol=2e-16)
    np.testing.assert_allclose(w, wref, rtol=0, atol=4e-16)


@pytest.mark.parametrize("p", range(1, 8))
def test_gauss_quadrature_exact_to_degree_2p_plus_1(p):
    x, w = orc.gauss(p)
    for k in range(2 * p + 2):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) <= 4e-15, k
    # and not beyond: degree 2p + 2 is integrated inexactly
    assert abs(np.dot(w, x ** (2 * p + 2)) - 2.0 / (2 * p + 3)) > 1e-6


@pytest.mark.parametrize("p", range(1, 8))
def test_gauss_generalized_sbp(p):
    # D on Gauss nodes differentiates polynomials of degree <= p exactly, and (M, D, R, B) satisfy
    # M D + (M D)^T = R^T B R with R the Lagrange basis at -1, +1 and B = diag(-1, 1) (Sec. 6)
    x, w = orc.gauss(p)
    D = orc.dmat_nodes(p, x)
    for k in range(p + 1):
        np.testing.assert_allclose(D @ x ** k, k * x ** max(k - 1, 0) * (k > 0), rtol=0, atol=2e-12)
    R = np.stack([orc.lagrange_at(p, x, -1.0), orc.lagrange_at(p, x, 1.0)])
    for m in range(p + 1):
        np.testing.assert_allclose(R @ x ** m, [(-1.0) ** m, 1.0], rtol=0, atol=1e-13)
    M = np.diag(w)
    B = np.diag([-1.0, 1.0])
    np.testing.assert_allclose(M @ D + (M @ D).T, R.T @ B @ R, rtol=0, atol=1e-13)


@pytest.mark.parametrize("nd", [2, 3])
def test_inverse_entropy_map(nd):
    rng = np.random.Generator(np.random.PCG64(5))
    n = 2000
    rho = rng.uniform(0.2, 3.0, n)
    v = rng.uniform(-2.0, 2.0, (nd, n))
    pr = rng.uniform(0.1, 5.0, n)
    u = inputs.prim_to_cons(rho, list(v), pr, 1.4)  # [n, nvar]
    _, w = orc.entropy(u, nd)
    back = orc.cons_from_entropy(w, nd)
    np.testing.assert_allclose(back, u, rtol=2e-13, atol=0)


def gauss_case(nd, nelem, p, ic, seed=0, box=None):
    lo, hi = box if box is not None else ([-1.0] * nd, [1.0] * nd)
    xyz = orc.gauss_coords(nd, nelem, lo, hi, p)
    L = [h - l for l, h in zip(lo, hi)]
    if ic == "free_stream":
        u = inputs.free_stream(xyz)
    elif ic == "rough":
        u = inputs.smooth_random(xyz, seed=seed, lengths=L) + 0.05 * inputs.random_state(xyz, seed + 1)
    elif ic == "random":
        u = inputs.random_state(xyz, seed=seed)
    else:
        raise ValueError(ic)
    return lo, hi, xyz, u


@pytest.mark.parametrize("nd,nelem,p", [(2, [3, 4], 3), (2, [2, 3], 6), (3, [2, 3, 2], 2), (3, [2, 2, 2], 4)])
def test_gauss_free_stream(nd, nelem, p):
    lo, hi, xyz, u = gauss_case(nd, nelem, p, "free_stream")
    du = orc.gauss_rhs(nd, p, nelem, lo, hi, u)
    assert np.abs(du).max() <= 2e-13


@pytest.mark.parametrize("nd,nelem,p", [(2, [3, 4], 3), (2, [3, 2], 5), (3, [2, 3, 2], 2), (3, [2, 2, 2], 3)])
@pytest.mark.parametrize("seed", [7, 8])
def test_gauss_conservation_and_entropy(nd, nelem, p, seed):
    # smooth states with 5% nodal noise: the entropy projection extrapolates w(u) to the faces (|l_k(+-1)| > 1),
    # which for independent random nodal states can leave the admissible set (rho/p < 0) -- no face state exists
    lo, hi, xyz, u = gauss_case(nd, nelem, p, "rough", seed=seed)
    _, wg = orc.gauss(p)
    W = tensor_weights(wg, nd)
    _, wv = orc.entropy(np.ascontiguousarray(np.moveaxis(u, 1, 2)), nd)
    wv = np.moveaxis(wv, 2, 1)
    for llf in (False, True):
        du = orc.gauss_rhs(nd, p, nelem, lo, hi, u, llf=llf)
        tot = np.einsum("evi,i->v", du, W)
        ab = np.einsum("evi,i->v", np.abs(du), W)
        assert np.all(np.abs(tot) <= 1e-13 * ab), (llf, tot / ab)
        S = np.einsum("evi,evi,i->", wv, du, W)
        Sab = np.einsum("evi,evi,i->", np.abs(wv), np.abs(du), W)
        if llf:
            assert S < -1e-6 * Sab  # dissipation at interfaces
        else:
            assert abs(S) <= 1e-13 * Sab  # entropy conservation with entropy projection and EC fluxes


@pytest.mark.parametrize("nd,p,meshes", [(2, 2, (4, 8, 16)), (2, 3, (8, 16, 32)), (3, 2, (2, 4, 8))])
def test_gauss_convergence_density_wave(nd, p, meshes):
    # rho = 1 + 0.2 sin(sum x), constant v and p: du/dt = -(v . grad rho) (1, v, |v|^2/2) exactly
    v = [0.1, 0.2, 0.3][:nd]
    errs = []
    for n in meshes:
        lo, hi = [0.0] * nd, [2 * math.pi] * nd
        xyz = orc.gauss_coords(nd, [n] * nd, lo, hi, p)
        u = inputs.density_wave(xyz, amp=0.2, k=[1.0] * nd, v=v, p=1.0)
        du = orc.gauss_rhs(nd, p, [n] * nd, lo, hi, u)
        drho = -sum(v) * 0.2 * np.cos(xyz.sum(axis=1))
        ex = np.stack([drho] + [vj * drho for vj in v] + [0.5 * np.dot(v, v) * drho], axis=1)
        errs.append(np.abs(du - ex).max())
    rate = math.log2(errs[-2] / errs[-1])
    assert rate > p - 0.35, (errs, rate)


@pytest.mark.parametrize("nd,p", [(2, 2), (2, 4), (3, 2), (3, 3)])
def test_gauss_entropy_projection_exact_for_polynomial_entropy_variables(nd, p):
    # w(u) of degree <= p in every coordinate on each element: R w(u) is exact, so the projected face states are
    # u(w) evaluated at the face points (xi_n = +-1, Gauss points across)
    nelem = [2] * nd
    lo, hi = [-1.0] * nd, [1.0] * nd
    xyz = orc.gauss_coords(nd, nelem, lo, hi, p)
    X = [xyz[:, m] for m in range(nd)]

    def wfield(X):
        w0 = 0.5 + 0.1 * X[0] - 0.05 * X[1] ** 2 + 0.02 * X[0] * X[1]
        wv = [0.1 + 0.05 * X[1], 0.2 - 0.03 * X[0] ** 2, 0.05 * X[0]][:nd]
        wE = -(1.2 + 0.1 * X[0] * X[1] + 0.05 * X[-1] ** 2)
        return np.stack([w0] + wv + [wE], axis=-1)

    w = wfield(X)  # [E, Nd, nvar]
    u = np.ascontiguousarray(np.moveaxis(orc.cons_from_entropy(np.ascontiguousarray(w), nd), 2, 1))
    uf = orc.gauss_project(nd, p, u)
    x, _ = orc.gauss(p)
    N, NL = p + 1, (p + 1) ** (nd - 1)
    h = 1.0  # element size (2 elements on [-1, 1])
    for e in range(u.shape[0]):
        ec = [(e // (2 ** m)) % 2 for m in range(nd)]
        for n in range(nd):
            others = [m for m in range(nd) if m != n]
            for s in range(2):
                for t in range(NL):
                    ti = [(t // N ** k) % N for k in range(nd - 1)]
                    pt = [0.0] * nd
                    pt[n] = -1.0 + h * (ec[n] + s)
                    for k, m in enumerate(others):
                        pt[m] = -1.0 + h * (ec[m] + 0.5 * (x[ti[k]] + 1.0))
                    wexact = wfield([np.array(c) for c in pt])
                    uexact = orc.cons_from_entropy(np.ascontiguousarray(wexact[None, :]), nd)[0]
                    np.testing.assert_allclose(uf[e, (n * 2 + s) * NL + t], uexact, rtol=1e-12, atol=1e-14)
