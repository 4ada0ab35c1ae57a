"""Pins of the CPU oracle to facts fixed outside it (closed forms, invariants the paper states, exact
solutions, brute force on tiny inputs). No GPU. Each test names the passage of the paper it follows.

A plausible mistake anywhere in the oracle (a dropped term, a wrong sign or index, a transposed
operand) fails at least one of these: see the comments on each group.
"""
import math
import os

import numpy as np
import pytest

import oracle as orc
from paper_2112_10517_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
G = 1.4


def random_states(n, nd, seed, rho=(0.5, 2.0), vmax=1.0, p=(0.5, 2.0)):
    rng = np.random.Generator(np.random.PCG64(seed))
    r = rng.uniform(*rho, size=n)
    v = [rng.uniform(-vmax, vmax, size=n) for _ in range(nd)]
    pp = rng.uniform(*p, size=n)
    u = inputs.prim_to_cons(r[:, None], [vj[:, None] for vj in v], pp[:, None])  # [n, nvar, 1]
    return np.ascontiguousarray(u[:, :, 0])


# ------------------------------------------------------------------------------------------------
# Reference element (Sec. 2: Def. derivative matrix, Def. SBP operator, LGL example)
# ------------------------------------------------------------------------------------------------

def test_lgl_closed_forms():
    rows = []
    with open(os.path.join(GOLDEN, "lgl_closed_forms.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            p, xs, ws = line.split()
            rows.append((int(p), eval(xs, {"sqrt": math.sqrt}), eval(ws, {"sqrt": math.sqrt})))
    for p in sorted({r[0] for r in rows}):
        x, w = orc.lgl(p)
        xe = np.array([r[1] for r in rows if r[0] == p])
        we = np.array([r[2] for r in rows if r[0] == p])
        np.testing.assert_allclose(x, xe, rtol=0, atol=2e-16)
        np.testing.assert_allclose(w, we, rtol=4e-16, atol=0)


@pytest.mark.parametrize("p", range(1, 15))
def test_lgl_quadrature_exact_to_degree_2p_minus_1(p):
    x, w = orc.lgl(p)
    for k in range(2 * p):
        exact = (1.0 - (-1.0) ** (k + 1)) / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 2e-15, (p, k)
    # degree 2p is NOT integrated exactly by Lobatto quadrature (sanity: the nodes are not Gauss nodes)
    assert abs(np.dot(w, x ** (2 * p)) - 2.0 / (2 * p + 1)) > 1e-12


@pytest.mark.parametrize("p", range(1, 15))
def test_dmat_differentiates_polynomials(p):
    # Def. derivative matrix: D x^k = k x^(k-1) for k <= p
    x, _ = orc.lgl(p)
    D = orc.dmat(p)
    for k in range(p + 1):
        lhs = D @ x ** k
        rhs = k * x ** (k - 1) if k > 0 else np.zeros_like(x)
        np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * max(1, p ** 2))


@pytest.mark.parametrize("p", range(1, 15))
def test_sbp_property(p):
    # Eq. SBP in 1D: M D + D^T M = R^T B N R = diag(-1, 0, ..., 0, 1)
    _, w = orc.lgl(p)
    D = orc.dmat(p)
    M = np.diag(w)
    B = np.zeros((p + 1, p + 1))
    B[0, 0], B[-1, -1] = -1.0, 1.0
    np.testing.assert_allclose(M @ D + D.T @ M, B, rtol=0, atol=2e-13 * max(1, p ** 2))


# ------------------------------------------------------------------------------------------------
# Logarithmic mean (Sec. 3.1, Eq. logmean)
# ------------------------------------------------------------------------------------------------

def test_logmean_special_cases():
    assert orc.logmean([3.7], [3.7])[0] == 3.7
    np.testing.assert_allclose(orc.logmean([1.0], [math.e]), [math.e - 1.0], rtol=2e-16)
    np.testing.assert_allclose(orc.logmean([1.0], [4.0]), [3.0 / math.log(4.0)], rtol=4e-16)
    a = np.array([0.3, 1.0, 7.0]); b = np.array([0.9, 1.0 + 1e-12, 2.0])
    np.testing.assert_allclose(orc.logmean(5.0 * a, 5.0 * b), 5.0 * orc.logmean(a, b), rtol=4e-16)
    np.testing.assert_allclose(orc.logmean(a, b), orc.logmean(b, a), rtol=4e-16, atol=0)


def test_logmean_against_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.Generator(np.random.PCG64(1))
    ratios = np.concatenate([1.0 + np.logspace(-15, 1, 400), 1.0 - np.logspace(-15, -0.01, 200)])
    a = rng.uniform(0.1, 10.0, size=ratios.size)
    b = a * ratios
    got = orc.logmean(a, b)
    worst = 0.0
    for ai, bi, gi in zip(a, b, got):
        A, B = mpmath.mpf(float(ai)), mpmath.mpf(float(bi))
        ref = A if A == B else (B - A) / (mpmath.log(B) - mpmath.log(A))
        worst = max(worst, float(abs((mpmath.mpf(float(gi)) - ref) / ref)))
    assert worst < 1e-15, worst


def test_logmean_derivatives_against_high_precision():
    # the dual-number derivatives of the oracle's mean (used by its JVP), including arguments equal to rounding
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    rng = np.random.Generator(np.random.PCG64(5))
    ratios = np.concatenate([1.0 + np.logspace(-16, 0.5, 120), 1.0 - np.logspace(-16, -0.1, 60), [1.0]])
    a = rng.uniform(0.2, 5.0, size=ratios.size)
    b = a * ratios
    ga, gb = orc.logmean_grad(a, b)
    for x, y, da, db in zip(a, b, ga, gb):
        X, Y = mpmath.mpf(float(x)), mpmath.mpf(float(y))
        if X == Y:
            ra = rb = mpmath.mpf(0.5)
        else:
            ln = mpmath.log(Y) - mpmath.log(X)
            ra = ((Y - X) / X - ln) / ln ** 2
            rb = (ln - (Y - X) / Y) / ln ** 2
        assert abs(da - float(ra)) <= 2e-14 and abs(db - float(rb)) <= 2e-14, (x, y, da, float(ra), db, float(rb))


# ------------------------------------------------------------------------------------------------
# Euler flux (Eq. Euler): pinned by the eigenvalues of its Jacobian, v.n and v.n +- c|n|.
# A wrong sign or a dropped pressure term anywhere changes them.
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd", [2, 3])
def test_euler_flux_jacobian_eigenvalues(nd):
    nv = nd + 2
    u = random_states(6, nd, seed=2)
    rng = np.random.Generator(np.random.PCG64(3))
    for s in range(u.shape[0]):
        n = rng.standard_normal(nd)
        A = np.zeros((nv, nv))
        for c in range(nv):
            h = 1e-6 * max(1.0, abs(u[s, c]))
            up = u[s].copy(); up[c] += h
            um = u[s].copy(); um[c] -= h
            fp = sum(n[j] * orc.euler_flux(up[None], j, nd)[0] for j in range(nd))
            fm = sum(n[j] * orc.euler_flux(um[None], j, nd)[0] for j in range(nd))
            A[:, c] = (fp - fm) / (2 * h)
        rho = u[s, 0]; v = u[s, 1:nd + 1] / rho
        p = (G - 1) * (u[s, -1] - 0.5 * rho * v @ v)
        c_s = math.sqrt(G * p / rho)
        vn = v @ n
        expected = np.sort([vn - c_s * np.linalg.norm(n)] + [vn] * nd + [vn + c_s * np.linalg.norm(n)])
        got = np.sort(np.linalg.eigvals(A).real)
        np.testing.assert_allclose(got, expected, rtol=0, atol=1e-6)


# ------------------------------------------------------------------------------------------------
# Entropy pair (Sec. 2): w = dU/du, and the flux potential psi^j = w.f^j - F^j equals rho v_j.
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd", [2, 3])
def test_entropy_variables_are_the_gradient(nd):
    u = random_states(20, nd, seed=4)
    U, w = orc.entropy(u, nd)
    for c in range(nd + 2):
        h = 1e-6 * np.maximum(1.0, np.abs(u[:, c]))
        up = u.copy(); up[:, c] += h
        um = u.copy(); um[:, c] -= h
        dU = (orc.entropy(up, nd)[0] - orc.entropy(um, nd)[0]) / (2 * h)
        np.testing.assert_allclose(w[:, c], dU, rtol=1e-7, atol=1e-8)


@pytest.mark.parametrize("nd", [2, 3])
def test_flux_potential_closed_form(nd):
    u = random_states(50, nd, seed=5)
    U, w = orc.entropy(u, nd)
    rho = u[:, 0]
    for j in range(nd):
        f = orc.euler_flux(u, j, nd)
        vj = u[:, 1 + j] / rho
        psi = np.sum(w * f, axis=1) - U * vj  # w.f^j - F^j with F^j = U v_j
        np.testing.assert_allclose(psi, u[:, 1 + j], rtol=1e-12, atol=1e-13)


# ------------------------------------------------------------------------------------------------
# Ranocha flux (Eq. flux_ranocha) and the surface flux: Def. numerical-fluxes and Def. EC/ED.
# The EC identity fails for a dropped or mis-signed term in any component.
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd", [2, 3])
def test_ranocha_consistency_and_symmetry(nd):
    n = 2000
    a = random_states(n, nd, seed=6)
    b = random_states(n, nd, seed=7)
    m = np.random.Generator(np.random.PCG64(8)).standard_normal((n, nd))
    fa = orc.flux_ranocha(a, a, m, nd)
    phys = sum(m[:, j:j + 1] * orc.euler_flux(a, j, nd) for j in range(nd))
    np.testing.assert_allclose(fa, phys, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(orc.flux_ranocha(a, b, m, nd), orc.flux_ranocha(b, a, m, nd),
                               rtol=1e-14, atol=1e-14)
    # linear in the direction
    np.testing.assert_allclose(orc.flux_ranocha(a, b, 2.5 * m, nd), 2.5 * orc.flux_ranocha(a, b, m, nd),
                               rtol=1e-14, atol=1e-14)


@pytest.mark.parametrize("nd", [2, 3])
def test_ranocha_is_entropy_conservative(nd):
    n = 20000
    a = random_states(n, nd, seed=9)
    b = random_states(n, nd, seed=10)
    m = np.random.Generator(np.random.PCG64(11)).standard_normal((n, nd))
    f = orc.flux_ranocha(a, b, m, nd)
    _, wa = orc.entropy(a, nd)
    _, wb = orc.entropy(b, nd)
    psi_jump = np.sum(m * (b[:, 1:nd + 1] - a[:, 1:nd + 1]), axis=1)  # psi^j = rho v_j
    r = np.sum((wb - wa) * f, axis=1) - psi_jump
    scale = np.sum(np.abs((wb - wa) * f), axis=1) + np.abs(psi_jump)
    assert np.max(np.abs(r) / scale) < 1e-13


@pytest.mark.parametrize("nd", [2, 3])
def test_ranocha_kinetic_energy_and_pressure_structure(nd):
    n = 500
    a = random_states(n, nd, seed=12)
    b = random_states(n, nd, seed=13)
    m = np.random.Generator(np.random.PCG64(14)).standard_normal((n, nd))
    f = orc.flux_ranocha(a, b, m, nd)
    va = a[:, 1:nd + 1] / a[:, :1]
    vb = b[:, 1:nd + 1] / b[:, :1]
    pa = (G - 1) * (a[:, -1] - 0.5 * np.sum(a[:, 1:nd + 1] * va, axis=1))
    pb = (G - 1) * (b[:, -1] - 0.5 * np.sum(b[:, 1:nd + 1] * vb, axis=1))
    # KEP: f_rhov = f_rho {{v}} + {{p}} m
    np.testing.assert_allclose(f[:, 1:nd + 1], f[:, :1] * 0.5 * (va + vb) + 0.5 * (pa + pb)[:, None] * m,
                               rtol=1e-13, atol=1e-13)
    # mass flux: {{rho}}_log {{v.m}}
    lm = orc.logmean(a[:, 0], b[:, 0])
    np.testing.assert_allclose(f[:, 0], lm * 0.5 * np.sum((va + vb) * m, axis=1), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("nd", [2, 3])
def test_llf_surface_flux_properties(nd):
    n = 5000
    a = random_states(n, nd, seed=15)
    b = random_states(n, nd, seed=16)
    m = np.random.Generator(np.random.PCG64(17)).standard_normal((n, nd))
    fab = orc.surface_flux(a, b, m, nd, llf=True)
    # consistency and directional anti-symmetry (Def. numerical-fluxes)
    phys = sum(m[:, j:j + 1] * orc.euler_flux(a, j, nd) for j in range(nd))
    np.testing.assert_allclose(orc.surface_flux(a, a, m, nd, llf=True), phys, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(fab, -orc.surface_flux(b, a, -m, nd, llf=True), rtol=1e-14, atol=1e-14)
    # entropy dissipative (Def. EC/ED): [w].f* - [psi].m <= 0
    _, wa = orc.entropy(a, nd)
    _, wb = orc.entropy(b, nd)
    psi_jump = np.sum(m * (b[:, 1:nd + 1] - a[:, 1:nd + 1]), axis=1)
    r = np.sum((wb - wa) * fab, axis=1) - psi_jump
    assert np.all(r <= 1e-12 * (1 + np.abs(psi_jump)))
    assert np.mean(r < -1e-10) > 0.99  # strictly dissipative for distinct states
    # the dissipation is lambda/2 [u] with lambda the largest |v.m| + c|m|
    diss = orc.flux_ranocha(a, b, m, nd) - fab
    ratio = diss / (b - a)
    np.testing.assert_allclose(ratio, np.repeat(ratio[:, :1], nd + 2, axis=1), rtol=1e-9, atol=1e-12)


# ------------------------------------------------------------------------------------------------
# Metric terms (Sec. 2.3)
# ------------------------------------------------------------------------------------------------

def _apply_dir(D, g, nd, N, n):
    """Apply 1D D along reference direction n to nodal arrays g[..., Nd] (i1 fastest)."""
    shape = g.shape[:-1] + (N,) * nd
    gt = g.reshape(shape)
    axis = g.ndim - 1 + (nd - 1 - n)
    out = np.moveaxis(np.tensordot(D, np.moveaxis(gt, axis, 0), axes=(1, 0)), 0, axis)
    return out.reshape(g.shape)


@pytest.mark.parametrize("nd", [2, 3])
def test_affine_metrics(nd):
    p = 3
    nelem = [3, 4, 5][:nd]
    lo, hi = [-1.0, -2.0, 0.0][:nd], [1.0, 2.0, 5.0][:nd]
    xyz = orc.coords(nd, nelem, lo, hi, p)
    Ja, J = orc.metrics(nd, p, xyz)
    h = [(hi[m] - lo[m]) / nelem[m] / 2 for m in range(nd)]
    np.testing.assert_allclose(J, np.prod(h), rtol=1e-13)
    for n in range(nd):
        for j in range(nd):
            expected = np.prod(h) / h[n] if n == j else 0.0
            np.testing.assert_allclose(Ja[:, n, j], expected, rtol=1e-13, atol=1e-13 * np.max(np.abs(Ja)))


def test_curl_metrics_satisfy_discrete_identity_and_converge():
    nd, nelem = 3, [2, 2, 2]
    lo, hi = [-math.pi] * 3, [math.pi] * 3
    errs = []
    for p in [2, 4, 6, 8]:
        N = p + 1
        D = orc.dmat(p)
        xyz = orc.coords(nd, nelem, lo, hi, p, mapping=1, amp=0.1)
        Ja, J = orc.metrics(nd, p, xyz, curl_form=True)
        for j in range(3):
            div = sum(_apply_dir(D, Ja[:, n, j], nd, N, n) for n in range(3))
            assert np.max(np.abs(div)) < 1e-13 * max(1, p ** 2), (p, j)
        # continuous metric of the sine mapping: x = xi + a prod sin(xi_k); Ja^n = a_{n+1} x a_{n+2}
        # with a_k = dx/dxi_k (physical xi); reference derivatives add the factor h/2 per direction
        hh = (2 * math.pi / 2) / 2
        xg, _ = orc.lgl(p)
        Ja_ex = np.zeros_like(Ja)
        E = xyz.shape[0]
        for e in range(E):
            eidx = [e % 2, (e // 2) % 2, e // 4]
            for i in range(N ** 3):
                ii = [i % N, (i // N) % N, i // (N * N)]
                xi = [lo[m] + 2 * hh * (eidx[m] + 0.5 * (xg[ii[m]] + 1)) for m in range(3)]
                s = [math.sin(v) for v in xi]
                c = [math.cos(v) for v in xi]
                grad = [0.1 * c[0] * s[1] * s[2], 0.1 * s[0] * c[1] * s[2], 0.1 * s[0] * s[1] * c[2]]
                a = np.array([[(1.0 if m == k else 0.0) + grad[k] for m in range(3)] for k in range(3)]) * hh
                for n in range(3):
                    Ja_ex[e, n, :, i] = np.cross(a[(n + 1) % 3], a[(n + 2) % 3])
        errs.append(np.max(np.abs(Ja - Ja_ex)))
    # spectral convergence of the discrete metric to the exact one as p grows
    assert all(a > 10 * b for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-4, errs


def twisted_coords(nd, nelem, p, amp=0.1):
    """Affine nodes on [-pi, pi]^d moved by a smooth periodic map with a different perturbation per
    component. (The sine mapping x_m = xi_m + a prod sin(xi_k) moves every component by the same
    scalar, so even cross-product metrics satisfy the discrete identities on it.)"""
    xyz = orc.coords(nd, nelem, [-math.pi] * nd, [math.pi] * nd, p)
    X = [xyz[:, m].copy() for m in range(nd)]
    out = np.empty_like(xyz)
    for m in range(nd):
        a, b = X[(m + 1) % nd], X[(m + 2) % nd] if nd == 3 else X[m]
        out[:, m] = X[m] + amp * np.sin(a) * np.cos(b + 0.3 * m)
    return out


def test_cross_product_metrics_break_the_identity():
    # negative control: on a general curved mesh the cross-product form violates the discrete identity
    p, nd, N = 3, 3, 4
    D = orc.dmat(p)
    xyz = twisted_coords(nd, [2, 2, 2], p)
    Ja, _ = orc.metrics(nd, p, xyz, curl_form=False)
    div = sum(_apply_dir(D, Ja[:, n, 0], nd, N, n) for n in range(3))
    assert np.max(np.abs(div)) > 1e-6
    Ja, _ = orc.metrics(nd, p, xyz, curl_form=True)
    for j in range(3):
        div = sum(_apply_dir(D, Ja[:, n, j], nd, N, n) for n in range(3))
        assert np.max(np.abs(div)) < 1e-13


# ------------------------------------------------------------------------------------------------
# Semidiscretization (Eq. strong-form-SBP + Eq. fluxdiff-SBP): invariants the paper states
# ------------------------------------------------------------------------------------------------

def mesh(nd, nelem, p, curved, box=None):
    lo, hi = box if box is not None else ([-math.pi] * nd, [math.pi] * nd)
    xyz = orc.coords(nd, nelem, lo, hi, p, mapping=1 if curved else 0, amp=0.1 if curved else 0.0)
    Ja, J = orc.metrics(nd, p, xyz)
    return xyz, Ja, J


@pytest.mark.parametrize("nd,nelem,p", [(2, [4, 3], 3), (3, [3, 2, 3], 2)])
@pytest.mark.parametrize("curved", [False, True])
def test_free_stream_preservation(nd, nelem, p, curved):
    xyz, Ja, J = mesh(nd, nelem, p, curved)
    u = inputs.free_stream(xyz)
    for llf in (False, True):
        du = orc.rhs(nd, p, nelem, Ja, J, u, llf=llf)
        scale = orc.rhs(nd, p, nelem, Ja, J, u, llf=llf, scale=True)
        assert np.max(np.abs(du)) < 1e-12
        assert np.max(np.abs(du)) < 1e-13 * np.max(scale)


def test_free_stream_on_twisted_mesh_needs_curl_metrics():
    nd, nelem, p = 3, [3, 2, 3], 3
    xyz = twisted_coords(nd, nelem, p)
    Ja, J = orc.metrics(nd, p, xyz, curl_form=True)
    du = orc.rhs(nd, p, nelem, Ja, J, inputs.free_stream(xyz))
    assert np.max(np.abs(du)) < 1e-12
    Ja, J = orc.metrics(nd, p, xyz, curl_form=False)
    du = orc.rhs(nd, p, nelem, Ja, J, inputs.free_stream(xyz))
    assert np.max(np.abs(du)) > 1e-8


@pytest.mark.parametrize("nd,nelem,p", [(2, [4, 3], 3), (3, [3, 2, 3], 3)])
@pytest.mark.parametrize("llf", [False, True])
def test_discrete_conservation(nd, nelem, p, llf):
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u = inputs.smooth_random(xyz, seed=3)
    u = u + 0.01 * inputs.random_state(xyz, seed=4)  # non-smooth part: exercises every flux term
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=llf)
    tot, ab = orc.integrate(nd, p, J, du)
    assert np.all(np.abs(tot) <= 1e-13 * ab), (tot, ab)


@pytest.mark.parametrize("nd,nelem,p", [(2, [4, 3], 3), (3, [3, 2, 3], 3)])
def test_entropy_conservation_and_dissipation(nd, nelem, p):
    # EC volume + EC surface flux => semi-discrete entropy conservation (Sec. 2, after Eq. fluxdiff-SBP);
    # the LLF surface flux is ED => dS/dt <= 0
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u = inputs.random_state(xyz, seed=5)
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=False)
    s, ab = orc.entropy_rate(nd, p, J, u, du)
    assert abs(s) <= 1e-13 * ab, (s, ab)
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=True)
    s, ab = orc.entropy_rate(nd, p, J, u, du)
    assert s < -1e-6 * ab


@pytest.mark.parametrize("nd,nelem,p", [(2, [4, 3], 3), (3, [3, 2, 3], 2)])
@pytest.mark.parametrize("curved", [False, True])
def test_pressure_equilibrium(nd, nelem, p, curved):
    # Ranocha's flux preserves pressure equilibria (Sec. 3.2): v, p constant stay constant
    xyz, Ja, J = mesh(nd, nelem, p, curved)
    v = [0.1, -0.2, 0.3][:nd]
    u = inputs.pressure_equilibrium(xyz, seed=6, v=v)
    for llf in (False, True):
        du = orc.rhs(nd, p, nelem, Ja, J, u, llf=llf)
        scale = np.max(np.abs(du[:, 0]))
        assert scale > 1e-3
        for j in range(nd):
            np.testing.assert_allclose(du[:, 1 + j], v[j] * du[:, 0], rtol=0, atol=1e-12 * scale)
        np.testing.assert_allclose(du[:, -1], 0.5 * np.dot(v, v) * du[:, 0], rtol=0, atol=1e-12 * scale)


@pytest.mark.parametrize("nd,nelem,p", [(2, [4, 3], 3), (3, [3, 2, 3], 3)])
@pytest.mark.parametrize("curved", [False, True])
def test_mass_and_momentum_rhs_ignore_a_constant_pressure_shift(nd, nelem, p, curved):
    # Ranocha's mass flux rho_log {{v}}.n does not involve p and its momentum flux f_rho {{v}} + {{p}} n changes by
    # dp {{n}} when p -> p + dp: with the EC surface flux that part of the RHS is dp times the free-stream
    # residual (volume terms and lifted surface terms of a constant, cancelled by the discrete metric identities),
    # so the mass and momentum RHS stay the same up to rounding. The energy RHS changes (p {{v.n}} terms), and the
    # LLF dissipation changes with the sound speed: both must differ (controls).
    xyz, Ja, J = mesh(nd, nelem, p, curved)
    u = inputs.smooth_random(xyz, seed=21) + 0.01 * inputs.random_state(xyz, seed=22)  # jumps at interfaces
    dp = 25.0
    v = u.copy()
    v[:, -1] += dp / (G - 1.0)  # E = p/(gamma - 1) + rho |v|^2 / 2: p -> p + dp at fixed rho, v
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=False)
    dv = orc.rhs(nd, p, nelem, Ja, J, v, llf=False)
    scale = orc.rhs(nd, p, nelem, Ja, J, v, llf=False, scale=True)
    for c in range(nd + 1):
        assert np.max(np.abs(dv[:, c] - du[:, c])) <= 1e-13 * np.max(scale[:, c]), c
    assert np.max(np.abs(dv[:, -1] - du[:, -1])) > 1e-6 * np.max(scale[:, -1])
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=True)
    dv = orc.rhs(nd, p, nelem, Ja, J, v, llf=True)
    assert np.max(np.abs(dv[:, 0] - du[:, 0])) > 1e-6 * np.max(scale[:, 0])


def test_scale_mode_bounds_the_rhs():
    # scale = (1/J) sum |terms| >= |(1/J) sum terms| = |du| at every node (triangle inequality), and it is
    # equal for a single term: free stream on an affine mesh makes every term cancel against another one
    nd, nelem, p = 3, [3, 2, 3], 3
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u = inputs.smooth_random(xyz, seed=3)
    du = orc.rhs(nd, p, nelem, Ja, J, u)
    sc = orc.rhs(nd, p, nelem, Ja, J, u, scale=True)
    assert np.all(sc >= np.abs(du) * (1 - 1e-14))
    assert np.all(sc > 0)


# ---- exact time derivatives of smooth solutions: pins every term of the RHS on curved meshes ----

def _sympy_euler_dudt(nd, prim_exprs, X, gamma=G):
    """-div f(u) for primitive fields given as sympy expressions of the coordinates X."""
    sp = pytest.importorskip("sympy")
    rho, v, p = prim_exprs
    E = p / (gamma - 1) + rho * sum(vi ** 2 for vi in v) / 2
    flux = []
    for j in range(nd):
        fj = [rho * v[j]] + [rho * v[j] * v[i] + (p if i == j else 0) for i in range(nd)] + [(E + p) * v[j]]
        flux.append(fj)
    dudt = [-sum(sp.diff(flux[j][c], X[j]) for j in range(nd)) for c in range(nd + 2)]
    return [sp.lambdify(X, expr, "numpy") for expr in dudt]


def _eval(fns, xyz):
    cols = [xyz[:, m, :] for m in range(xyz.shape[1])]
    return np.stack([np.broadcast_to(f(*cols), cols[0].shape) for f in fns], axis=1)


def test_rhs_converges_to_exact_derivative_tgv_curved():
    # the semidiscretization is consistent with -div f(u) to the order of D (Sec. 2, after
    # Eq. fluxdiff-SBP): the pointwise RHS error of a smooth field decays like h^p on the curved mesh.
    # Mach 0.5 keeps the energy equation's cancellation (p/(gamma-1) div v) out of the rate.
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    M = 0.5
    prim = (sp.Integer(1), [sp.sin(x) * sp.cos(y) * sp.cos(z), -sp.cos(x) * sp.sin(y) * sp.cos(z), sp.Integer(0)],
            1 / (G * M ** 2) + (sp.cos(2 * x) + sp.cos(2 * y)) * (sp.cos(2 * z) + 2) / 16)
    fns = _sympy_euler_dudt(3, prim, (x, y, z))
    p = 3
    errs = []
    for ne in [8, 16]:
        nelem = [ne] * 3
        xyz, Ja, J = mesh(3, nelem, p, True)
        u = inputs.taylor_green(xyz, mach=M)
        du = orc.rhs(3, p, nelem, Ja, J, u, llf=True)
        ex = _eval(fns, xyz)
        errs.append(np.array([np.max(np.abs(du[:, c] - ex[:, c])) for c in range(5)]))
    order = np.log2(errs[0] / errs[1])
    assert np.all(order > p - 0.6), (errs, order)
    assert np.max(errs[1][1:4]) < 5e-3


def test_rhs_converges_to_exact_derivative_vortex_2d_curved():
    # exact solution u(x - v0 t): du/dt = -v0 . grad u (Sec. 4.1 isentropic vortex, planar)
    sp = pytest.importorskip("sympy")
    x, y = sp.symbols("x y")
    eps, g = 5.0, G
    r2 = x ** 2 + y ** 2
    T = 10.0 - (g - 1) * eps ** 2 / (8 * g * sp.pi ** 2) * sp.exp(1 - r2)
    rho = (T / 10.0) ** (1 / (g - 1))
    gg = eps / (2 * sp.pi) * sp.exp((1 - r2) / 2)
    prim = (rho, [1 - gg * y, 1 + gg * x], rho * T)
    fns = _sympy_euler_dudt(2, prim, (x, y))
    box = ([-10.0, -10.0], [10.0, 10.0])
    errs = []
    for p in [3, 5, 7]:
        nelem = [16, 16]
        xyz = orc.coords(2, nelem, box[0], box[1], p, mapping=1, amp=0.1)
        Ja, J = orc.metrics(2, p, xyz)
        u = inputs.isentropic_vortex(xyz, eps=eps)
        du = orc.rhs(2, p, nelem, Ja, J, u, llf=True)
        ex = _eval(fns, xyz)
        errs.append(max(np.max(np.abs(du[:, c] - ex[:, c])) / np.max(np.abs(ex[:, c])) for c in range(4)))
    # spectral convergence in p at fixed mesh
    assert errs[0] > 8 * errs[1] > 64 * errs[2] and errs[2] < 1e-3, errs


# ---- brute force on a tiny mesh: the RHS from dense curved SBP operators (Eq. curved-SBP-operators) ----

def test_rhs_matches_dense_curved_sbp_formulation():
    nd, nelem, p = 2, [2, 3], 2
    N = p + 1
    Nd = N ** nd
    nv = nd + 2
    xyz = orc.coords(nd, nelem, [-1.0, -1.0], [1.0, 1.0], p, mapping=1, amp=0.15)
    Ja, J = orc.metrics(nd, p, xyz)
    u = inputs.smooth_random(xyz, seed=9, lengths=[2.0, 2.0]) + 0.02 * inputs.random_state(xyz, seed=10)
    x1, w1 = orc.lgl(p)
    D1 = orc.dmat(p)
    I = np.eye(N)
    Dref = [np.kron(I, D1), np.kron(D1, I)]  # node i = i1 + N i2: D along xi_1 acts on i1
    W = np.kron(w1, w1)  # tensor weights, same node order
    E = xyz.shape[0]
    du = np.zeros_like(u)
    for e in range(E):
        e1, e2 = e % nelem[0], e // nelem[0]
        Dx = []
        for j in range(nd):
            Dj = np.zeros((Nd, Nd))
            for n in range(nd):
                A = np.diag(Ja[e, n, j])
                Dj += A @ Dref[n] + Dref[n] @ A
            Dx.append(0.5 * np.diag(1.0 / J[e]) @ Dj)
        ue = u[e].T  # [Nd, nv]
        vol = np.zeros((Nd, nv))
        for i in range(Nd):
            for k in range(Nd):
                for j in range(nd):
                    if Dx[j][i, k] != 0.0:
                        ej = np.eye(nd)[j]
                        vol[i] += 2 * Dx[j][i, k] * orc.flux_ranocha(ue[i:i + 1], ue[k:k + 1], ej[None], nd)[0]
        surf = np.zeros((Nd, nv))
        for i in range(Nd):
            ii = [i % N, i // N]
            for n in range(nd):
                for side, face_idx in ((+1, p), (-1, 0)):
                    if ii[n] != face_idx:
                        continue
                    nb = [e1, e2]
                    nb[n] = (nb[n] + side) % nelem[n]
                    enb = nb[0] + nelem[0] * nb[1]
                    jj = list(ii)
                    jj[n] = 0 if side > 0 else p
                    inb = jj[0] + N * jj[1]
                    m = side * Ja[e, n, :, i]
                    fstar = orc.surface_flux(ue[i:i + 1], u[enb][:, inb][None], m[None], nd, llf=True)[0]
                    fn = sum(m[j] * orc.euler_flux(ue[i:i + 1], j, nd)[0] for j in range(nd))
                    surf[i] += (fstar - fn) / (J[e, i] * w1[face_idx])
        du[e] = -(vol + surf).T
    ref = orc.rhs(nd, p, nelem, Ja, J, u, llf=True)
    np.testing.assert_allclose(ref, du, rtol=0, atol=1e-12 * np.max(np.abs(du)))
    assert np.all(W > 0)


# ------------------------------------------------------------------------------------------------
# Time integration (Sec. 4.1): order conditions of CK(5,4) and observed order on the DG system
# ------------------------------------------------------------------------------------------------

def test_ck45_order_conditions():
    A, B = orc.ck45_coefficients()
    s = 5
    # track U and K as coefficient vectors over (dt f_1 .. dt f_5); f_s is evaluated at U before stage s
    Kc = np.zeros(s)
    Uc = np.zeros(s)
    a = np.zeros((s, s))
    for st in range(s):
        a[st] = Uc
        Kc = A[st] * Kc
        Kc[st] += 1.0
        Uc = Uc + B[st] * Kc
    b = Uc
    c = a.sum(axis=1)
    conds = [
        (b.sum(), 1.0), (b @ c, 1 / 2), (b @ c ** 2, 1 / 3), (b @ a @ c, 1 / 6),
        (b @ c ** 3, 1 / 4), (b @ (c * (a @ c)), 1 / 8), (b @ a @ c ** 2, 1 / 12), (b @ a @ a @ c, 1 / 24),
    ]
    for got, want in conds:
        assert abs(got - want) < 1e-12, (got, want)


@pytest.mark.parametrize("scheme", [orc.RK4_CLASSIC, orc.LSRK45_CK])
def test_rk_step_fourth_order_on_dg_system(scheme):
    nd, nelem, p = 2, [3, 3], 2
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u0 = inputs.smooth_random(xyz, seed=11)
    T = 0.2

    def integrate(nsteps):
        # EC surface flux: the LLF dissipation's max/abs make the RHS only Lipschitz, which hides the order
        u = u0
        for _ in range(nsteps):
            u = orc.rk_step(scheme, nd, p, nelem, Ja, J, u, T / nsteps, llf=False)
        return u

    ref = integrate(64)
    e1 = np.max(np.abs(integrate(4) - ref))
    e2 = np.max(np.abs(integrate(8) - ref))
    order = math.log2(e1 / e2)
    assert order > 3.6, (e1, e2, order)


# ------------------------------------------------------------------------------------------------
# The oracle's JVP (oracle.c compiled with dual numbers): pinned by its value part (the double oracle) and by
# central finite differences of the double oracle
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd,nelem,p,llf", [(3, [2, 3, 2], 3, True), (2, [3, 4], 4, False), (3, [2, 2, 2], 2, True)])
def test_dual_jvp_value_and_finite_differences(nd, nelem, p, llf):
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u = inputs.smooth_random(xyz, seed=21) + 0.01 * inputs.random_state(xyz, seed=22)
    delta = inputs.perturbation(u.shape, seed=23) * np.abs(u)
    val, jd = orc.jvp(nd, p, nelem, Ja, J, u, delta, llf=llf)
    np.testing.assert_array_equal(val, orc.rhs(nd, p, nelem, Ja, J, u, llf=llf))
    # eps small enough that no LLF switch (max, abs) lies within u +- eps delta for these seeds
    eps = 1e-6
    fd = (orc.rhs(nd, p, nelem, Ja, J, u + eps * delta, llf=llf) -
          orc.rhs(nd, p, nelem, Ja, J, u - eps * delta, llf=llf)) / (2 * eps)
    for c in range(nd + 2):
        scale = np.max(np.abs(jd[:, c]))
        assert np.max(np.abs(jd[:, c] - fd[:, c])) <= 1e-6 * scale, c


def test_dual_logmean_derivative_at_equal_arguments():
    # d/da {{a, b}}_log at a = b is 1/2 per argument; the dual JVP of a constant-density state sees it
    nd, nelem, p = 3, [2, 2, 2], 2
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u = inputs.free_stream(xyz)
    delta = inputs.perturbation(u.shape, seed=24)
    _, jd = orc.jvp(nd, p, nelem, Ja, J, u, delta, llf=True)
    eps = 1e-6
    fd = (orc.rhs(nd, p, nelem, Ja, J, u + eps * delta) - orc.rhs(nd, p, nelem, Ja, J, u - eps * delta)) / (2 * eps)
    np.testing.assert_allclose(jd, fd, rtol=0, atol=1e-6 * np.max(np.abs(jd)))


# ------------------------------------------------------------------------------------------------
# Flux of Shima et al. (Sec. 3.2, Eq. flux_shima_etal): consistent, symmetric, kinetic-energy and pressure-
# equilibrium preserving, conservative and order-p accurate in the scheme, but not entropy conservative
# ------------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nd", [2, 3])
def test_shima_flux_consistency_symmetry_and_structure(nd):
    n = 2000
    a = random_states(n, nd, seed=30)
    b = random_states(n, nd, seed=31)
    m = np.random.Generator(np.random.PCG64(32)).standard_normal((n, nd))
    phys = sum(m[:, j:j + 1] * orc.euler_flux(a, j, nd) for j in range(nd))
    np.testing.assert_allclose(orc.flux_dir(a, a, m, nd, flux="shima"), phys, rtol=1e-13, atol=1e-13)
    f = orc.flux_dir(a, b, m, nd, flux="shima")
    np.testing.assert_allclose(f, orc.flux_dir(b, a, m, nd, flux="shima"), rtol=1e-14, atol=1e-14)
    va, vb = a[:, 1:nd + 1] / a[:, :1], b[:, 1:nd + 1] / b[:, :1]
    pa = (G - 1) * (a[:, -1] - 0.5 * np.sum(a[:, 1:nd + 1] * va, axis=1))
    pb = (G - 1) * (b[:, -1] - 0.5 * np.sum(b[:, 1:nd + 1] * vb, axis=1))
    vn = 0.5 * np.sum((va + vb) * m, axis=1)
    # mass flux {{rho}}{{v.n}}; momentum f_rho {{v}} + {{p}} n; energy as printed
    np.testing.assert_allclose(f[:, 0], 0.5 * (a[:, 0] + b[:, 0]) * vn, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(f[:, 1:nd + 1], f[:, :1] * 0.5 * (va + vb) + 0.5 * (pa + pb)[:, None] * m,
                               rtol=1e-13, atol=1e-13)
    ener = (f[:, 0] * 0.5 * np.sum(va * vb, axis=1) + 0.5 * (pa + pb) * vn / (G - 1)
            + 0.5 * (pa * np.sum(vb * m, axis=1) + pb * np.sum(va * m, axis=1)))
    np.testing.assert_allclose(f[:, -1], ener, rtol=1e-12, atol=1e-12)


def test_shima_scheme_conservative_pep_not_ec():
    nd, nelem, p = 3, [3, 2, 3], 3
    xyz, Ja, J = mesh(nd, nelem, p, True)
    u = inputs.random_state(xyz, seed=33)
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=True, flux="shima")
    tot, ab = orc.integrate(nd, p, J, du)
    assert np.all(np.abs(tot) <= 1e-13 * ab)
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=False, flux="shima")
    s, ab = orc.entropy_rate(nd, p, J, u, du)
    assert abs(s) > 1e-6 * ab  # not entropy conservative (contrast with Ranocha's flux)
    v = [0.1, -0.2, 0.3]
    u = inputs.pressure_equilibrium(xyz, seed=34, v=v)
    du = orc.rhs(nd, p, nelem, Ja, J, u, llf=True, flux="shima")
    scale = np.max(np.abs(du[:, 0]))
    for j in range(nd):
        np.testing.assert_allclose(du[:, 1 + j], v[j] * du[:, 0], rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(du[:, 4], 0.5 * np.dot(v, v) * du[:, 0], rtol=0, atol=1e-12 * scale)


def test_shima_rhs_converges_to_exact_derivative_tgv_curved():
    sp = pytest.importorskip("sympy")
    x, y, z = sp.symbols("x y z")
    M = 0.5
    prim = (sp.Integer(1), [sp.sin(x) * sp.cos(y) * sp.cos(z), -sp.cos(x) * sp.sin(y) * sp.cos(z), sp.Integer(0)],
            1 / (G * M ** 2) + (sp.cos(2 * x) + sp.cos(2 * y)) * (sp.cos(2 * z) + 2) / 16)
    fns = _sympy_euler_dudt(3, prim, (x, y, z))
    p = 3
    errs = []
    for ne in [8, 16]:
        nelem = [ne] * 3
        xyz, Ja, J = mesh(3, nelem, p, True)
        u = inputs.taylor_green(xyz, mach=M)
        du = orc.rhs(3, p, nelem, Ja, J, u, llf=True, flux="shima")
        ex = _eval(fns, xyz)
        errs.append(np.array([np.max(np.abs(du[:, c] - ex[:, c])) for c in range(5)]))
    order = np.log2(errs[0] / errs[1])
    assert np.all(order > p - 0.6), (errs, order)
