"""Seeded synthetic inputs for the compressible Euler RHS: initial conditions at given node coordinates.

This module is shared by the tests, the benchmark and the smoke check, and serves both the CUDA path
and the CPU oracle. It holds none of the method's arithmetic (no numerical flux, no derivative
operator, no metric term, no logarithmic mean): only closed-form initial conditions evaluated at node
coordinates that the caller supplies, the map from primitive (rho, v, p) to conserved
(rho, rho v, rho e) that defines a state of Eq. Euler, and seeded noise.

Coordinates are ``xyz[E, ndims, Nd]``; returned states are ``u[E, ndims+2, Nd]`` float64.
"""
from __future__ import annotations

import numpy as np

GAMMA = 1.4


def prim_to_cons(rho, v, p, gamma: float = GAMMA) -> np.ndarray:
    """(rho, v_1..v_d, p) -> (rho, rho v_1..rho v_d, rho e) with rho e = p/(gamma-1) + rho|v|^2/2."""
    rho = np.asarray(rho, dtype=np.float64)
    v = [np.broadcast_to(np.asarray(vj, dtype=np.float64), rho.shape) for vj in v]
    p = np.broadcast_to(np.asarray(p, dtype=np.float64), rho.shape)
    kin = 0.5 * rho * sum(vj * vj for vj in v)
    comps = [rho] + [rho * vj for vj in v] + [p / (gamma - 1.0) + kin]
    return np.ascontiguousarray(np.stack(comps, axis=1))


def _split(xyz):
    xyz = np.asarray(xyz, dtype=np.float64)
    return [xyz[:, m, :] for m in range(xyz.shape[1])]


def taylor_green(xyz, gamma: float = GAMMA, mach: float = 0.1) -> np.ndarray:
    """Inviscid Taylor-Green vortex: rho = 1, v = (sin x cos y cos z, -cos x sin y cos z, 0),
    p = 1/(gamma M^2) + (cos 2x + cos 2y)(cos 2z + 2)/16."""
    x, y, z = _split(xyz)
    rho = np.ones_like(x)
    v1 = np.sin(x) * np.cos(y) * np.cos(z)
    v2 = -np.cos(x) * np.sin(y) * np.cos(z)
    v3 = np.zeros_like(x)
    p = 1.0 / (gamma * mach * mach) + (np.cos(2 * x) + np.cos(2 * y)) * (np.cos(2 * z) + 2.0) / 16.0
    return prim_to_cons(rho, [v1, v2, v3], p, gamma)


def noisy_sine_2d(xyz, seed: int = 0, amplitude: float = 1e-2, gamma: float = GAMMA) -> np.ndarray:
    """rho = 1 + 0.1 sin(pi x) sin(pi y), v = (0.1, 0.2), p = 1, plus independent seeded
    uniform(-amplitude, amplitude) noise on each primitive (rho, v_1, v_2, p) at each node."""
    x, y = _split(xyz)
    rng = np.random.Generator(np.random.PCG64(seed))
    noise = rng.uniform(-amplitude, amplitude, size=(x.shape[0], 4, x.shape[1]))
    rho = 1.0 + 0.1 * np.sin(np.pi * x) * np.sin(np.pi * y) + noise[:, 0]
    v1 = 0.1 + noise[:, 1]
    v2 = 0.2 + noise[:, 2]
    p = 1.0 + noise[:, 3]
    return prim_to_cons(rho, [v1, v2], p, gamma)


def isentropic_vortex(xyz, eps: float = 20.0, gamma: float = GAMMA, planar: bool = False,
                      v0=(1.0, 1.0, 0.0), rho0: float = 1.0, p0: float = 10.0) -> np.ndarray:
    """Isentropic vortex (Sec. 4.1, Eq. isentropic-vortex): T = T0 - (gamma-1) eps^2/(8 gamma pi^2)
    exp(1 - r^2), rho = rho0 (T/T0)^(1/(gamma-1)), v = v0 + eps/(2 pi) exp((1-r^2)/2) (-x2, x1, 0),
    p = rho T. r is the distance from the origin; planar=True measures r in the x1-x2 plane only,
    which makes the 3D field an exact travelling solution."""
    X = _split(xyz)
    nd = len(X)
    r2 = X[0] ** 2 + X[1] ** 2 + (X[2] ** 2 if (nd == 3 and not planar) else 0.0)
    T0 = p0 / rho0
    T = T0 - (gamma - 1.0) * eps * eps / (8.0 * gamma * np.pi ** 2) * np.exp(1.0 - r2)
    rho = rho0 * (T / T0) ** (1.0 / (gamma - 1.0))
    g = eps / (2.0 * np.pi) * np.exp(0.5 * (1.0 - r2))
    v = [v0[0] - g * X[1], v0[1] + g * X[0]] + ([v0[2] + 0.0 * X[0]] if nd == 3 else [])
    return prim_to_cons(rho, v, rho * T, gamma)


def density_wave(xyz, amp: float = 0.2, k=None, v=None, p: float = 1.0, gamma: float = GAMMA) -> np.ndarray:
    """rho = 1 + amp sin(k . x), constant v and p: an exact travelling solution of Eq. Euler."""
    X = _split(xyz)
    nd = len(X)
    k = k if k is not None else [1.0] * nd
    v = v if v is not None else [0.1, 0.2, 0.3][:nd]
    phase = sum(kj * xj for kj, xj in zip(k, X))
    rho = 1.0 + amp * np.sin(phase)
    return prim_to_cons(rho, [vj + 0.0 * rho for vj in v], p + 0.0 * rho, gamma)


def free_stream(xyz, rho: float = 1.0, v=None, p: float = 1.0, gamma: float = GAMMA) -> np.ndarray:
    """Constant state (default rho = 1, v = (0.1, 0.2, 0.3), p = 1)."""
    X = _split(xyz)
    nd = len(X)
    v = v if v is not None else [0.1, 0.2, 0.3][:nd]
    one = np.ones_like(X[0])
    return prim_to_cons(rho * one, [vj * one for vj in v], p * one, gamma)


def pressure_equilibrium(xyz, seed: int = 0, v=None, p: float = 1.0, gamma: float = GAMMA) -> np.ndarray:
    """Seeded positive density field with constant velocity and pressure."""
    X = _split(xyz)
    nd = len(X)
    rng = np.random.Generator(np.random.PCG64(seed))
    rho = 1.0 + 0.5 * rng.uniform(0.0, 1.0, size=X[0].shape)
    v = v if v is not None else [0.1, -0.2, 0.3][:nd]
    return prim_to_cons(rho, [vj + 0.0 * rho for vj in v], p + 0.0 * rho, gamma)


def sine_paper(xyz, gamma: float = GAMMA) -> np.ndarray:
    """Sinusoidal initial condition of Sec. 7.2: rho = 2 + prod_m sin(pi x_m / 5), p = rho^gamma, v = 0."""
    X = _split(xyz)
    rho = 2.0 + np.prod([np.sin(np.pi * xm / 5.0) for xm in X], axis=0)
    return prim_to_cons(rho, [0.0 * rho for _ in X], rho ** gamma, gamma)


def random_state(xyz, seed: int = 0, gamma: float = GAMMA) -> np.ndarray:
    """Seeded random nodal state (the random initial condition of Sec. 7.2; the paper does not give its
    distribution): rho, p ~ uniform(0.5, 1.5), v_m ~ uniform(-0.5, 0.5), independent per node."""
    X = _split(xyz)
    rng = np.random.Generator(np.random.PCG64(seed))
    shape = X[0].shape
    rho = rng.uniform(0.5, 1.5, size=shape)
    v = [rng.uniform(-0.5, 0.5, size=shape) for _ in X]
    p = rng.uniform(0.5, 1.5, size=shape)
    return prim_to_cons(rho, v, p, gamma)


def smooth_random(xyz, seed: int = 0, lengths=None, gamma: float = GAMMA, modes: int = 3) -> np.ndarray:
    """Seeded smooth periodic state from `modes` random low Fourier modes per field, scaled so that
    rho in 1 +- 0.2, |v| < 0.3 and p in 1 +- 0.2. `lengths` are the periodic box sizes (default 2 pi)."""
    X = _split(xyz)
    nd = len(X)
    L = lengths if lengths is not None else [2.0 * np.pi] * nd
    rng = np.random.Generator(np.random.PCG64(seed))

    def field():
        f = np.zeros_like(X[0])
        for _ in range(modes):
            kvec = rng.integers(-2, 3, size=nd)
            phase = rng.uniform(0.0, 2.0 * np.pi)
            arg = sum(2.0 * np.pi * kvec[m] * X[m] / L[m] for m in range(nd)) + phase
            f = f + np.sin(arg) / modes
        return f  # |f| <= 1

    rho = 1.0 + 0.2 * field()
    v = [0.3 / np.sqrt(nd) * 0.99 * field() for _ in range(nd)]
    p = 1.0 + 0.2 * field()
    return prim_to_cons(rho, v, p, gamma)


def perturbation(shape, seed: int, scale: float = 1.0) -> np.ndarray:
    """Seeded standard-normal array (directions for derivative checks), times scale."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return scale * rng.standard_normal(size=shape)
