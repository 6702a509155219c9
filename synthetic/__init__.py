"""Seeded synthetic workloads shared by the GPU library's tests/bench and the oracle.

This module draws random numbers and evaluates the smooth space-time fields that
stand in for the paper's flow data. It holds none of the method's arithmetic:
no operator, no quadrature, no solver and no guess formula. Each side passes in
its own node coordinates.

Workload (the paper's fence-flow runs are not available; these stand in for
the slowly varying right-hand sides of Sec. 6):

    x*(t; x, y, z) = sum_j cos(w_j t + phi_j) sin(a_j pi x) sin(b_j pi y) sin(c_j pi z)

with integer wavenumbers a_j, b_j, c_j ~ U{1..kmax}, w_j ~ U[1, 5] and
phi_j ~ U[0, 2 pi).  b_k = A x*(t_k) (+ optional Gaussian noise whose standard
deviation is a multiple of RMS(A x*(t_k))).
"""
import numpy as np

# name: (elements per direction, degree p, lambda, steps, dt, modes, kmax, s, tol)
CONFIGS = {
    "poisson_4x4x4_p3": dict(E=(4, 4, 4), p=3, lam=0.0, steps=20, dt=0.01, modes=8, kmax=4, s=4,
               tol=1e-8, noise=0.0, seed=1),
    "helmholtz_16x16x16_p7": dict(E=(16, 16, 16), p=7, lam=1.0 / (1e-2 * 1e-3), steps=200, dt=1e-3,
               modes=32, kmax=6, s=8, tol=1e-10, noise=1e-6, seed=2),
    "poisson_32x32x32_p7": dict(E=(32, 32, 32), p=7, lam=0.0, steps=100, dt=0.01, modes=8, kmax=4, s=8,
               tol=1e-10, noise=0.0, seed=3),
    "heat_16x16x16_p7": dict(E=(16, 16, 16), p=7, lam=1.0 / (1e-2 * 1e-3), steps=50, dt=1e-3,
               modes=64, kmax=8, s=6, tol=1e-10, noise=0.0, seed=5),
}

# batched: four independent sequences (3 Helmholtz lam=1e3, 1 Poisson); the
# Poisson one uses projection QR(8), the Helmholtz ones EXTRAP(3,8)
BATCHED = [
    dict(E=(24, 24, 24), p=7, lam=0.0, seed=40, method="qr", m=0),
    dict(E=(20, 20, 20), p=7, lam=1e3, seed=41, method="extrap", m=3),
    dict(E=(16, 16, 16), p=7, lam=1e3, seed=42, method="extrap", m=3),
    dict(E=(12, 12, 12), p=7, lam=1e3, seed=43, method="extrap", m=3),
]
BATCHED_COMMON = dict(steps=100, dt=0.01, modes=8, kmax=4, s=8, tol=1e-10, noise=0.0)


class Modes:
    """Mode parameters of one synthetic solution field."""

    def __init__(self, seed, nmodes, kmax):
        rng = np.random.default_rng(seed)
        self.a = rng.integers(1, kmax + 1, nmodes)
        self.b = rng.integers(1, kmax + 1, nmodes)
        self.c = rng.integers(1, kmax + 1, nmodes)
        self.w = rng.uniform(1.0, 5.0, nmodes)
        self.phi = rng.uniform(0.0, 2.0 * np.pi, nmodes)
        self.seed = seed

    def amplitudes(self, t):
        return np.cos(self.w * t + self.phi)

    def factors(self, cx, cy, cz):
        """Per-mode 1D factors sin(a pi x), sin(b pi y), sin(c pi z): (J, n) arrays."""
        sx = np.sin(np.pi * self.a[:, None] * np.asarray(cx)[None, :])
        sy = np.sin(np.pi * self.b[:, None] * np.asarray(cy)[None, :])
        sz = np.sin(np.pi * self.c[:, None] * np.asarray(cz)[None, :])
        return sx, sy, sz

    def field(self, cx, cy, cz, t):
        """x*(t) on the tensor grid, flattened with x fastest (small grids)."""
        sx, sy, sz = self.factors(cx, cy, cz)
        amp = self.amplitudes(t)
        return np.einsum('j,jk,jy,jx->kyx', amp, sz, sy, sx).reshape(-1)

    def mode_field(self, j, cx, cy, cz):
        sx, sy, sz = self.factors(cx, cy, cz)
        return np.einsum('k,y,x->kyx', sz[j], sy[j], sx[j]).reshape(-1)


def noise(seed, step, n):
    """Standard normal vector for time step ``step`` (scaled by the caller)."""
    return np.random.default_rng([seed, 7919, step]).standard_normal(n)


def random_vectors(seed, count, n):
    """Generic seeded test vectors (uniform in [-1, 1])."""
    return np.random.default_rng([seed, 104729]).uniform(-1.0, 1.0, (count, n))


def forcing_basis_indices(nmodes):
    """(a, b, c) of the ``nmodes`` Dirichlet sine modes with smallest a^2+b^2+c^2,
    ties broken lexicographically."""
    cand = [(a * a + b * b + c * c, a, b, c) for a in range(1, 12)
            for b in range(1, 12) for c in range(1, 12)]
    cand.sort()
    return np.array([(a, b, c) for _, a, b, c in cand[:nmodes]])


def adjoint_parameters(seed, nparam):
    """theta* ~ N(0, 1) and frequencies w_j ~ U[1, 5] for the forcing."""
    rng = np.random.default_rng([seed, 31337])
    return rng.standard_normal(nparam), rng.uniform(1.0, 5.0, nparam)
