"""Pins for the oracle's GLL basis, SEM operator and PCG (CPU only).

Each test checks the oracle against something other than itself: closed-form
node/weight values, exact polynomial integrals, the textbook p = 1 reduction to
the 7-point finite-difference Laplacian, a dense Cholesky solve, and the
continuous eigenvalue 3 pi^2.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
from numpy.polynomial import Polynomial as Poly

from oracle.gll import gll_nodes_weights, gll_derivative
from oracle.sem import SemOperator
from oracle.pcg import pcg, REL_B, INITRESID, RHS

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# ---------------------------------------------------------------- GLL basis
def test_gll_closed_forms():
    x, w = gll_nodes_weights(2)
    assert np.allclose(x, [-1, 0, 1], atol=1e-15)
    assert np.allclose(w, [1 / 3, 4 / 3, 1 / 3], atol=1e-15)
    x, w = gll_nodes_weights(3)
    r = 1 / np.sqrt(5)
    assert np.allclose(x, [-1, -r, r, 1], atol=1e-15)
    assert np.allclose(w, [1 / 6, 5 / 6, 5 / 6, 1 / 6], atol=1e-15)
    x, w = gll_nodes_weights(1)
    assert np.allclose(x, [-1, 1]) and np.allclose(w, [1, 1])


@pytest.mark.parametrize("p", [1, 2, 3, 4, 5, 6, 7, 8, 10])
def test_gll_quadrature_exact_to_degree_2p_minus_1(p):
    x, w = gll_nodes_weights(p)
    assert abs(w.sum() - 2.0) < 1e-14
    for k in range(2 * p):
        exact = 0.0 if k % 2 else 2.0 / (k + 1)
        assert abs(np.dot(w, x ** k) - exact) < 1e-13
    # and NOT exact at degree 2p (GLL is one order short of Gauss)
    k = 2 * p
    assert abs(np.dot(w, x ** k) - 2.0 / (k + 1)) > 1e-6


@pytest.mark.parametrize("p", [1, 2, 3, 5, 7, 9])
def test_gll_derivative_exact_on_polynomials(p):
    x, _ = gll_nodes_weights(p)
    D = gll_derivative(p)
    rng = np.random.default_rng(p)
    for _ in range(3):
        c = rng.standard_normal(p + 1)
        f = Poly(c)
        assert np.allclose(D @ f(x), f.deriv()(x), atol=1e-11 * max(1, p ** 2))
    assert np.allclose(D.sum(axis=1), 0, atol=1e-12)


# ---------------------------------------------------------------- operator
@pytest.mark.parametrize("lam", [0.0, 3.7])
def test_p1_reduces_to_fd_laplacian(lam):
    """p = 1: GLL quadrature is the trapezoid rule, and the SEM operator on a
    uniform grid of spacing h is h * (7-point Laplacian stencil) + lam h^3 I."""
    E = 5
    op = SemOperator(E, E, E, 1, lam)
    h = 1.0 / E
    n1 = E + 1
    T = sp.diags([-np.ones(n1 - 1), 2 * np.ones(n1), -np.ones(n1 - 1)], [-1, 0, 1])
    I1 = sp.identity(n1)
    L7 = sp.kron(sp.kron(I1, I1), T) + sp.kron(sp.kron(I1, T), I1) + sp.kron(sp.kron(T, I1), I1)
    A_fd = (h * L7 + lam * h ** 3 * sp.identity(n1 ** 3)).toarray()
    m = op.interior
    A_fd = A_fd * m[:, None] * m[None, :]
    assert np.allclose(op.dense(), A_fd, atol=1e-13)


def _poly_integral(f, g):
    """Exact integral over [0, 1] of the product of two numpy Polynomials."""
    F = (f * g).integ()
    return F(1.0) - F(0.0)


@pytest.mark.parametrize("E,p,lam", [((1, 1, 1), 3, 0.0), ((2, 3, 1), 3, 2.5),
                                     ((2, 2, 2), 4, 0.0), ((1, 2, 3), 5, 11.0)])
def test_bilinear_form_exact_for_polynomials(E, p, lam):
    """u^T A v = int grad u . grad v + lam int u v exactly when every 1D
    integrand has degree <= 2p-1 (u of degree p, v of degree p-1 per
    variable); the unmasked (Neumann) operator is used."""
    op = SemOperator(*E, p, lam)
    cx, cy, cz = op.coords_1d()
    rng = np.random.default_rng(7)
    fu = [Poly(rng.standard_normal(p + 1)) for _ in range(3)]
    fv = [Poly(rng.standard_normal(p)) for _ in range(3)]
    u = np.einsum('k,j,i->kji', fu[2](cz), fu[1](cy), fu[0](cx)).reshape(-1)
    v = np.einsum('k,j,i->kji', fv[2](cz), fv[1](cy), fv[0](cx)).reshape(-1)
    I = [[_poly_integral(fu[d], fv[d]) for d in range(3)],
         [_poly_integral(fu[d].deriv(), fv[d].deriv()) for d in range(3)]]
    stiff = (I[1][0] * I[0][1] * I[0][2] + I[0][0] * I[1][1] * I[0][2]
             + I[0][0] * I[0][1] * I[1][2])
    mass = I[0][0] * I[0][1] * I[0][2]
    exact = stiff + lam * mass
    got = v @ op.apply(u, mask=False)
    assert abs(got - exact) <= 1e-11 * (abs(stiff) + abs(lam * mass) + 1)
    # symmetric in u, v
    assert abs(u @ op.apply(v, mask=False) - got) <= 1e-11 * (abs(got) + 1)


def test_symmetric_positive_definite_and_diagonal():
    op = SemOperator(3, 2, 2, 3, 1.5)
    A = op.dense()
    assert np.allclose(A, A.T, atol=1e-13)
    m = op.interior
    Ai = A[np.ix_(m, m)]
    sla.cholesky(Ai)                      # raises if not SPD
    d = op.diagonal()
    assert np.allclose(d[m], np.diag(A)[m], rtol=1e-13)
    assert np.all(d[~m] == 1.0)


def test_rayleigh_quotient_converges_to_3pi2():
    """sin(pi x) sin(pi y) sin(pi z) is the first Dirichlet eigenfunction of
    -Laplace with eigenvalue 3 pi^2; the discrete Rayleigh quotient
    (u^T K u) / (u^T M u) converges spectrally in p."""
    errs = []
    for p in (3, 5, 7):
        K = SemOperator(2, 2, 2, p, 0.0)
        Mop = SemOperator(2, 2, 2, p, 1.0)
        cx, cy, cz = K.coords_1d()
        u = np.einsum('k,j,i->kji', np.sin(np.pi * cz), np.sin(np.pi * cy),
                      np.sin(np.pi * cx)).reshape(-1)
        Ku = K.apply(u)
        Mu = Mop.apply(u) - Ku
        errs.append(abs((u @ Ku) / (u @ Mu) - 3 * np.pi ** 2) / (3 * np.pi ** 2))
    assert errs[0] < 1e-2 and errs[2] < 1e-8 and errs[2] < errs[1] < errs[0]


# ---------------------------------------------------------------- PCG
def test_pcg_matches_dense_cholesky_c1():
    op = SemOperator(4, 4, 4, 3, 0.0)
    m = op.interior
    rng = np.random.default_rng(3)
    b = rng.standard_normal(op.n) * m
    A = op.dense()
    Ai = A[np.ix_(m, m)]
    xd = np.zeros(op.n)
    xd[m] = sla.cho_solve(sla.cho_factor(Ai), b[m])
    x, it, rel, _ = pcg(op.apply, op.diagonal(), b, np.zeros(op.n), 1e-13, interior=m)
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)
    assert rel <= 1e-12 and 0 < it < 200


def test_pcg_stopping_rules():
    op = SemOperator(3, 3, 3, 2, 2.0)
    m = op.interior
    rng = np.random.default_rng(4)
    xs = rng.standard_normal(op.n) * m
    b = op.apply(xs)
    d = op.diagonal()
    # exact initial guess -> 0 iterations for every rule
    for crit in (REL_B, INITRESID, RHS):
        _, it, _, _ = pcg(op.apply, d, b, xs, 1e-8, criterion=crit, interior=m)
        assert it == 0
    # REL_B stops at ||r|| <= tol ||b|| on the recursive residual
    x, it, rel, hist = pcg(op.apply, d, b, np.zeros(op.n), 1e-9, interior=m)
    bn = np.linalg.norm(b)
    assert hist[-1] <= 1e-9 * bn and hist[-2] > 1e-9 * bn
    # INITRESID with a small initial residual collapses to an absolute test
    x0 = xs + 1e-6 * rng.standard_normal(op.n) * m
    _, it2, _, h2 = pcg(op.apply, d, b, x0, 1e-8, criterion=INITRESID, interior=m)
    assert h2[0] < 1.0 and h2[-1] < 1e-8 and h2[-2] >= 1e-8


def test_pcg_recovers_smooth_solution():
    """b = A x*  ->  PCG returns x* (to about cond * tol)."""
    from synthetic import Modes
    op = SemOperator(4, 4, 4, 3, 0.0)
    cx, cy, cz = op.coords_1d()
    xs = Modes(1, 8, 4).field(cx, cy, cz, 0.37) * op.interior
    b = op.apply(xs)
    x, it, rel, _ = pcg(op.apply, op.diagonal(), b, np.zeros(op.n), 1e-12, interior=op.interior)
    assert np.linalg.norm(x - xs) <= 1e-8 * np.linalg.norm(xs)
