"""Pins for the oracle's extrapolation and projection guesses (CPU only).

Extrapolation is checked against the paper's closed forms (Eq.
NaiveExtrapCoeffs, the M = 2 example, the Lebesgue constant 2^M - 1), an
exact-rational least-squares solve in the monomial basis, the exactness
identity beta^T V = v^T (Eq. PolyExactness) and the residual orders of the
comparison theorem (Sec. 4).  Projection (Algorithms 1 and 2) is checked
against a brute-force dense least-squares fit over the raw window of stored
solutions and the invariants B~^T B~ = I, A X~ = B~, B~ R = A X_window.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
from numpy.polynomial import Polynomial as Poly

from oracle import extrap as ex
from oracle.proj import ProjectionQR, ProjectionClassic, ProjectionEnergy
from oracle.sem import SemOperator

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ---------------------------------------------------------------- extrapolation
def test_naive_example_from_paper():
    for row in _golden_rows("naive_extrap_example.txt"):
        M = int(row[0])
        want = np.array([float(v) for v in row[1:]])
        assert np.allclose(ex.lsq_coeffs(M, M - 1), want, atol=1e-14)
        assert np.allclose(ex.naive_coeffs(M), want)


@pytest.mark.parametrize("M", range(1, 13))
def test_lsq_with_full_degree_is_naive_lagrange(M):
    beta = ex.lsq_coeffs(M, M - 1)
    naive = ex.naive_coeffs(M)
    assert np.allclose(beta, naive, rtol=1e-9, atol=1e-9 * np.abs(naive).max())


def test_naive_lebesgue_constant():
    for row in _golden_rows("naive_lebesgue.txt"):
        M, lam = int(row[0]), float(row[1])
        assert abs(ex.lebesgue_constant(ex.naive_coeffs(M)) - lam) < 1e-9
        assert abs(ex.lebesgue_constant(ex.lsq_coeffs(M, M - 1)) - lam) < 1e-6 * lam


@pytest.mark.parametrize("M", [1, 2, 3, 5, 8, 12])
def test_degree_zero_is_mean(M):
    assert np.allclose(ex.lsq_coeffs(M, 0), np.full(M, 1.0 / M), atol=1e-15)


@pytest.mark.parametrize("M", [2, 3, 4, 6, 8, 12])
def test_degree_one_closed_form(M):
    """Least-squares line through the points: beta_i = 1/M + t_new t_i / sum t_j^2
    (the t_i are symmetric about 0)."""
    t, tn = ex.time_points(M)
    want = 1.0 / M + tn * t / np.sum(t * t)
    assert np.allclose(ex.lsq_coeffs(M, 1), want, atol=1e-14)


def _exact_beta(M, m):
    """beta = V (V^T V)^{-1} v in exact rational arithmetic, monomial basis."""
    h = Fraction(2, M - 1)
    t = [Fraction(-1) + i * h for i in range(M)]
    tn = 1 + h
    V = [[ti ** j for j in range(m + 1)] for ti in t]
    v = [tn ** j for j in range(m + 1)]
    G = [[sum(V[i][a] * V[i][b] for i in range(M)) for b in range(m + 1)] for a in range(m + 1)]
    # Gauss-Jordan on G y = v
    n = m + 1
    Aug = [G[r][:] + [v[r]] for r in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if Aug[r][c] != 0)
        Aug[c], Aug[piv] = Aug[piv], Aug[c]
        for r in range(n):
            if r != c and Aug[r][c] != 0:
                f = Aug[r][c] / Aug[c][c]
                Aug[r] = [a - f * b for a, b in zip(Aug[r], Aug[c])]
    y = [Aug[r][n] / Aug[r][r] for r in range(n)]
    return [sum(V[i][j] * y[j] for j in range(n)) for i in range(M)]


@pytest.mark.parametrize("M,m", [(3, 1), (4, 2), (6, 2), (8, 2), (8, 3), (8, 4), (12, 3), (12, 5)])
def test_lsq_matches_exact_rational(M, m):
    """Legendre basis + Householder QR in floats vs monomial basis + normal
    equations in exact rationals: beta does not depend on the basis."""
    beta = ex.lsq_coeffs(M, m)
    exact = np.array([float(b) for b in _exact_beta(M, m)])
    assert np.allclose(beta, exact, rtol=1e-13, atol=1e-13 * np.abs(exact).max())


@pytest.mark.parametrize("M,m", [(4, 2), (6, 2), (8, 2), (8, 3), (12, 3), (12, 4)])
def test_polynomial_exactness_and_min_norm(M, m):
    t, tn = ex.time_points(M)
    V = ex.vandermonde(t, m)
    v = ex.vandermonde([tn], m)[0]
    beta = ex.lsq_coeffs(M, m)
    assert np.allclose(beta @ V, v, atol=1e-12)
    # minimum norm: beta is orthogonal to the null space of V^T
    Q, _ = np.linalg.qr(V, mode='complete')
    null = Q[:, m + 1:]
    assert np.allclose(null.T @ beta, 0, atol=1e-12)
    # vector data from a random degree-m polynomial is extrapolated exactly
    rng = np.random.default_rng(M * 10 + m)
    coefs = rng.standard_normal((m + 1, 5))
    hist = [sum(coefs[j] * ti ** j for j in range(m + 1)) for ti in t]
    truth = sum(coefs[j] * tn ** j for j in range(m + 1))
    assert np.allclose(ex.extrap_guess(hist, beta), truth, atol=1e-11)


@pytest.mark.parametrize("M,m", [(4, 2), (8, 2), (8, 3), (12, 3), (12, 4), (6, 5)])
def test_sparse_is_lagrange_through_chosen_points(M, m):
    beta = ex.sparse_coeffs(M, m)
    nz = np.flatnonzero(beta)
    assert len(nz) == m + 1
    t, tn = ex.time_points(M)
    V = ex.vandermonde(t, m)
    v = ex.vandermonde([tn], m)[0]
    assert np.allclose(beta @ V, v, atol=1e-11)
    # brute force: Lagrange basis through the chosen points, evaluated at t_new
    tp = t[nz]
    for a, i in enumerate(nz):
        others = np.delete(tp, a)
        lag = np.prod((tn - others) / (tp[a] - others))
        assert abs(beta[i] - lag) < 1e-11 * max(1, abs(lag))
    if m == M - 1:
        assert np.allclose(beta, ex.naive_coeffs(M), atol=1e-9)
    # min-norm LSQ beta is never larger in 2-norm
    assert np.linalg.norm(ex.lsq_coeffs(M, m)) <= np.linalg.norm(beta) + 1e-12


def test_startup_reading():
    assert np.allclose(ex.startup_coeffs(1, 8, 2), [1.0])
    assert np.allclose(ex.startup_coeffs(2, 8, 2), [-1.0, 2.0])
    assert np.allclose(ex.startup_coeffs(3, 8, 2), ex.naive_coeffs(3))
    assert np.allclose(ex.startup_coeffs(5, 8, 2), ex.lsq_coeffs(5, 2))
    assert np.allclose(ex.startup_coeffs(20, 8, 2), ex.lsq_coeffs(8, 2))


def _rate(hs, errs):
    return np.polyfit(np.log(hs), np.log(errs), 1)[0]


def test_residual_orders_theorem():
    """Sec. 4 theorem: ||r^P|| <= ||r^E||; r^P = O(h^M); r^E = O(h^{m+1})."""
    rng = np.random.default_rng(11)
    n = 40
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A = Q @ np.diag(np.linspace(1, 10, n)) @ Q.T
    K = 6
    cs, ws = rng.standard_normal((K, n)), rng.uniform(1, 3, K)

    def xt(t):
        return sum(np.sin(ws[k] * t + k) * cs[k] for k in range(K))

    M, m = 4, 1
    eP, eE = [], []
    hs = [0.08, 0.04, 0.02, 0.01]
    for h in hs:
        P = ProjectionQR(M, 0.0, lambda v: A @ v)
        E = ex.lsq_coeffs(M, m)
        xs = [xt(i * h) for i in range(1, M + 1)]
        for x in xs:
            P.update(x)
        b = A @ xt((M + 1) * h)
        rP = np.linalg.norm(b - A @ P.form(b, np.zeros(n)))
        rE = np.linalg.norm(b - A @ ex.extrap_guess(xs, E))
        assert rP <= rE * (1 + 1e-10)
        eP.append(rP)
        eE.append(rE)
    assert _rate(hs, eP) > M - 0.5
    assert abs(_rate(hs, eE) - (m + 1)) < 0.5


# ---------------------------------------------------------------- projection
def _small_problem(seed=5, lam=2.0):
    op = SemOperator(3, 3, 2, 2, lam)
    rng = np.random.default_rng(seed)
    return op, rng


def _check_invariants(P, op, tol=1e-12):
    B = np.array(P.B).T
    X = np.array(P.X).T
    d = P.d
    assert np.linalg.norm(B.T @ B - np.eye(d)) <= tol
    AX = np.array([op.apply(X[:, i]) for i in range(d)]).T
    assert np.linalg.norm(AX - B) <= tol * np.linalg.norm(B)
    Xw = np.array(P.accepted).T
    AXw = np.array([op.apply(Xw[:, i]) for i in range(d)]).T
    R = P.R[:d, :d]
    assert np.allclose(np.tril(R, -1), 0)
    # the paper's rotation (c = |a|/r) keeps the sign of a, so a downdated
    # diagonal entry may be negative; it is never zero.
    assert np.all(np.abs(np.diag(R)) > 0)
    assert np.linalg.norm(B @ R - AXw) <= tol * np.linalg.norm(AXw)


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_rolling_qr_invariants_and_bruteforce(M):
    op, rng = _small_problem()
    m = op.interior
    P = ProjectionQR(M, 1e-12, op.apply)
    base = rng.standard_normal((3, op.n)) * m
    for k in range(9):
        x = (np.cos(0.3 * k) * base[0] + np.sin(0.2 * k) * base[1]
             + 0.1 * k * base[2] + 1e-3 * rng.standard_normal(op.n) * m)
        P.update(x)
        assert P.d == min(k + 1, M)
        _check_invariants(P, op)
        # guess == brute-force argmin ||b - A X_window alpha||
        b = op.apply(rng.standard_normal(op.n) * m)
        g = P.form(b, np.zeros(op.n))
        Xw = np.array(P.accepted).T
        AXw = np.array([op.apply(Xw[:, i]) for i in range(P.d)]).T
        alpha, *_ = np.linalg.lstsq(AXw, b, rcond=None)
        assert np.linalg.norm(g - Xw @ alpha) <= 1e-10 * np.linalg.norm(Xw @ alpha)


def test_projection_exact_in_span_and_rejects_dependent():
    op, rng = _small_problem(6)
    m = op.interior
    P = ProjectionQR(4, 1e-8, op.apply)
    xs = rng.standard_normal((3, op.n)) * m
    for x in xs:
        assert P.update(x)
    xin = 0.3 * xs[0] - 1.7 * xs[2]
    b = op.apply(xin)
    assert np.linalg.norm(P.form(b, np.zeros(op.n)) - xin) <= 1e-12 * np.linalg.norm(xin)
    # a solution already in the span is rejected (d unchanged)
    assert not P.update(xin)
    assert P.d == 3
    _check_invariants(P, op)
    # zero guess when d = 0: caller's x0 returned untouched
    Q = ProjectionQR(4, 1e-8, op.apply)
    x0 = rng.standard_normal(op.n)
    assert np.array_equal(Q.form(b, x0), x0)


def test_projection_beats_extrapolation_same_window():
    """Sec. 4 theorem (i) on the SEM operator with the synthetic workload."""
    from synthetic import Modes
    op = SemOperator(3, 3, 3, 3, 0.0)
    cx, cy, cz = op.coords_1d()
    modes = Modes(1, 8, 4)
    M, m = 4, 2
    P = ProjectionQR(M, 0.0, op.apply)
    xs = [modes.field(cx, cy, cz, 0.01 * k) * op.interior for k in range(1, M + 1)]
    for x in xs:
        P.update(x)
    b = op.apply(modes.field(cx, cy, cz, 0.01 * (M + 1)) * op.interior)
    rP = np.linalg.norm(b - op.apply(P.form(b, np.zeros(op.n))))
    rE = np.linalg.norm(b - op.apply(ex.extrap_guess(xs, ex.lsq_coeffs(M, m))))
    assert rP <= rE


def _check_energy_invariants(P, op, tol=1e-11):
    B = np.array(P.B).T
    X = np.array(P.X).T
    d = P.d
    AX = np.array([op.apply(X[:, i]) for i in range(d)]).T
    assert np.linalg.norm(X.T @ AX - np.eye(d)) <= tol            # A-orthonormal
    assert np.linalg.norm(AX - B) <= tol * np.linalg.norm(B)
    Xw = np.array(P.accepted).T
    R = P.R[:d, :d]
    assert np.allclose(np.tril(R, -1), 0)
    assert np.all(np.abs(np.diag(R)) > 0)
    assert np.linalg.norm(X @ R - Xw) <= tol * np.linalg.norm(Xw)  # X_window = X~ R


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_energy_projection_invariants_and_bruteforce(M):
    """Energy-norm projection: X~ stays A-orthonormal through CGS2 and the
    Givens downdate, and the guess equals the brute-force minimiser of
    ||x - A^{-1} b||_A over the raw accepted window (normal equations of the
    window in the A-inner product, solved densely)."""
    op, rng = _small_problem(11)
    m = op.interior
    P = ProjectionEnergy(M, 1e-12, op.apply)
    base = rng.standard_normal((3, op.n)) * m
    for k in range(9):
        x = (np.cos(0.3 * k) * base[0] + np.sin(0.2 * k) * base[1]
             + 0.1 * k * base[2] + 1e-3 * rng.standard_normal(op.n) * m)
        P.update(x)
        assert P.d == min(k + 1, M)
        _check_energy_invariants(P, op)
        b = op.apply(rng.standard_normal(op.n) * m)
        g = P.form(b, np.zeros(op.n))
        Xw = np.array(P.accepted).T
        AXw = np.array([op.apply(Xw[:, i]) for i in range(P.d)]).T
        alpha = np.linalg.solve(Xw.T @ AXw, Xw.T @ b)
        assert np.linalg.norm(g - Xw @ alpha) <= 1e-9 * np.linalg.norm(Xw @ alpha)


def test_energy_projection_minimises_the_energy_error():
    """Same window: the energy-norm guess has the smaller A-norm error, the
    Euclidean (Algorithm 2) guess the smaller residual; a solution in the span
    is reproduced and then rejected as dependent."""
    from synthetic import Modes
    op = SemOperator(3, 3, 3, 3, 0.0)
    cx, cy, cz = op.coords_1d()
    modes = Modes(2, 8, 4)
    A = op.dense()
    idx = np.flatnonzero(op.interior)
    xs = [modes.field(cx, cy, cz, 0.01 * k) * op.interior for k in range(1, 6)]
    E = ProjectionEnergy(5, 0.0, op.apply)
    Q = ProjectionQR(5, 0.0, op.apply)
    for x in xs:
        E.update(x)
        Q.update(x)
    xt = modes.field(cx, cy, cz, 0.06) * op.interior
    b = op.apply(xt)

    def anorm(v):
        return float(np.sqrt(v[idx] @ A[np.ix_(idx, idx)] @ v[idx]))
    gE, gQ = E.form(b, np.zeros(op.n)), Q.form(b, np.zeros(op.n))
    assert anorm(gE - xt) <= anorm(gQ - xt) * (1 + 1e-12)
    assert np.linalg.norm(b - op.apply(gQ)) <= np.linalg.norm(b - op.apply(gE)) * (1 + 1e-12)
    rng = np.random.default_rng(12)
    ys = rng.standard_normal((3, op.n)) * op.interior
    F = ProjectionEnergy(6, 1e-8, op.apply)
    for y in ys:
        assert F.update(y)
    yin = 0.4 * ys[1] - 2.0 * ys[2]
    assert np.linalg.norm(F.form(op.apply(yin), np.zeros(op.n)) - yin) <= 1e-12 * np.linalg.norm(yin)
    assert not F.update(0.5 * ys[0] + 0.25 * ys[2])
    assert F.d == 3


def test_classic_restart_cycle():
    op, rng = _small_problem(8)
    m = op.interior
    P = ProjectionClassic(3, 1e-12, op.apply)
    ds = []
    for k in range(8):
        ds.append(P.d)
        P.update(rng.standard_normal(op.n) * m)
    assert ds == [0, 1, 2, 3, 1, 2, 3, 1]
    B = np.array(P.B).T
    assert np.linalg.norm(B.T @ B - np.eye(P.d)) < 1e-13


def test_table1_counts_golden():
    """Table 1 formulas evaluated at M = 8, m = 2 (the golden file quotes them)."""
    M, m = 8, 2
    want = {r[0]: tuple(int(v) for v in r[1:]) for r in _golden_rows("table1_memops.txt")}
    assert want["CLASSIC"] == (M + 3, 3 * M + 27, 4 * M + 30)
    assert want["QR"] == (2 * (M + 1), 10 * M + 24, 12 * M + 26)
    assert want["EXTRAP"] == (M + 1, 0, M + 1)
    assert want["SPEXTRAP"] == (m + 2, 0, m + 2)


def test_lebesgue_curves_golden_and_bounds():
    """The committed Lebesgue-constant curves (written from the oracle by
    tests/golden/make_lebesgue_curves.py) still follow from the oracle; every
    weight vector reproduces constants (sum beta = 1, hence Lambda >= 1); naive
    extrapolation has Lambda = 2^M - 1 and the degree-floor(sqrt(M)) fits stay
    below it (Sec. 6.6)."""
    rows = _golden_rows("lebesgue_curves.txt")
    assert [int(r[0]) for r in rows] == list(range(1, 17))
    for r in rows:
        M, m = int(r[0]), int(r[1])
        lam_naive, lam_lsq, lam_sp = float(r[2]), float(r[3]), float(r[4])
        b_lsq, b_sp = ex.lsq_coeffs(M, m), ex.sparse_coeffs(M, m)
        assert abs(ex.lebesgue_constant(b_lsq) - lam_lsq) <= 1e-12 * lam_lsq
        assert abs(ex.lebesgue_constant(b_sp) - lam_sp) <= 1e-12 * lam_sp
        assert lam_naive == 2.0 ** M - 1
        for b in (b_lsq, b_sp):
            assert abs(np.sum(b) - 1.0) <= 1e-12
        assert lam_lsq >= 1.0 - 1e-12 and lam_sp >= 1.0 - 1e-12
        assert lam_lsq <= lam_naive + 1e-9 and lam_sp <= lam_naive + 1e-9
        if m < M - 1:
            assert lam_lsq < lam_naive


# ---------------------------------------------------------------- sparse extrapolation pivots
def _greedy_farthest_points(M, m, tie_rel=1e-9):
    """Brute force of the pivot rule of Eq. CPQRCoeffs, independent of any QR:
    pivot k is the time point whose Legendre vector psi(t_i) = V^T e_i lies
    farthest (2-norm) from the span of the points already chosen, the distance
    taken from a dense least-squares fit; equal distances go to the most recent
    point.  Returns the pivot order and, per pivot, the relative margin between
    the winner's distance and the best distance that is not tied with it."""
    t, _ = ex.time_points(M)
    VT = ex.vandermonde(t, m).T
    chosen, margins = [], []
    for _ in range(m + 1):
        dist = {}
        for i in range(M):
            if i in chosen:
                continue
            col = VT[:, i]
            if chosen:
                B = VT[:, chosen]
                coef, *_ = np.linalg.lstsq(B, col, rcond=None)
                col = col - B @ coef
            dist[i] = float(np.linalg.norm(col))
        best = max(dist.values())
        tied = [i for i, d in dist.items() if d >= best * (1.0 - tie_rel)]
        rest = [d for i, d in dist.items() if i not in tied]
        margins.append((best - max(rest)) / best if rest else 1.0)
        chosen.append(max(tied))
    return chosen, margins


@pytest.mark.parametrize("M,m", [(4, 1), (6, 1), (8, 2), (10, 2), (12, 3), (16, 3), (16, 4), (12, 5), (8, 7)])
def test_sparse_pivots_are_greedy_farthest_points(M, m):
    """The oracle's column-pivoted QR picks, pivot by pivot, the same time points
    as the brute-force greedy rule (largest distance to the span of the chosen
    columns, ties to the most recent point).  Every non-tied runner-up is far
    from the winner, so the tie tolerance cannot decide the outcome."""
    want, margins = _greedy_farthest_points(M, m)
    assert min(margins) > 1e-6
    assert ex.sparse_pivots(M, m) == want
    assert sorted(np.flatnonzero(ex.sparse_coeffs(M, m)).tolist()) == sorted(want)


@pytest.mark.parametrize("M,m", [(8, 2), (12, 3), (16, 4), (16, 3), (12, 5)])
def test_sparse_points_cluster_at_the_ends(M, m):
    """Sec. 3.3: the chosen points show the end-point clustering of Chebyshev
    points -- both ends of the window are taken first (their Legendre vectors
    are the longest, |P_j(+-1)| = 1 >= |P_j(t)|), the most recent before the
    oldest, and no gap between chosen points next to an end is wider than the
    widest gap in the interior."""
    piv = ex.sparse_pivots(M, m)
    assert piv[:2] == [M - 1, 0]
    pts = sorted(piv)
    gaps = np.diff(pts)
    if len(gaps) >= 3:
        assert max(gaps[0], gaps[-1]) <= max(gaps[1:-1])
