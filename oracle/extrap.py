"""Polynomial extrapolation coefficients and the extrapolated guess (FP64, CPU).

Sec. 3.2 (stabilised least squares).  History data x_{n-M+1}, ..., x_n sit at
the equispaced points t_i = -1 + (i-1) h, h = 2/(M-1), i = 1..M, and the guess
is evaluated at t_new = 1 + h.  With V_ij = psi_j(t_i) (Legendre psi_j,
j = 0..m) and v_j = psi_j(t_new), Eq. LSQRCoeffs gives

    beta^T = v^T (V^T V)^{-1} V^T,

computed here through a Householder QR of V (V = Q R, so beta = Q R^{-T} v)
rather than the normal equations.  Eq. ExtrapExpn forms the guess
x_hat = sum_i beta_i x_{n-M+i}, beta_1 multiplying the oldest solution.

Sec. 3.3 (sparse extrapolation), Eq. CPQRCoeffs: with a column-pivoted QR
V^T P = Q R, R = [R_hat R_tilde], beta = P [R_hat^{-1} Q^T v ; 0] has m+1
non-zeros.

Readings where the paper is silent:
* M = 1: h is undefined; beta = [1] (the previous-solution guess, Sec. 3.1).
* start-up (fewer than M solutions stored): use M' = min(k, M) solutions and
  degree m' = min(m, M'-1).
* column pivoting (sparse): Businger-Golub, largest remaining column 2-norm,
  norms recomputed at every step; ties within 64 ulp go to the most recent
  time point.
"""
import numpy as np
from numpy.polynomial import legendre as L


def time_points(M):
    """Equispaced points t_1..t_M on [-1, 1] and the new point t_{n+1} = 1 + h."""
    if M == 1:
        return np.array([0.0]), None
    h = 2.0 / (M - 1)
    t = -1.0 + h * np.arange(M)
    return t, 1.0 + h


def vandermonde(t, m):
    """V_ij = P_j(t_i), Legendre P_j, j = 0..m."""
    return L.legvander(np.asarray(t, dtype=np.float64), m)


def lsq_coeffs(M, m):
    """beta for EXTRAP(m, M) by Eq. LSQRCoeffs, via Householder QR of V."""
    if M < 1 or m < 0 or m > M - 1:
        raise ValueError("need 0 <= m <= M-1")
    if M == 1:
        return np.array([1.0])
    t, tn = time_points(M)
    V = vandermonde(t, m)
    v = vandermonde([tn], m)[0]
    Q, R = np.linalg.qr(V, mode='reduced')
    y = np.linalg.solve(R.T, v)          # R^T y = v
    return Q @ y


def _cpqr(M, m):
    """Column-pivoted Householder QR of V^T (Sec. 3.3, Eq. CPQRCoeffs).

    Returns the pivot order (time-point indices, first pivot first) and the
    m+1 non-zero coefficients R_hat^{-1} Q^T v in that order.  Pivot j is the
    remaining column of largest 2-norm below row j, i.e. the time point whose
    Legendre vector psi(t_i) is farthest from the span of the points already
    chosen (Businger & Golub, Numer. Math. 7, 1965)."""
    t, tn = time_points(M)
    VT = vandermonde(t, m).T.copy()      # (m+1) x M
    v = vandermonde([tn], m)[0]
    k = m + 1
    A = VT.copy()
    perm = list(range(M))
    Qt = np.eye(k)                       # accumulates Q^T
    for j in range(k):
        norms = np.array([np.linalg.norm(A[j:, c]) for c in range(j, M)])
        best = np.max(norms)
        tolx = 64.0 * np.finfo(float).eps * best
        cands = [j + c for c in range(len(norms)) if norms[c] >= best - tolx]
        piv = max(cands, key=lambda c: perm[c])   # tie -> most recent time point
        A[:, [j, piv]] = A[:, [piv, j]]
        perm[j], perm[piv] = perm[piv], perm[j]
        # Householder reflector zeroing A[j+1:, j]
        xcol = A[j:, j].copy()
        alpha = -np.copysign(np.linalg.norm(xcol), xcol[0] if xcol[0] != 0 else 1.0)
        u = xcol.copy()
        u[0] -= alpha
        un = np.linalg.norm(u)
        if un > 0:
            u /= un
            A[j:, :] -= 2.0 * np.outer(u, u @ A[j:, :])
            Qt[j:, :] -= 2.0 * np.outer(u, u @ Qt[j:, :])
    Rhat = np.triu(A[:, :k])
    bhat = np.linalg.solve(Rhat, Qt @ v)
    return perm[:k], bhat


def sparse_pivots(M, m):
    """Time-point indices (0 = oldest) chosen by the pivoted QR, in pivot order."""
    if M < 1 or m < 0 or m > M - 1:
        raise ValueError("need 0 <= m <= M-1")
    if M == 1:
        return [0]
    return _cpqr(M, m)[0]


def sparse_coeffs(M, m):
    """beta for SPEXTRAP(m, M) by Eq. CPQRCoeffs (column-pivoted QR of V^T)."""
    if M < 1 or m < 0 or m > M - 1:
        raise ValueError("need 0 <= m <= M-1")
    if M == 1:
        return np.array([1.0])
    piv, bhat = _cpqr(M, m)
    beta = np.zeros(M)
    for j, i in enumerate(piv):
        beta[i] = bhat[j]
    return beta


def startup_coeffs(k, M, m, sparse=False):
    """Coefficients when only k solutions are stored (reading: M'=min(k,M))."""
    Mp = min(k, M)
    if Mp == 0:
        return np.zeros(0)
    mp = min(m, Mp - 1)
    return sparse_coeffs(Mp, mp) if sparse else lsq_coeffs(Mp, mp)


def naive_coeffs(M):
    """Eq. NaiveExtrapCoeffs: beta_i = (-1)^(M-i) * C(M, i-1)."""
    from math import comb
    return np.array([(-1) ** (M - i) * comb(M, i - 1) for i in range(1, M + 1)], dtype=np.float64)


def lebesgue_constant(beta):
    """Sec. 6.6: Lambda = ||beta||_1."""
    return float(np.sum(np.abs(beta)))


def extrap_guess(history, beta):
    """Eq. ExtrapExpn: sum_i beta_i x_{n-M+i}; ``history`` is oldest first."""
    x = np.zeros_like(np.asarray(history[0], dtype=np.float64))
    for b, h in zip(beta, history):
        x = x + b * np.asarray(h, dtype=np.float64)
    return x
