"""Right-hand-side projection guesses (FP64, CPU): Algorithms 1 and 2, and the
same rolling window in the energy inner product (ProjectionEnergy).

Sec. 2: with an orthonormal basis B~ of the stored right-hand sides and the
matching solutions X~ (A X~ = B~), the guess for A x = b is x0 = X~ B~^T b,
the combination of stored solutions that minimises ||b - A x||_2 over their
span.  Updates use twice-iterated classical Gram-Schmidt (CGS2): all inner
products of a pass are taken before the pass subtracts anything.

Algorithm 2 ("rolling QR", Christensen): once d = M, the oldest column is
dropped by deleting the first column of R and restoring the triangular shape
with d-1 Givens rotations applied to R's rows and to column pairs of B~, X~.

Readings where the printed text is garbled or silent:
* Givens step: after R <- R(:, 2:d) the entry to annihilate is R(i+1, i).
  a = R(i,i), b = R(i+1,i), r = sqrt(a^2+b^2), c = |a|/r, s = sign(a) b / r,
  G = [[c, s], [-s, c]]; the new diagonal is sign(a) r (it keeps the sign
  of a, so R may carry negative diagonal entries).  sign(0) = +1.
* epsilon test: "small relative to b" -- accept the new direction when
  ||b~ after CGS2|| > eps_rel * ||A x|| (A x before orthogonalisation).
* d = 0 with ||A x|| = 0 (a zero solution): nothing is stored.
* Algorithm 1 restarts (keeps only the new vector) when d = 0 or d >= M,
  which gives the 1..M cycle used for its average data movement (App. A).
"""
import numpy as np


def _sign(a):
    return 1.0 if a >= 0.0 else -1.0


class ProjectionQR:
    """Algorithm 2 with history size M."""

    def __init__(self, M, eps_rel, apply_A):
        self.M, self.eps_rel, self.apply_A = int(M), float(eps_rel), apply_A
        self.B = []          # orthonormal right-hand-side basis, oldest first
        self.X = []          # matching solutions
        self.R = np.zeros((self.M + 1, self.M + 1))
        self.accepted = []   # bookkeeping for tests: raw solutions in the window

    @property
    def d(self):
        return len(self.B)

    def form(self, b, x0):
        """x0 = X~ B~^T b when d > 0, else the caller's x0."""
        if self.d == 0:
            return np.array(x0, dtype=np.float64, copy=True)
        c = np.array([np.dot(Bi, b) for Bi in self.B])
        x = np.zeros_like(np.asarray(b, dtype=np.float64))
        for ci, Xi in zip(c, self.X):
            x = x + ci * Xi
        return x

    def _downdate(self):
        d = self.d
        R = self.R[:d, 1:d].copy()           # d x (d-1), upper Hessenberg
        B = [v.copy() for v in self.B]
        X = [v.copy() for v in self.X]
        for i in range(d - 1):
            a, bb = R[i, i], R[i + 1, i]
            r = np.hypot(a, bb)
            if r == 0.0:
                c, s = 1.0, 0.0
            else:
                c, s = abs(a) / r, _sign(a) * bb / r
            G = np.array([[c, s], [-s, c]])
            R[i:i + 2, :] = G @ R[i:i + 2, :]
            Bi, Bj = B[i], B[i + 1]
            B[i], B[i + 1] = c * Bi + s * Bj, -s * Bi + c * Bj     # [Bi Bj] G^T
            Xi, Xj = X[i], X[i + 1]
            X[i], X[i + 1] = c * Xi + s * Xj, -s * Xi + c * Xj
        self.R[:, :] = 0.0
        self.R[:d - 1, :d - 1] = R[:d - 1, :]
        self.B, self.X = B[:d - 1], X[:d - 1]
        self.accepted = self.accepted[1:]

    def update(self, x, b=None):
        """History update after the solve (Algorithm 2, after the solve line)."""
        xt = np.array(x, dtype=np.float64, copy=True)
        bt = self.apply_A(xt)
        nrm0 = np.linalg.norm(bt)
        if self.d == self.M:
            self._downdate()
        d = self.d
        if d == 0:
            if nrm0 > 0.0:
                self.R[0, 0] = nrm0
                self.B, self.X = [bt / nrm0], [xt / nrm0]
                self.accepted = [np.array(x, dtype=np.float64)]
            return True
        rcol = np.zeros(d)
        for _ in range(2):                    # CGS2
            c = np.array([np.dot(Bi, bt) for Bi in self.B])
            for ci, Bi, Xi in zip(c, self.B, self.X):
                bt = bt - ci * Bi
                xt = xt - ci * Xi
            rcol += c
        nb = np.linalg.norm(bt)
        if nb > self.eps_rel * nrm0:
            self.R[:d, d] = rcol
            self.R[d, d] = nb
            self.B.append(bt / nb)
            self.X.append(xt / nb)
            self.accepted.append(np.array(x, dtype=np.float64))
            return True
        return False


class ProjectionClassic:
    """Algorithm 1 (hard restart) with history size M."""

    def __init__(self, M, eps_rel, apply_A):
        self.M, self.eps_rel, self.apply_A = int(M), float(eps_rel), apply_A
        self.B, self.X = [], []

    @property
    def d(self):
        return len(self.B)

    form = ProjectionQR.form

    def update(self, x, b=None):
        xt = np.array(x, dtype=np.float64, copy=True)
        bt = self.apply_A(xt)
        nrm0 = np.linalg.norm(bt)
        if self.d == 0 or self.d >= self.M:
            if nrm0 > 0.0:
                self.B, self.X = [bt / nrm0], [xt / nrm0]
            else:
                self.B, self.X = [], []
            return True
        for _ in range(2):
            c = np.array([np.dot(Bi, bt) for Bi in self.B])
            for ci, Bi, Xi in zip(c, self.B, self.X):
                bt = bt - ci * Bi
                xt = xt - ci * Xi
        nb = np.linalg.norm(bt)
        if nb > self.eps_rel * nrm0:
            self.B.append(bt / nb)
            self.X.append(xt / nb)
            return True
        return False


class ProjectionEnergy:
    """Projection in the energy inner product (x, y)_A = x^T A y, history size M.

    Fischer's form of the projection (Comput. Methods Appl. Mech. Engrg. 163,
    1998) keeps X~ A-orthonormal (X~^T A X~ = I) with B~ = A X~; the guess
    x0 = X~ X~^T b is the A-orthogonal projection of the solution A^{-1} b onto
    span(X~), i.e. it minimises ||x - A^{-1} b||_A there (Sec. 2 states the
    Euclidean ||b - A x||_2 form).  The history is the rolling window of
    Algorithm 2 with every inner product taken in the A-inner product: CGS2
    coefficients c = X~^T (A x) (= (x~_j, x)_A), the norm ||x~||_A =
    sqrt(x~^T b~), the R factor X_window = X~ R, and the same Givens downdate
    when d = M (a rotation of A-orthonormal columns stays A-orthonormal).
    Reading of the acceptance test: keep the new direction when
    ||x~ after CGS2||_A > eps_rel * ||x||_A.
    """

    def __init__(self, M, eps_rel, apply_A):
        self.M, self.eps_rel, self.apply_A = int(M), float(eps_rel), apply_A
        self.B, self.X = [], []
        self.R = np.zeros((self.M + 1, self.M + 1))
        self.accepted = []

    @property
    def d(self):
        return len(self.X)

    def form(self, b, x0):
        """x0 = X~ X~^T b when d > 0, else the caller's x0."""
        if self.d == 0:
            return np.array(x0, dtype=np.float64, copy=True)
        c = np.array([np.dot(Xi, b) for Xi in self.X])
        x = np.zeros_like(np.asarray(b, dtype=np.float64))
        for ci, Xi in zip(c, self.X):
            x = x + ci * Xi
        return x

    _downdate = ProjectionQR._downdate

    def update(self, x, b=None):
        xt = np.array(x, dtype=np.float64, copy=True)
        bt = self.apply_A(xt)
        nrm0 = np.sqrt(max(float(np.dot(xt, bt)), 0.0))
        if self.d == self.M:
            self._downdate()
        d = self.d
        if d == 0:
            if nrm0 > 0.0:
                self.R[0, 0] = nrm0
                self.B, self.X = [bt / nrm0], [xt / nrm0]
                self.accepted = [np.array(x, dtype=np.float64)]
            return True
        rcol = np.zeros(d)
        for _ in range(2):                    # CGS2 in the A-inner product
            c = np.array([np.dot(Xi, bt) for Xi in self.X])
            for ci, Bi, Xi in zip(c, self.B, self.X):
                bt = bt - ci * Bi
                xt = xt - ci * Xi
            rcol += c
        nn = float(np.dot(xt, bt))
        nb = np.sqrt(nn) if nn > 0.0 else 0.0
        if nb > self.eps_rel * nrm0:
            self.R[:d, d] = rcol
            self.R[d, d] = nb
            self.B.append(bt / nb)
            self.X.append(xt / nb)
            self.accepted.append(np.array(x, dtype=np.float64))
            return True
        return False
