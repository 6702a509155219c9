"""Per-time-step driver: form guess, solve with Jacobi-PCG, update history.

Sec. 5.2 / 6.2: one linear system per time step, each solved by PCG from an
initial guess built out of the stored history.  Methods (Sec. 4, Table 1
nomenclature): ZERO, LAST, EXTRAP(m, M), SPEXTRAP(m, M), QR(M), CLASSIC(M), and
ENERGY(M), the rolling window of QR(M) in the energy inner product.
"""
import numpy as np

from . import extrap as ex
from .pcg import pcg, REL_B
from .proj import ProjectionQR, ProjectionClassic, ProjectionEnergy

ZERO, LAST, EXTRAP, PROJ_QR, PROJ_CLASSIC, SPEXTRAP, PROJ_ENERGY = 0, 1, 2, 3, 4, 5, 6


class ExtrapHistory:
    """Ring of the last M solutions; guess by Eq. ExtrapExpn."""

    def __init__(self, M, m, sparse=False):
        self.M, self.m, self.sparse = int(M), int(m), bool(sparse)
        self.hist = []      # oldest first

    def coeffs(self):
        return ex.startup_coeffs(len(self.hist), self.M, self.m, self.sparse)

    def form(self, b, x0):
        if not self.hist:
            return np.array(x0, dtype=np.float64, copy=True)
        return ex.extrap_guess(self.hist, self.coeffs())

    def update(self, x, b=None):
        self.hist.append(np.array(x, dtype=np.float64, copy=True))
        if len(self.hist) > self.M:
            self.hist.pop(0)
        return True


class ZeroGuess:
    def form(self, b, x0):
        return np.zeros_like(np.asarray(b, dtype=np.float64))

    def update(self, x, b=None):
        return True


class LastGuess:
    def __init__(self):
        self.last = None

    def form(self, b, x0):
        if self.last is None:
            return np.array(x0, dtype=np.float64, copy=True)
        return self.last.copy()

    def update(self, x, b=None):
        self.last = np.array(x, dtype=np.float64, copy=True)
        return True


def make_guesser(method, op, s, m=None, eps_rel=1e-10):
    if method == ZERO:
        return ZeroGuess()
    if method == LAST:
        return LastGuess()
    if method in (EXTRAP, SPEXTRAP):
        m = int(np.floor(np.sqrt(s))) if m is None else m
        return ExtrapHistory(s, m, sparse=(method == SPEXTRAP))
    if method == PROJ_QR:
        return ProjectionQR(s, eps_rel, op.apply)
    if method == PROJ_CLASSIC:
        return ProjectionClassic(s, eps_rel, op.apply)
    if method == PROJ_ENERGY:
        return ProjectionEnergy(s, eps_rel, op.apply)
    raise ValueError("unknown method")


def run_sequence(op, rhs, method, s, m=None, tol=1e-10, maxit=10000,
                 criterion=REL_B, eps_rel=None, keep=False):
    """Solve A x_k = b_k for every b_k in ``rhs`` (an iterable).

    Returns a list of per-step dicts: iterations, true relative residual,
    initial relative residual ||b - A x0|| / ||b||, and (if ``keep``) x0, x.
    """
    eps_rel = tol if eps_rel is None else eps_rel
    g = make_guesser(method, op, s, m, eps_rel)
    diag = op.diagonal()
    out = []
    for b in rhs:
        b = np.asarray(b, dtype=np.float64)
        x0 = g.form(b, np.zeros_like(b))
        r0 = np.linalg.norm((b - op.apply(x0)) * op.interior)
        bn = np.linalg.norm(b * op.interior)
        x, it, rel, _ = pcg(op.apply, diag, b, x0, tol, maxit, criterion, op.interior)
        g.update(x, b)
        rec = {"iters": it, "relres": rel, "r0": r0 / bn if bn > 0 else r0}
        if keep:
            rec["x0"], rec["x"] = x0, x
        out.append(rec)
    return out
