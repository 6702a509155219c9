"""Time-stepped Helmholtz sequence, its loss and its reverse-time adjoint (FP64, CPU).

The sequence is the implicit time stepping whose systems the paper's guesses
serve (Sec. 5.2: each step solves a Helmholtz system (L + c I) u = rhs built
from the previous step, Eq. VelocityEqn).  In the form used here (backward
Euler for a forced heat equation, nu dt absorbed into lambda):

    A x_k = M (lam x_{k-1} + f_k),   A = K + lam M,   x_0 = 0,   k = 1..K

with K the SEM stiffness and M the GLL mass matrix (Sec. 5.1).  Loss
L = sum_k ||x_k - x*_k||^2.  With A and M symmetric, the adjoint variables
solve, backward in time,

    A g_k = 2 (x_k - x*_k) + lam M g_{k+1},   g_{K+1} = 0,

and the gradients are dL/df_k = M g_k and dL/dlam = sum_k g_k^T M (x_{k-1} - x_k)
(A depends on lam through M, the right-hand side through lam M x_{k-1}).
"""
import numpy as np
import scipy.linalg as sla

from .sem import SemOperator
from .pcg import pcg


class HeatSequence:
    def __init__(self, ex, ey, ez, p, lam, tol=1e-12, exact=False):
        self.E, self.p, self.lam, self.tol, self.exact = (ex, ey, ez), p, float(lam), tol, exact
        self.op = SemOperator(ex, ey, ez, p, lam)
        self.mass = SemOperator(ex, ey, ez, p, 1.0).diagonal() - SemOperator(ex, ey, ez, p, 0.0).diagonal()
        self.mass = self.mass * self.op.interior
        self.m = self.op.interior
        if exact:
            A = self.op.dense()
            idx = np.flatnonzero(self.m)
            self._idx = idx
            self._chol = sla.cho_factor(A[np.ix_(idx, idx)])
        else:
            self._diag = self.op.diagonal()

    def solve(self, b):
        if self.exact:
            x = np.zeros(self.op.n)
            x[self._idx] = sla.cho_solve(self._chol, b[self._idx])
            return x
        x, _, _, _ = pcg(self.op.apply, self._diag, b, np.zeros(self.op.n), self.tol, interior=self.m)
        return x

    def forward(self, F):
        """Solutions x_1..x_K for forcing rows F[k-1] (masked)."""
        x = np.zeros(self.op.n)
        xs = []
        for f in F:
            x = self.solve(self.mass * (self.lam * x + f))
            xs.append(x)
        return xs

    def loss(self, F, Xstar):
        return float(sum(np.sum((x - xt) ** 2 * self.m) for x, xt in zip(self.forward(F), Xstar)))

    def gradients(self, F, Xstar):
        """(loss, dL/dF (K x n), dL/dlam) by the reverse-time adjoint."""
        xs = self.forward(F)
        K = len(xs)
        L = float(sum(np.sum((x - xt) ** 2 * self.m) for x, xt in zip(xs, Xstar)))
        dF = np.zeros((K, self.op.n))
        dlam = 0.0
        g_next = np.zeros(self.op.n)
        for k in range(K - 1, -1, -1):
            rhs = (2.0 * (xs[k] - Xstar[k]) + self.lam * self.mass * g_next) * self.m
            g = self.solve(rhs)
            dF[k] = self.mass * g
            x_prev = xs[k - 1] if k > 0 else np.zeros(self.op.n)
            dlam += float(g @ (self.mass * (x_prev - xs[k])))
            g_next = g
        return L, dF, dlam
