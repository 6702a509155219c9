"""Differentiable time-stepped Helmholtz sequence (reverse-time adjoint).

Sequence (implicit time stepping; Helmholtz systems as in the paper's velocity
solves): A x_k = M (lam x_{k-1} + f_k), A = K + lam M, x_0 = 0, k = 1..K.
Loss L = sum_k ||x_k - x*_k||^2.  ``SequenceLoss`` is a torch.autograd.Function
of the forcing rows F (K x n) and lam.  Its backward runs the adjoint solves
A g_k = 2 (x_k - x*_k) + lam M g_{k+1} backward in time, each with its own
extrapolation/projection guess history, and returns dL/df_k = M g_k and
dL/dlam = sum_k g_k^T M (x_{k-1} - x_k).  The forward keeps only every
``checkpoint``-th solution; the backward recomputes each segment from its
checkpoint.  Every solve, right-hand side and accumulation runs in the
library's kernels; torch provides memory, the stream and the autograd plumbing.
"""
import ctypes

import torch

from . import Op, Guess, lib, _check, _ptr, _stream


class HeatSequence:
    def __init__(self, ex, ey, ez, p, tol=1e-10, s=6, m=2, method="extrap", checkpoint=10, maxit=20000):
        self.E, self.p = (int(ex), int(ey), int(ez)), int(p)
        self.tol, self.s, self.m, self.method = float(tol), int(s), int(m), method
        self.checkpoint, self.maxit = int(checkpoint), int(maxit)
        self._ops = {}
        self.last_iters = {"forward": [], "adjoint": []}

    def op(self, lam):
        lam = float(lam)
        if lam not in self._ops:
            if len(self._ops) > 4:
                self._ops.clear()
            self._ops[lam] = Op(*self.E, self.p, lam, "f64")
        return self._ops[lam]

    def _ws(self, op):
        nb = int(lib().sg_seq_workspace_bytes(op.h))
        return torch.zeros(nb, dtype=torch.uint8, device="cuda")

    def _guess(self, op):
        return Guess(op.n, self.s, self.method, m=self.m, eps_rel=self.tol, op=op)

    def _step(self, op, g, lam, x_prev, f, rhs, iters):
        """x_k for A x_k = M (lam x_{k-1} + f_k), solved in the guess's next slot."""
        _check(lib().sg_mass_rhs(op.h, float(lam), _ptr(x_prev) if x_prev is not None else None,
                                 _ptr(f), _ptr(rhs), _stream()))
        x = g.next_slot()
        if x is None:
            x = op.zeros()
        g.form(rhs, x)
        # no true-residual pass: the sequence needs the solution and the count only
        it, _ = op.pcg(rhs, x, self.tol, maxit=self.maxit, true_residual=False)
        g.update(x)
        iters.append(it)
        return x

    def forward_loss(self, F, lam, Xstar):
        """Loss (device 0-d FP64 tensor) and the checkpoints {k: x_k}."""
        op = self.op(lam)
        K = F.shape[0]
        ws = self._ws(op)
        acc = torch.zeros(1, dtype=torch.float64, device="cuda")
        g = self._guess(op)
        rhs = op.empty()
        x_prev = None
        ckpt = {0: op.zeros()}
        iters = []
        for k in range(K):
            x = self._step(op, g, lam, x_prev, F[k], rhs, iters)
            _check(lib().sg_sqdiff_accum(op.h, _ptr(x), _ptr(Xstar[k]), ctypes.c_void_p(acc.data_ptr()),
                                         _ptr(ws), _stream()))
            if (k + 1) % self.checkpoint == 0 and k + 1 < K:
                ckpt[k + 1] = x.clone()
            x_prev = x
        self.last_iters["forward"] = iters
        return acc[0], ckpt

    def adjoint(self, F, lam, Xstar, ckpt):
        """dL/dF (K x n) and dL/dlam by the reverse-time adjoint with recomputation."""
        op = self.op(lam)
        K = F.shape[0]
        ws = self._ws(op)
        dlam = torch.zeros(1, dtype=torch.float64, device="cuda")
        dF = torch.empty_like(F)
        g_adj = self._guess(op)              # the adjoint sequence's own history
        rhs = op.empty()
        g_next = None
        starts = sorted(ckpt.keys())
        iters_adj, iters_fwd = [], []
        gbuf = [op.zeros(), op.zeros()]       # projection guesses have no ring slot
        nstep = 0
        for c0 in reversed(starts):
            c1 = min(K, next((c for c in starts if c > c0), K))
            # recompute x_{c0+1..c1} from the checkpoint (fresh forward history)
            gf = self._guess(op)
            xs = [ckpt[c0]]
            for k in range(c0, c1):
                x = self._step(op, gf, lam, xs[-1] if k > 0 else None, F[k], rhs, iters_fwd)
                xs.append(x.clone())
            for k in range(c1 - 1, c0 - 1, -1):          # 0-based step k solves for x_{k+1}
                x_k, x_km1 = xs[k - c0 + 1], xs[k - c0]
                _check(lib().sg_adjoint_rhs(op.h, 2.0, _ptr(x_k), _ptr(Xstar[k]), float(lam),
                                            _ptr(g_next) if g_next is not None else None, _ptr(rhs), _stream()))
                gk = g_adj.next_slot()
                if gk is None:
                    gk = gbuf[nstep % 2]
                nstep += 1
                g_adj.form(rhs, gk)
                it, _ = op.pcg(rhs, gk, self.tol, maxit=self.maxit, true_residual=False)
                g_adj.update(gk)
                iters_adj.append(it)
                _check(lib().sg_adjoint_accum(op.h, _ptr(gk), _ptr(x_km1) if k > 0 else None, _ptr(x_k),
                                              _ptr(dF[k]), ctypes.c_void_p(dlam.data_ptr()), _ptr(ws), _stream()))
                g_next = gk
        self.last_iters["adjoint"] = iters_adj
        self.last_iters["recompute"] = iters_fwd
        return dF, dlam[0]


class SequenceLoss(torch.autograd.Function):
    """L(F, lam) = sum_k ||x_k - x*_k||^2 for the sequence of ``seq``."""

    @staticmethod
    def forward(ctx, F, lam, Xstar, seq):
        F = F.detach().contiguous()
        lam_v = float(lam)
        L, ckpt = seq.forward_loss(F, lam_v, Xstar)
        ctx.seq, ctx.lam, ctx.ckpt = seq, lam_v, ckpt
        ctx.save_for_backward(F, Xstar)
        return L.clone()

    @staticmethod
    def backward(ctx, gL):
        F, Xstar = ctx.saved_tensors
        dF, dlam = ctx.seq.adjoint(F, ctx.lam, Xstar, ctx.ckpt)
        return gL * dF, (gL * dlam).reshape(()), None, None
