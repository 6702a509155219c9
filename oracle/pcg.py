"""Jacobi-preconditioned conjugate gradients (FP64, CPU).

Sec. 5.3: the velocity Helmholtz systems are solved by PCG with a point-Jacobi
preconditioner; this library uses the same solver for every system.  The
iteration is the textbook preconditioned Hestenes-Stiefel CG.

Stopping rules (Sec. 6.4), checked on the recursively updated, unpreconditioned
residual r_k before each iteration (0 iterations if the initial guess already
satisfies the rule):

* ``REL_B`` (0):  ||r_k|| <= tol * ||b||              -- "relative residual"
* ``INITRESID`` (1): ||r_k|| < tol * max(||r_0||, 1)  -- Eq. StopCritINITRESID
* ``RHS`` (2):    ||r_k|| < tol * max(||b||, 1)       -- Eq. StopCritRHS
"""
import numpy as np

REL_B, INITRESID, RHS = 0, 1, 2


def stop_threshold(criterion, tol, bnorm, r0norm):
    if criterion == REL_B:
        return tol * bnorm, False
    if criterion == INITRESID:
        return tol * max(r0norm, 1.0), True
    if criterion == RHS:
        return tol * max(bnorm, 1.0), True
    raise ValueError("unknown criterion")


def converged(rnorm, thr, strict):
    return rnorm < thr if strict else rnorm <= thr


def pcg(apply_A, diag, b, x0, tol, maxit=10000, criterion=REL_B, interior=None):
    """Solve A x = b.  Returns (x, iterations, true relative residual, history).

    ``interior`` masks the Dirichlet nodes: r, z and p are kept 0 there.
    """
    b = np.asarray(b, dtype=np.float64)
    x = np.array(x0, dtype=np.float64, copy=True)
    m = np.ones_like(b) if interior is None else interior.astype(np.float64)
    x *= m
    r = (b - apply_A(x)) * m
    bnorm = np.sqrt(np.dot(b * m, b * m))
    rnorm = np.sqrt(np.dot(r, r))
    thr, strict = stop_threshold(criterion, tol, bnorm, rnorm)
    hist = [rnorm]
    it = 0
    if not converged(rnorm, thr, strict):
        z = r / diag * m
        p = z.copy()
        rz = np.dot(r, z)
        while it < maxit:
            q = apply_A(p)
            pq = np.dot(p, q)
            if not pq > 0.0:
                raise FloatingPointError("PCG breakdown: p^T A p <= 0")
            alpha = rz / pq
            x += alpha * p
            r -= alpha * q
            it += 1
            rnorm = np.sqrt(np.dot(r, r))
            hist.append(rnorm)
            if converged(rnorm, thr, strict):
                break
            z = r / diag * m
            rz_new = np.dot(r, z)
            beta = rz_new / rz
            rz = rz_new
            p = z + beta * p
    true_res = np.linalg.norm((b - apply_A(x)) * m)
    rel = true_res / bnorm if bnorm > 0 else true_res
    return x, it, rel, hist
