"""FP64 CPU oracle for the initial-guess / SEM / Jacobi-PCG path.

This package is TEST INFRASTRUCTURE. It is a plain, slow, obviously correct
restatement in numpy (float64) of what the GPU library computes. Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl reference``
legs of ``bench.py`` may import it. The GPU library never imports it. The two
share no code: the only module both sides use is ``synthetic``, the seeded
workload generator, and it holds none of the method's arithmetic.

Each function cites the part of Austin, Chalmers & Warburton, "Initial Guesses
for Sequences of Linear Systems in a GPU-Accelerated Incompressible Flow
Solver" (arXiv:2009.10863) that it follows:

* ``gll``     -- tensor-product GLL basis (Sec. 5.1).
* ``sem``     -- matrix-free SEM Poisson/Helmholtz operator, element by element
                 with an explicit gather-scatter (Sec. 5.1, Eqs. VelocityEqn and
                 PressureEqn).
* ``pcg``     -- Jacobi-preconditioned CG with the paper's stopping rules
                 (Sec. 5.3; Sec. 6.4, Eqs. StopCritINITRESID and StopCritRHS).
* ``extrap``  -- least-squares (Eq. LSQRCoeffs) and sparse (Eq. CPQRCoeffs)
                 polynomial extrapolation (Sec. 3).
* ``proj``    -- right-hand-side projection: rolling QR (Algorithm 2) and the
                 classic restarted form (Algorithm 1).
* ``sequence``-- the per-time-step driver: form guess, solve, update history.
* ``adjoint`` -- reverse-time adjoint of a time-stepped Helmholtz sequence.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against
something other than itself (closed forms, textbook reductions, brute force).
"""
