"""Small driver that runs every kernel of the library once or a few times on a
mesh of the bench's shapes, for profiling (ncu) and quick timing.

    python -m paper_2009_10863_gb300.profile_run --elements 16 --dtype f64
    python -m paper_2009_10863_gb300.profile_run --steps 6
    python -m paper_2009_10863_gb300.profile_run --batched

The first form applies the operator `--reps` times (timed with CUDA events),
runs a few PCG iterations (host-launched, as with kernel timing on), forms an
EXTRAP(2,8) guess and performs QR(8) history updates.  The second runs time
steps of bench.py's main sequence (FP64 16^3 p = 7 Helmholtz, EXTRAP(2,8),
1e-10) with every library launch timed by CUDA events, so that the PCG
iterations are host launches that a profiler lists one by one (bench.py's
timed steps run them inside CUDA-graph WHILE loops).  The third solves the
four batched systems once (the persistent kernel, one launch per iteration).
"""
import argparse

import numpy as np
import torch

import paper_2009_10863_gb300 as sg


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--elements", type=int, default=16)
    ap.add_argument("--p", type=int, default=7)
    ap.add_argument("--lam", type=float, default=1e5)
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--pcg-iters", type=int, default=6)
    ap.add_argument("--s", type=int, default=8)
    ap.add_argument("--steps", type=int, default=0)
    ap.add_argument("--batched", action="store_true")
    args = ap.parse_args()
    from paper_2009_10863_gb300 import build
    build.build()
    if args.steps > 0:
        return sequence_steps(args.steps)
    if args.batched:
        return batched_solve()
    E = args.elements
    op = sg.Op(E, E, E, args.p, args.lam, args.dtype)
    gen = torch.Generator(device="cuda").manual_seed(0)
    x = torch.randn(op.n, dtype=op.dtype, device="cuda", generator=gen)
    y = op.empty()
    for _ in range(args.reps):
        op.apply(x, out=y)
    b = op.apply(x)
    xs = op.zeros()
    sg.profile_reset()
    sg.profile_enable(True)      # host-launched iterations: each kernel is a separate launch
    it, _ = op.pcg(b, xs, 1e-10, maxit=args.pcg_iters)
    sg.profile_enable(False)
    t_apply, n_apply = sg.profile_read(sg.PROF_PCG_APPLY)
    t_upd, n_upd = sg.profile_read(sg.PROF_PCG_UPDATE)
    g = sg.Guess(op.n, args.s, "extrap", m=2, dtype=args.dtype)
    q = sg.Guess(op.n, args.s, "qr", eps_rel=1e-6, op=op, dtype=args.dtype)
    for k in range(args.s + 1):          # independent vectors: the QR history fills to d = s
        v = x + 0.1 * torch.randn(op.n, dtype=op.dtype, device="cuda", generator=gen)
        g.update(v)
        q.update(v)
    x0 = op.zeros()
    g.form(None, x0)
    q.form(b, x0)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(20):
        op.apply(x, out=y)
    e1.record()
    torch.cuda.synchronize()
    print("nodes %d dtype %s apply %.1f us, pcg iterations %d (step %.1f us, update %.1f us), qr d=%d" %
          (op.n, args.dtype, 1000 * e0.elapsed_time(e1) / 20, it, 1e3 * t_apply / max(n_apply, 1),
           1e3 * t_upd / max(n_upd, 1), q.info()[0]))


def batched_solve():
    """One solve of the four batched systems (24^3 Poisson, 20^3, 16^3, 12^3
    Helmholtz, p = 7; FP32 PCG in FP64 refinement, one persistent launch per
    CG iteration) from zero, right-hand sides A x for random x; no tuning."""
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from synthetic import BATCHED
    meshes = [(c["E"][0], c["E"][1], c["E"][2], c["lam"]) for c in BATCHED]
    solver = sg.BatchSolver(meshes)
    gen = torch.Generator(device="cuda").manual_seed(0)
    bs, xs = [], []
    for c in BATCHED:
        op = sg.Op(*c["E"], c["p"], c["lam"], "f64")
        bs.append(op.apply(torch.randn(op.n, dtype=torch.float64, device="cuda", generator=gen)))
        xs.append(op.zeros())
    sg.profile_enable(True)      # replay form: the persistent launches are plain graph kernel nodes
    outer, inner, rel = solver.solve(bs, xs, 1e-10)
    torch.cuda.synchronize()
    sg.profile_enable(False)
    print("batched: outer", outer, "inner", inner, "relres %.2e" % max(rel))


def sequence_steps(steps):
    import os
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    from bench import Workload, CFG
    wl = Workload(sg, torch, steps, torch.device("cuda", 0))
    op = wl.op
    g = sg.Guess(op.n, CFG["s"], "extrap", m=2, eps_rel=CFG["tol"], op=op)
    sg.profile_reset()
    sg.profile_enable(True)
    iters = []
    for k in range(steps):
        x = g.next_slot()
        g.form(wl.rhs[k], x)
        it, _ = op.pcg(wl.rhs[k], x, CFG["tol"], true_residual=False)
        g.update(x)
        iters.append(it)
    torch.cuda.synchronize()
    sg.profile_enable(False)
    for name, kid in (("pcg_apply", sg.PROF_PCG_APPLY), ("pcg_update", sg.PROF_PCG_UPDATE),
                      ("extrap", sg.PROF_EXTRAP)):
        t, c = sg.profile_read(kid)
        print("%-10s %5d launches %9.1f us" % (name, c, 1e3 * t))
    print("iterations per step", iters)


if __name__ == "__main__":
    main()
