"""Benchmark: ms per time-step solve at 1e-10 relative residual, CG iterations,
and guess-kernel HBM bandwidth, on one GB300 (or N replicas).

Workload (one "step" = form guess + Jacobi-PCG solve + history update, i.e.
one pass of the whole hot path over one right-hand side):
  FP64 Helmholtz -Lap + lambda on 16x16x16 elements, p = 7 (113^3 = 1,442,897
  nodes), lambda = 1/(nu dt) = 1e5; b_k = A x*(t_k) + noise, x* = 32 seeded
  space-time sine modes, noise std 1e-6 RMS(A x*); history s = 8; PCG to
  ||r|| <= 1e-10 ||b||.  Headline guess: EXTRAP(2, 8) (stabilised least
  squares, Sec. 3.2); ZERO, LAST and QR(8) (Algorithm 2) are reported beside.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Profiling drivers (short runs for ncu; they print no bench line):
  python bench.py --profile-driver ops --elements 16 --dtype f64   each kernel once or a few times
  python bench.py --profile-driver steps --prof-steps 14          headline steps, launches timed one by one
  python bench.py --profile-driver batched                        one solve of the four batched systems
"""
import argparse
import datetime
import json
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synthetic import forcing_basis_indices, adjoint_parameters, BATCHED, BATCHED_COMMON, CONFIGS, Modes, noise  # noqa: E402

METRIC = "ms per time-step solve at 1e-10 rel. residual + CG iters; guess-kernel HBM GB/s"
CFG = CONFIGS["helmholtz_16x16x16_p7"]
HEADLINE = ("extrap", 2)          # EXTRAP(m=2, s=8)
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12   # SMs x DFMA/clk/SM x 2 flop x max clock
L2_FLUSH_BYTES = 512 << 20
CPU_BASELINE_STEPS = 5            # complete oracle steps timed for cpu_baseline (~1.3 s each)
# DRAM bytes per launch of the dominant kernel (k_sem<double,7,1>, not the first
# PCG iteration) from one ncu capture of the current kernel; None once it changes
PCG_APPLY_TRAFFIC = 33921792 + 256  # read + write of the not-first MODE 1 launch (sem16d capture)


def aggregate_max(value, dist, device):
    """Max of a per-rank value over all ranks (replicas: the slowest rank decides)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload_name():
    E = CFG["E"]
    return "helmholtz-%dx%dx%d-p%d-fp64-%s" % (E[0], E[1], E[2], CFG["p"], "extrap(2,8)")


def fp64_frac(ops_per_node, n, avg_ms):
    """Fraction of the FP64 operation rate (2 per clock per SM) a kernel of
    ops_per_node FP64 operations per node over n nodes reaches in avg_ms."""
    if not avg_ms:
        return None
    return ops_per_node * n / (avg_ms * 1e-3) / (FP64_PEAK_TFLOPS * 1e12 / 2)


def sem_flops_per_element(p):
    """Algorithmic flops of one operator application per element, the affine
    sum-factorised count: per direction an (p+1)x(p+1) matrix on each of the
    (p+1)^2 element lines, 2 (p+1)^4 flop, three directions 6 (p+1)^4, plus the
    O((p+1)^3) pointwise work (mass term, sums, weights) counted as 8 (p+1)^3.
    p = 7: 28,672 flop per element."""
    return 6.0 * (p + 1) ** 4 + 8.0 * (p + 1) ** 3


def sem_flops_per_node(p):
    """Algorithmic flops per node of one assembled sum-factorised operator
    application on the affine box: per direction an element-line dot of p+1
    terms (plus the neighbouring element's line for the 1/p shared nodes and
    the z-carry), i.e. 3 (p+1)(1 + 1/p) FMAs, plus mass term and two weight
    multiplies."""
    return 2.0 * 3.0 * (p + 1) * (1.0 + 1.0 / p) + 4.0


# ------------------------------------------------------------------ clocks
class Clocks:
    """nvidia-smi clock and throttle-reason samples every 50 ms (kept in memory)."""

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        """Start sampling; returns once the first sample has arrived."""
        self.window = None
        self.lines = []
        try:
            q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            first = self.proc.stdout.readline()      # blocks until nvidia-smi has sampled once
            if first:
                self.lines.append(first)
            else:
                self.proc = None
        except Exception:
            self.proc = None

    def mark(self, t0, t1):
        """Host wall-clock interval of the timed region."""
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        self.lines.extend((out or "").splitlines())
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((t, float(parts[1]), float(parts[2]),
                             [nm for nm, v in zip(names, parts[5:9]) if v.lower().startswith("active")]))
            except ValueError:
                continue
        inside = [r for r in rows if self.window and self.window[0] - 0.05 <= r[0] <= self.window[1] + 0.05]
        use = inside or rows
        if not use:
            return None
        return {"sm_mhz": statistics.median(r[1] for r in use), "sm_max_mhz": use[-1][2],
                "reasons": sorted({nm for r in use for nm in r[3]}), "samples": len(use),
                "window": "timed region" if inside else "whole run"}


# ------------------------------------------------------------------ workload
class Workload:
    """Right-hand sides b_k = A x*(t_k) + noise built on the device (untimed)."""

    def __init__(self, sg, torch, nsteps, device, cfg=None):
        self.torch = torch
        c = CFG if cfg is None else cfg
        self.cfg = c
        self.op = sg.Op(*c["E"], c["p"], c["lam"], "f64")
        cx, cy, cz = self.op.coords_1d()
        modes = Modes(c["seed"], c["modes"], c["kmax"])
        sx, sy, sz = modes.factors(cx, cy, cz)
        n = self.op.n
        phi = torch.empty((c["modes"], n), dtype=torch.float64, device=device)
        aphi = torch.empty_like(phi)
        for j in range(c["modes"]):
            f = np.einsum('k,y,x->kyx', sz[j], sy[j], sx[j]).reshape(-1)
            phi[j].copy_(torch.from_numpy(f))
            self.op.apply(phi[j], out=aphi[j])
        self.rhs = []
        for k in range(1, nsteps + 1):
            amp = torch.from_numpy(modes.amplitudes(c["dt"] * k)).to(device)
            b = amp @ aphi
            if c["noise"] > 0:
                rms = torch.sqrt(torch.mean(b * b))
                eta = torch.from_numpy(noise(c["seed"], k, n)).to(device)
                mask = (b != 0).to(torch.float64)
                b = b + c["noise"] * rms * eta * mask
            self.rhs.append(b.contiguous())
        del phi, aphi
        torch.cuda.synchronize()


MIXED_PROF_STEPS = 2


def run_mixed(sg, torch, wl, s, m, steps, warmup, flush, mode, delta=None):
    """Mixed-precision steps (32^3 Poisson shape): mode 'ir' = FP32 history + FP32 PCG in restarted FP64
    refinement, 'ru' = the same with FP64 residual replacement instead of
    restarts, 'f64' = FP64 history + FP64 PCG.  Returns per-step ms and iterations.
    The timed steps run the solves as in production (iterations in graph
    launches); MIXED_PROF_STEPS further steps, untimed, time every kernel
    launch with CUDA events for the per-kernel breakdown."""
    c = wl.cfg
    tol = c["tol"]
    n = wl.op.n
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    its, outs, rels = [], [], []
    if mode in ("ir", "ru"):
        ms = sg.MixedSolver(*c["E"], c["p"], c["lam"])
        g = sg.Guess(n, s, "extrap", m=m, dtype="f32")
        x64 = ms.op64.zeros()
    else:
        op = wl.op
        g = sg.Guess(n, s, "extrap", m=m, dtype="f64")
    for k in range(warmup + steps + MIXED_PROF_STEPS):
        timed = warmup <= k < warmup + steps
        if k == warmup + steps:
            torch.cuda.synchronize()
            sg.profile_reset()
            sg.profile_enable(True)
        if timed:
            ev[k - warmup][0].record()
        b = wl.rhs[k]
        slot = g.next_slot()
        g.form(None, slot)
        if mode in ("ir", "ru"):
            sg.convert(slot, x64)
            o, i, r = ms.solve(b, x64, tol, inner_tol=delta, method="restart" if mode == "ir" else "replace")
            sg.convert(x64, slot)
            if timed:
                outs.append(o)
        else:
            i, _ = op.pcg(b, slot, tol, true_residual=False)
        g.update(slot)
        if timed:
            ev[k - warmup][1].record()
            its.append(i)
            rels.append(r if mode in ("ir", "ru") else op.residual_norm(b, slot))   # FP64 check, untimed
        flush()
    torch.cuda.synchronize()
    sg.profile_enable(False)
    ex_ms, ex_cnt = sg.profile_read(sg.PROF_EXTRAP)
    kern = {}
    for name, kid in (("pcg_apply", sg.PROF_PCG_APPLY), ("pcg_update", sg.PROF_PCG_UPDATE)):
        t, cnt = sg.profile_read(kid)
        kern[name] = {"avg_us": 1e3 * t / max(cnt, 1), "launches_per_step": cnt / MIXED_PROF_STEPS,
                      "ms_per_step": t / MIXED_PROF_STEPS}
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    return {"ms": sum(ms_steps) / len(ms_steps), "iters": sum(its) / len(its), "max_relres": max(rels),
            "outer": (sum(outs) / len(outs)) if outs else None,
            "extrap_avg_ms": ex_ms / max(ex_cnt, 1), "kernels": kern}


def run_adjoint(sg, torch, device, steps):
    """One loss + gradient evaluation of the time-stepped Helmholtz sequence
    (16^3 p = 7, lambda = 1e5, 64 forcing modes, EXTRAP(2,6) guesses in both
    directions, checkpoints every 10 steps) through ``SequenceLoss``: forward
    solves, then backward (segment recomputation + reverse-time adjoint solves).
    Targets come from a forward run with theta*; the gradient is taken at
    theta = theta*/2.  Timed with CUDA events after one untimed evaluation."""
    from paper_2009_10863_gb300.adjoint import HeatSequence, SequenceLoss
    c = CONFIGS["heat_16x16x16_p7"]
    E, p, lam, dt, nparam = c["E"], c["p"], c["lam"], c["dt"], c["modes"]
    seq = HeatSequence(*E, p, tol=c["tol"], s=c["s"], m=2, checkpoint=10)
    op = seq.op(lam)
    cx, cy, cz = op.coords_1d()
    inner = [(v > 0) & (v < 1) for v in (cx, cy, cz)]
    idx = forcing_basis_indices(nparam)
    phi = torch.empty((nparam, op.n), dtype=torch.float64, device=device)
    for j, (a, b_, cc) in enumerate(idx):
        f = np.einsum('k,y,x->kyx', np.sin(np.pi * cc * cz) * inner[2], np.sin(np.pi * b_ * cy) * inner[1],
                      np.sin(np.pi * a * cx) * inner[0]).reshape(-1)
        phi[j].copy_(torch.from_numpy(f))
    theta_star, w = adjoint_parameters(5, nparam)
    C = torch.from_numpy(np.cos(np.outer(dt * np.arange(1, steps + 1), w))).to(device)
    Fstar = (C * torch.from_numpy(theta_star).to(device)) @ phi
    # targets: the forward solutions for theta*
    xs, x_prev = [], None
    g = sg.Guess(op.n, c["s"], "extrap", m=2)
    rhs = op.empty()
    for k in range(steps):
        sg.lib().sg_mass_rhs(op.h, float(lam), sg._ptr(x_prev) if x_prev is not None else None,
                             sg._ptr(Fstar[k]), sg._ptr(rhs), sg._stream())
        x = g.next_slot()
        g.form(rhs, x)
        op.pcg(rhs, x, c["tol"], true_residual=False)
        g.update(x)
        xs.append(x.clone())
        x_prev = xs[-1]
    Xs = torch.stack(xs)
    del xs, Fstar
    lam_t = torch.tensor(lam, dtype=torch.float64, device=device, requires_grad=True)
    res = {}
    for rep in range(2):
        theta = torch.from_numpy(0.5 * theta_star).to(device).requires_grad_(True)
        lam_t.grad = None
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        torch.cuda.synchronize()
        e0.record()
        L = SequenceLoss.apply((C * theta) @ phi, lam_t, Xs, seq)
        e1.record()
        L.backward()
        e2.record()
        torch.cuda.synchronize()
        if rep == 1:
            it = seq.last_iters
            res = {"steps": steps, "params": nparam + 1, "checkpoint_every": 10,
                   "forward_ms": e0.elapsed_time(e1), "backward_ms": e1.elapsed_time(e2),
                   "total_ms": e0.elapsed_time(e2),
                   "ms_per_solve": e0.elapsed_time(e2) / (3 * steps),
                   "cg_iters_per_solve": {"forward": sum(it["forward"]) / len(it["forward"]),
                                          "recompute": sum(it["recompute"]) / len(it["recompute"]),
                                          "adjoint": sum(it["adjoint"]) / len(it["adjoint"])},
                   "loss": float(L.detach()), "grad_norm_theta": float(theta.grad.norm()),
                   "dL_dlambda": float(lam_t.grad)}
    return res


def run_batched(sg, torch, device, steps, warmup, flush, mode, tune=True):
    """Four sequences (24^3 Poisson with QR(8); 20^3, 16^3, 12^3 Helmholtz with
    EXTRAP(3,8)), FP32 histories, FP32 PCG inside FP64 refinement.  mode
    'batched': one persistent launch per CG iteration for all four systems;
    'sequential': one mixed-precision solve per system after another."""
    cfgs = [dict(c, **BATCHED_COMMON) for c in BATCHED]
    wls = [Workload(sg, torch, warmup + steps, device, cfg=c) for c in cfgs]
    tol = BATCHED_COMMON["tol"]
    s = BATCHED_COMMON["s"]
    guesses, x64s, x32s, b32s = [], [], [], []
    for c, wl in zip(cfgs, wls):
        op32 = sg.Op(*c["E"], c["p"], c["lam"], "f32")
        g = sg.Guess(wl.op.n, s, c["method"], m=c["m"], eps_rel=1e-5, op=op32, dtype="f32")
        guesses.append((g, op32))
        x64s.append(torch.zeros(wl.op.n, dtype=torch.float64, device=device))
        x32s.append(torch.zeros(wl.op.n, dtype=torch.float32, device=device))
        b32s.append(torch.zeros(wl.op.n, dtype=torch.float32, device=device))
    tuned = None
    if mode == "batched":
        solver = sg.BatchSolver([(c["E"][0], c["E"][1], c["E"][2], c["lam"]) for c in cfgs])
        if tune:
            tuned = solver.tune()
    else:
        solvers = [sg.MixedSolver(*c["E"], c["p"], c["lam"]) for c in cfgs]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    inner_tot = [0] * len(cfgs)
    outer_tot = [0] * len(cfgs)
    launches = 0
    for k in range(warmup + steps):
        timed = k >= warmup
        if timed and k == warmup:
            torch.cuda.synchronize()
            launches = sg.launch_count()
        if timed:
            ev[k - warmup][0].record()
        bs = [wl.rhs[k] for wl in wls]
        for i, (g, op32) in enumerate(guesses):
            slot = g.next_slot()
            x0 = slot if slot is not None else x32s[i]
            if slot is None:
                sg.convert(bs[i], b32s[i])
            g.form(b32s[i] if slot is None else None, x0)
            sg.convert(x0, x64s[i])
        if mode == "batched":
            outer, inner, rel = solver.solve(bs, x64s, tol)
        else:
            outer, inner, rel = [], [], []
            for i, ms in enumerate(solvers):
                o, ii, r = ms.solve(bs[i], x64s[i], tol)
                outer.append(o); inner.append(ii); rel.append(r)
        for i, (g, op32) in enumerate(guesses):
            slot = g.next_slot()
            dst = slot if slot is not None else x32s[i]
            sg.convert(x64s[i], dst)
            g.update(dst)
        if timed:
            ev[k - warmup][1].record()
            for i in range(len(cfgs)):
                inner_tot[i] += inner[i]
                outer_tot[i] += outer[i]
            assert max(rel) <= tol * 1.0001
        flush()
    torch.cuda.synchronize()
    launches = sg.launch_count() - launches
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"ms_per_step": sum(ms) / len(ms),
            "inner_fp32_iters_per_step": [t / steps for t in inner_tot],
            "outer_steps_per_step": [t / steps for t in outer_tot],
            "library_launches_per_step": launches / steps,
            "tuned": {"zl": tuned[0], "ctas_per_sm": tuned[1], "ms_per_iter": tuned[2]} if tuned else None}


def run_method(sg, torch, wl, method, m, s, steps, warmup, flush, prof=False, clocks=None, e2e=False,
               criterion=0):
    """Run warmup + steps time steps; returns per-step ms, iterations, residuals.

    Without ``prof`` every solve is enqueued with ``Op.pcg_async`` (set-up
    kernels and one graph launch for the iterations) and its iteration count
    read after the step's end event.  With ``prof`` the library times every
    kernel launch with CUDA events, which needs the host-launched iterations
    of ``Op.pcg``; that pass gives the per-kernel durations of the roofline."""
    op = wl.op
    tol = CFG["tol"]
    g = sg.Guess(op.n, s, method, m=m, eps_rel=tol, op=op, dtype="f64")
    xbuf = op.zeros()
    ring = method in ("extrap", "last", "spextrap")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    iters, rels = [], []
    # e2e: b_k comes from pinned host memory and x_k goes back to it.  The
    # copies are double-buffered on two side streams: during step k's timed
    # interval the input of step k+1 is copied in and the result of step k-1
    # copied out, and the step's end event waits for both, so every interval
    # holds one host-to-device and one device-to-host vector copy (b_k itself
    # arrived during step k-1, x_k leaves during step k+1)
    overlap = e2e and method in ("extrap", "last", "zero", "spextrap")   # guess without b_k
    if e2e:
        host_b = [wl.rhs[k].cpu().pin_memory() for k in range(warmup + steps)]
        host_x = [torch.empty(op.n, dtype=torch.float64).pin_memory() for _ in range(2)]
        dev_b = [op.empty(), op.empty()]
        h2d_stream, d2h_stream = torch.cuda.Stream(), torch.cuda.Stream()
        h2d_done = [torch.cuda.Event(), torch.cuda.Event()]
        d2h_done = torch.cuda.Event()
        solved = [torch.cuda.Event(), torch.cuda.Event()]
        dev_b[0].copy_(host_b[0], non_blocking=True)
        h2d_done[0].record()
        prev_x = None
    launches = 0
    if clocks:
        clocks.start()
    t_timed = None
    for k in range(warmup + steps):
        timed = k >= warmup
        if timed and k == warmup:
            torch.cuda.synchronize()
            if prof:
                sg.profile_reset()
                sg.profile_enable(True)
            t_timed = time.time()
            launches = sg.launch_count()
        if timed:
            ev[k - warmup][0].record()
        main = torch.cuda.current_stream()
        if e2e:
            if k + 1 < warmup + steps:           # b_{k+1} into the buffer step k-1 used
                if k >= 1:
                    h2d_stream.wait_event(solved[(k - 1) % 2])
                with torch.cuda.stream(h2d_stream):
                    dev_b[(k + 1) % 2].copy_(host_b[k + 1], non_blocking=True)
                h2d_done[(k + 1) % 2].record(h2d_stream)
            if prev_x is not None:               # x_{k-1} out
                d2h_stream.wait_event(solved[(k - 1) % 2])
                with torch.cuda.stream(d2h_stream):
                    host_x[(k - 1) % 2].copy_(prev_x, non_blocking=True)
                d2h_done.record(d2h_stream)
            b = dev_b[k % 2]
        else:
            b = wl.rhs[k]
        x = g.next_slot() if ring else xbuf
        if method == "zero":
            x.zero_()
        if e2e and not overlap:
            main.wait_event(h2d_done[k % 2])
        g.form(b, x)
        if e2e and overlap:                      # the extrapolation does not read b_k
            main.wait_event(h2d_done[k % 2])
        if prof:
            it, _ = op.pcg(b, x, tol, criterion=criterion, true_residual=False)
        else:
            op.pcg_async(b, x, tol, criterion=criterion)
        g.update(x)
        if e2e:
            solved[k % 2].record(main)
            if k + 1 < warmup + steps:
                main.wait_event(h2d_done[(k + 1) % 2])
            if prev_x is not None:
                main.wait_event(d2h_done)
            prev_x = x
        if not prof:
            if timed:
                ev[k - warmup][1].record()
            it = op.pcg_result()          # waits for the step; outside the timed interval
        if timed:
            if prof:
                ev[k - warmup][1].record()
            iters.append(it)
            # verification, outside the timed interval: the true residual of x_k
            # (still held by x after the update)
            rels.append(op.residual_norm(b, x))
        flush()
    if e2e:                                      # the last result out (after the timed steps)
        host_x[(warmup + steps - 1) % 2].copy_(prev_x)
    torch.cuda.synchronize()
    launches = sg.launch_count() - launches
    if prof:
        sg.profile_enable(False)
    if clocks:
        clocks.mark(t_timed, time.time())
    clk = clocks.stop() if clocks else None
    ms = [a.elapsed_time(b) for a, b in ev]
    return {"ms": ms, "iters": iters, "rels": rels, "launches": launches, "clocks": clk}


# ------------------------------------------------------------------ oracle timing
def bench_config(n=None):
    """The ``config`` object of the JSON line, identical for both arms."""
    E = CFG["E"]
    nodes = n if n is not None else (CFG["p"] * E[0] + 1) * (CFG["p"] * E[1] + 1) * (CFG["p"] * E[2] + 1)
    return {"workload": workload_name(), "elements": list(E), "p": CFG["p"], "nodes": nodes,
            "lambda": CFG["lam"], "s": CFG["s"], "method": "EXTRAP(2,8)", "tol": CFG["tol"],
            "criterion": "||r|| <= tol ||b||", "l2": "flushed (512 MiB write) between timed steps",
            "parallelism": "replicas (one independent sequence per GPU)"}


def oracle_steps(steps, warmup):
    """Complete time steps of the FP64 CPU oracle on the headline workload, each
    timed with the host clock: the EXTRAP(2,8) guess from the last 8 solutions,
    the Jacobi-PCG solve from it to ||r|| <= 1e-10 ||b||, and the history update.
    The history starts from the exact solutions x*(t_1..t_8), so every step has
    a full ring; right-hand sides (with the bench's noise) are built untimed.
    Returns per-step milliseconds and CG iterations of the timed steps."""
    from oracle.sem import SemOperator
    from oracle.pcg import pcg
    from oracle import extrap as ex
    c = CFG
    op = SemOperator(*c["E"], c["p"], c["lam"])
    cx, cy, cz = op.coords_1d()
    modes = Modes(c["seed"], c["modes"], c["kmax"])
    s, m = c["s"], HEADLINE[1]
    hist = [modes.field(cx, cy, cz, c["dt"] * k) * op.interior for k in range(1, s + 1)]
    diag = op.diagonal()
    beta = ex.lsq_coeffs(s, m)
    ms, its = [], []
    for k in range(s + 1, s + 1 + warmup + steps):
        b = op.apply(modes.field(cx, cy, cz, c["dt"] * k) * op.interior)
        b = b + c["noise"] * np.sqrt(np.mean(b * b)) * noise(c["seed"], k, op.n) * (b != 0)
        t0 = time.perf_counter()
        x0 = ex.extrap_guess(hist, beta)
        x, it, _, _ = pcg(op.apply, diag, b, x0, c["tol"], interior=op.interior)
        hist.append(x)
        hist.pop(0)
        t1 = time.perf_counter()
        if k >= s + 1 + warmup:
            ms.append(1e3 * (t1 - t0))
            its.append(it)
    return ms, its


def oracle_threads():
    """Threads the oracle's numpy/BLAS calls may use (the bench pins them to 1)."""
    return int(os.environ.get("OMP_NUM_THREADS", "1"))


def run_reference(args, rank):
    if rank != 0:
        return
    t0 = time.perf_counter()
    ms, its = oracle_steps(args.steps, args.warmup)
    value = sum(ms) / len(ms)
    sample = ("FP64 numpy oracle, %d thread(s) of %d host cores: %d untimed + %d timed complete steps of the "
              "16^3 p=7 Helmholtz sequence (EXTRAP(2,8) guess, Jacobi-PCG to 1e-10, history update), "
              "host clock per step" % (oracle_threads(), os.cpu_count() or 0, args.warmup, args.steps))
    line = {"metric": METRIC, "value": value, "unit": "ms/step", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": bench_config(),
            "cg_iters_per_step": sum(its) / len(its),
            "cpu_baseline": {"value": value, "unit": "ms/step", "cores": oracle_threads(),
                             "host_cores": os.cpu_count(), "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ profiling drivers
def profile_ops(sg, torch, args):
    """Every kernel of the library on one mesh: the operator ``--reps`` times,
    a few PCG iterations (host-launched, each a separate launch), an
    EXTRAP(2,s) guess and QR(s) history updates until d = s."""
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
    sg.profile_enable(True)
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


def profile_steps(sg, torch, steps):
    """Headline time steps with every library launch timed by CUDA events, so
    the PCG iterations are host launches that a profiler lists one by one."""
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


def profile_batched(sg, torch):
    """One solve of the four batched systems from zero (right-hand sides A x for
    random x), persistent launches replayed as plain graph kernel nodes; no tuning."""
    meshes = [(c["E"][0], c["E"][1], c["E"][2], c["lam"]) for c in BATCHED]
    solver = sg.BatchSolver(meshes)
    gen = torch.Generator(device="cuda").manual_seed(0)
    bs, xs = [], []
    for c in BATCHED:
        op = sg.Op(*c["E"], c["p"], c["lam"], "f64")
        bs.append(op.apply(torch.randn(op.n, dtype=torch.float64, device="cuda", generator=gen)))
        xs.append(op.zeros())
    sg.profile_enable(True)
    outer, inner, rel = solver.solve(bs, xs, 1e-10)
    torch.cuda.synchronize()
    sg.profile_enable(False)
    print("batched: outer", outer, "inner", inner, "relres %.2e" % max(rel))


# ------------------------------------------------------------------ main
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the ZERO/LAST/QR comparison runs")
    ap.add_argument("--no-mixed", action="store_true", help="skip the FP32+IR vs FP64 comparison")
    ap.add_argument("--mixed-steps", type=int, default=8)
    ap.add_argument("--mixed-warmup", type=int, default=10)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-sequences comparison")
    ap.add_argument("--batched-steps", type=int, default=8)
    ap.add_argument("--batched-warmup", type=int, default=8)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint (loss + gradient) timing")
    ap.add_argument("--adjoint-steps", type=int, default=50)
    ap.add_argument("--profile-driver", choices=["ops", "steps", "batched"], default=None,
                    help="run a short profiling driver instead of the benchmark")
    ap.add_argument("--elements", type=int, default=16, help="profile-driver ops: elements per axis")
    ap.add_argument("--p", type=int, default=7, help="profile-driver ops: degree")
    ap.add_argument("--lam", type=float, default=1e5, help="profile-driver ops: lambda")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32"], help="profile-driver ops: dtype")
    ap.add_argument("--reps", type=int, default=3, help="profile-driver ops: operator applications")
    ap.add_argument("--pcg-iters", type=int, default=6, help="profile-driver ops: PCG iterations")
    ap.add_argument("--s", type=int, default=8, help="profile-driver ops: history size")
    ap.add_argument("--prof-steps", type=int, default=14, help="profile-driver steps: time steps")
    args = ap.parse_args()
    if args.profile_driver:
        import torch
        import paper_2009_10863_gb300 as sg
        from paper_2009_10863_gb300 import build as sgbuild
        sgbuild.build()
        torch.cuda.set_device(0)
        if args.profile_driver == "ops":
            profile_ops(sg, torch, args)
        elif args.profile_driver == "steps":
            profile_steps(sg, torch, args.prof_steps)
        else:
            profile_batched(sg, torch)
        return
    if args.warmup < 3:
        raise SystemExit("warmup must be >= 3")

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch
    import paper_2009_10863_gb300 as sg
    from paper_2009_10863_gb300 import build as sgbuild
    if rank == 0 or world == 1:
        sgbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist.barrier()
        sgbuild.build()
    sg.lib()
    device = torch.device("cuda", local)
    nsteps = args.warmup + args.steps
    wl = Workload(sg, torch, nsteps + MIXED_PROF_STEPS, device)
    flush_buf = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=device)

    def flush():
        flush_buf.zero_()

    s = CFG["s"]
    n = wl.op.n
    # headline: EXTRAP(2, 8), timed K steps bracketed by barrier + synchronize
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    t_wall = time.perf_counter()
    head = run_method(sg, torch, wl, HEADLINE[0], HEADLINE[1], s, args.steps, args.warmup, flush,
                      clocks=clocks)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    ms_step = aggregate_max(sum(head["ms"]) / len(head["ms"]), dist, device)

    # kernel timing: the same K steps again with every library launch timed by
    # CUDA events on its stream (host-launched iterations)
    kt = run_method(sg, torch, wl, HEADLINE[0], HEADLINE[1], s, args.steps, args.warmup, flush, prof=True)
    prof = {}
    for name, kid in (("sem", sg.PROF_SEM), ("pcg_apply", sg.PROF_PCG_APPLY), ("pcg_update", sg.PROF_PCG_UPDATE),
                      ("extrap", sg.PROF_EXTRAP)):
        tot, cnt = sg.profile_read(kid)
        prof[name] = (tot, cnt)
    p = CFG["p"]
    # A solve launches its iterations in chunks sized from the previous solve;
    # launches after convergence return at once.  Their time is charged to the
    # iterations that did the work: per-iteration duration = all launch time of
    # the kernel / iterations.
    kt_iters = sum(kt["iters"])
    tot_apply, cnt_apply = prof["pcg_apply"]
    avg_apply_ms = tot_apply / max(kt_iters, 1)
    nel = CFG["E"][0] * CFG["E"][1] * CFG["E"][2]
    flop_alg = sem_flops_per_element(p) * nel          # the roofline's algorithmic unit
    flop_apply = sem_flops_per_node(p) * n             # the even-odd kernel's own operator count
    achieved = flop_alg / (avg_apply_ms * 1e-3) / 1e12
    achieved_own = flop_apply / (avg_apply_ms * 1e-3) / 1e12
    hbm_gbs, hbm_src = peaks()
    ex_tot, ex_cnt = prof["extrap"]
    ex_bytes = (s + 1) * 8 * n
    ex_gbs = ex_bytes / (ex_tot / max(ex_cnt, 1) * 1e-3) / 1e9 if ex_cnt else None
    up_tot, up_cnt = prof["pcg_update"]
    up_gbs = 8 * 8 * n / (up_tot / max(kt_iters, 1) * 1e-3) / 1e9 if up_cnt else None

    # all-step mean: the same sequence from an empty history (a fresh guess on
    # the warmed operator and workspace), every step timed -- the start-up steps
    # with fewer than s past solutions included
    allst = run_method(sg, torch, wl, HEADLINE[0], HEADLINE[1], s, args.warmup + args.steps, 0, flush)

    out = {"metric": METRIC, "value": ms_step, "unit": "ms/step", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": bench_config(n),
           "cg_iters_per_step": sum(head["iters"]) / len(head["iters"]),
           "max_relres": max(head["rels"]),
           "timed_wall_s": t_wall}
    out["all_steps"] = {"ms_per_step": sum(allst["ms"]) / len(allst["ms"]),
                        "cg_iters_per_step": sum(allst["iters"]) / len(allst["iters"]),
                        "steps": len(allst["ms"]), "max_relres": max(allst["rels"]),
                        "note": "the same sequence from an empty history, every step timed (start-up steps "
                                "with fewer than s = 8 past solutions included); value and ms_per_step are "
                                "the steps with a full history"}

    out["roofline"] = {"kernel": "pcg_apply (SEM operator + fused p update, FP64)", "bound": "alu",
                       "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                       "frac": achieved / FP64_PEAK_TFLOPS, "traffic": PCG_APPLY_TRAFFIC,
                       "flops_per_launch": flop_alg,
                       "flop_count": "algorithmic: 6 (p+1)^4 + 8 (p+1)^3 = %d flop per element x %d elements "
                                     "(dense element-line products)" % (sem_flops_per_element(p), nel),
                       "achieved_own_count": achieved_own, "frac_own_count": achieved_own / FP64_PEAK_TFLOPS,
                       "flops_per_launch_own_count": flop_apply,
                       "own_count": "the even-odd operator's arithmetic: %.1f flop per node x %d nodes "
                                    "(stricter: the fraction of the FP64 peak the kernel's own operations reach)"
                                    % (sem_flops_per_node(p), n),
                       "traffic_note": "ncu dram__bytes_read+write per launch (cold reads of z, p, q; "
                                       "p and q writes retire to L2), profiles/kernels_helmholtz16_p7_fp64.md",
                       "algorithmic_bytes_per_launch": 5 * 8 * n,
                       "avg_launch_ms": avg_apply_ms, "launches": cnt_apply,
                       "iterations": kt_iters,
                       "timing": "kernel-timing pass: the headline's K steps again, every operator and update "
                                 "launch bracketed by CUDA events on its stream; avg_launch_ms = total launch "
                                 "time / iterations (launches after convergence included)",
                       "kernel_pass_ms_per_step": sum(kt["ms"]) / len(kt["ms"]),
                       "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz "
                                      "(DFMA measured at 1.256 TFLOP/s, profiles/fp64_pipes_dfma_vs_mma.md)"}
    ex_avg = ex_tot / max(ex_cnt, 1) if ex_cnt else None
    up_avg = up_tot / max(kt_iters, 1) if up_cnt else None
    out["guess_kernels"] = {
        "extrap": {"GB_s": ex_gbs, "frac_of_hbm": ex_gbs / hbm_gbs if ex_gbs else None,
                   "bytes_per_launch": ex_bytes, "launches": ex_cnt,
                   "fp64_ops_per_node": s, "frac_of_fp64_peak": fp64_frac(s, n, ex_avg)},
        "pcg_update": {"GB_s": up_gbs, "frac_of_hbm": up_gbs / hbm_gbs if up_gbs else None,
                       "bytes_per_launch": 8 * 8 * n, "launches": up_cnt, "iterations": kt_iters,
                       "fp64_ops_per_node": 5, "frac_of_fp64_peak": fp64_frac(5, n, up_avg)},
        "hbm_peak_GB_s": hbm_gbs, "hbm_peak_source": hbm_src,
        "fp64_peak_Gops": FP64_PEAK_TFLOPS * 1e3 / 2,
        "fp64_roof": "FP64 operations (DFMA, DMUL, DADD: one each) per node of the kernel's arithmetic at "
                     "2 per clock per SM (152 SMs, 2.07 GHz)"}
    out["gpu_launches"] = head["launches"]
    if head["clocks"]:
        out["clocks"] = head["clocks"]

    # end to end through the public API with host buffers (pinned), copies timed
    e2e = run_method(sg, torch, wl, HEADLINE[0], HEADLINE[1], s, args.steps, args.warmup, flush, e2e=True)
    e2e_ms = aggregate_max(sum(e2e["ms"]) / len(e2e["ms"]), dist, device)
    out["e2e"] = {"value": e2e_ms, "unit": "ms/step", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n,
                  "copies": "pinned host b_k in, x_k out; double-buffered on two side streams: each timed "
                            "step waits for the copy-in of b_{k+1} and the copy-out of x_{k-1}"}

    # the other guess methods on the same sequence (not part of the headline)
    if not args.no_compare:
        comp = {}
        # ZERO, LAST, QR(8) (Algorithm 2), and the rows beyond the paper's main
        # comparison: naive extrapolation EXTRAP(7,8) (degree M-1, the paper's
        # unstable baseline), SPEXTRAP(2,8), CLASSIC(8) (Algorithm 1), ENERGY(8)
        # (the QR(8) window in the energy inner product)
        for label, name, m in (("zero", "zero", 0), ("last", "last", 0), ("qr", "qr", 0),
                               ("naive extrap(7,8)", "extrap", 7), ("spextrap(2,8)", "spextrap", 2),
                               ("classic(8)", "classic", 0), ("energy(8)", "energy", 0)):
            r = run_method(sg, torch, wl, name, m, s, args.steps, args.warmup, flush)
            comp[label] = {"ms_per_step": sum(r["ms"]) / len(r["ms"]),
                           "cg_iters_per_step": sum(r["iters"]) / len(r["iters"]),
                           "max_relres": max(r["rels"])}
        comp["extrap(2,8)"] = {"ms_per_step": ms_step, "cg_iters_per_step": out["cg_iters_per_step"]}
        out["methods"] = comp
        # projection kernels of QR(8) with a full history (d = M = 8): kernel-timing
        # pass as for the headline; algorithmic words per node: guess 2(d+1)
        # (b and d columns of B~ read; d columns of X~ read, x0 written), update
        # 7M+2 (upd1 with the Givens downdate 4M-1, upd2 M+1, upd3 2M+2)
        rq = run_method(sg, torch, wl, "qr", 0, s, args.steps, args.warmup, flush, prof=True)
        qk = {}
        # FP64 operations per node: dots and lincomb one per column; the update
        # (d = s: downdate of s - 1 rotations on B~ and X~ at 2 each, s - 1 CGS
        # dots and the norm; then 2 (s - 1) and 2 (s - 1) + 1)
        upd_ops = 4 * (s - 1) + (s - 1) + 1 + 2 * (s - 1) + 2 * (s - 1) + 1
        for label, kid, words, ops in (("proj_dots", sg.PROF_PROJ_DOTS, s + 1, s),
                                       ("proj_lincomb", sg.PROF_PROJ_LINCOMB, s + 1, s),
                                       ("proj_update", sg.PROF_PROJ_UPDATE, 7 * s + 2, upd_ops)):
            t, c = sg.profile_read(kid)
            avg = t / max(c, 1)
            gbs = words * 8 * n / (avg * 1e-3) / 1e9 if c else None
            qk[label] = {"avg_us": 1e3 * avg, "launch_groups": c, "bytes_per_group": words * 8 * n, "GB_s": gbs,
                         "frac_of_hbm": gbs / hbm_gbs if gbs else None, "fp64_ops_per_node": ops,
                         "frac_of_fp64_peak": fp64_frac(ops, n, avg if c else None)}
        out["guess_kernels"]["qr(8)"] = qk
        # the paper's two stopping rules (Eqs. StopCritINITRESID, StopCritRHS) against
        # the workload's ||r|| <= tol ||b||, same EXTRAP(2,8) sequence
        crit = {}
        for label, code in (("||r|| < tol max(||r0||, 1)", sg.STOP_INITRESID),
                            ("||r|| < tol max(||b||, 1)", sg.STOP_RHS)):
            r = run_method(sg, torch, wl, HEADLINE[0], HEADLINE[1], s, args.steps, args.warmup, flush,
                           criterion=code)
            crit[label] = {"ms_per_step": sum(r["ms"]) / len(r["ms"]),
                           "cg_iters_per_step": sum(r["iters"]) / len(r["iters"]),
                           "max_relres": max(r["rels"])}
        out["stopping_rules"] = crit

    if not args.no_mixed:
        # the headline workload itself through FP32 PCG with FP64 residual
        # replacement and an FP32 EXTRAP(2,8) history: the same 1e-10 on the
        # FP64 residual, context beside the FP64 headline.  Replacement
        # threshold delta = 1e-4: on this mass-dominated Helmholtz system one
        # FP32 segment reaches 1e-10 (delta 0.1 / 1e-2 / 1e-3 / 1e-4 measured
        # 1.34 / 1.02 / 1.05 / 0.84 ms/step with 4 / 2 / 2 / 1 FP64 updates)
        r_h = run_mixed(sg, torch, wl, s, 2, args.steps, args.warmup, flush, "ru", delta=1e-4)
        out["mixed_precision_headline"] = {
            "workload": workload_name() + " solved by FP32 PCG with FP64 residual replacement "
                        "(delta 1e-4), FP32 history",
            "ms_per_step": r_h["ms"], "inner_fp32_iters_per_step": r_h["iters"],
            "fp64_updates_per_step": r_h["outer"], "max_relres_fp64": r_h["max_relres"],
            "speedup_vs_fp64_headline": ms_step / r_h["ms"], "kernels": r_h["kernels"]}
        c3 = CONFIGS["poisson_32x32x32_p7"]
        del wl
        torch.cuda.empty_cache()
        w3 = Workload(sg, torch, args.mixed_warmup + args.mixed_steps + MIXED_PROF_STEPS, device, cfg=c3)
        r_ir = run_mixed(sg, torch, w3, c3["s"], 2, args.mixed_steps, args.mixed_warmup, flush, "ir")
        r_ru = run_mixed(sg, torch, w3, c3["s"], 2, args.mixed_steps, args.mixed_warmup, flush, "ru")
        r_64 = run_mixed(sg, torch, w3, c3["s"], 2, args.mixed_steps, args.mixed_warmup, flush, "f64")
        n3 = w3.op.n
        ex32_gbs = (c3["s"] + 1) * 4 * n3 / (r_ir["extrap_avg_ms"] * 1e-3) / 1e9
        out["mixed_precision"] = {
            "workload": "poisson-32x32x32-p7 (%d nodes), EXTRAP(2,8), tol 1e-10 on the FP64 residual" % n3,
            "steps": args.mixed_steps, "warmup": args.mixed_warmup,
            "fp32_ir": {"ms_per_step": r_ir["ms"], "inner_fp32_iters_per_step": r_ir["iters"],
                        "outer_steps_per_step": r_ir["outer"], "max_relres_fp64": r_ir["max_relres"],
                        "kernels": r_ir["kernels"]},
            "fp32_replace": {"ms_per_step": r_ru["ms"], "inner_fp32_iters_per_step": r_ru["iters"],
                             "fp64_updates_per_step": r_ru["outer"], "max_relres_fp64": r_ru["max_relres"],
                             "kernels": r_ru["kernels"]},
            "fp64": {"ms_per_step": r_64["ms"], "cg_iters_per_step": r_64["iters"],
                     "max_relres": r_64["max_relres"], "kernels": r_64["kernels"]},
            "speedup_fp32_ir_vs_fp64": r_64["ms"] / r_ir["ms"],
            "speedup_fp32_replace_vs_fp64": r_64["ms"] / r_ru["ms"],
            "extrap_fp32": {"GB_s": ex32_gbs, "frac_of_hbm": ex32_gbs / hbm_gbs,
                            "bytes_per_launch": (c3["s"] + 1) * 4 * n3}}
        del w3

    if not args.no_batched:
        torch.cuda.empty_cache()
        rb = run_batched(sg, torch, device, args.batched_steps, args.batched_warmup, flush, "batched")
        rs = run_batched(sg, torch, device, args.batched_steps, args.batched_warmup, flush, "sequential")
        out["batched"] = {
            "workload": "4 sequences, p=7: 24^3 Poisson QR(8), 20^3/16^3/12^3 Helmholtz lam=1e3 EXTRAP(3,8); "
                        "FP32 history + FP32 PCG in FP64 refinement to 1e-10",
            "steps": args.batched_steps, "warmup": args.batched_warmup,
            "batched_persistent": rb, "sequential_solves": rs,
            "speedup_batched_vs_sequential": rs["ms_per_step"] / rb["ms_per_step"]}

    if not args.no_adjoint:
        torch.cuda.empty_cache()
        out["adjoint"] = dict(workload="time-stepped Helmholtz 16^3 p=7, lambda=1e5, 64 forcing modes, "
                                       "EXTRAP(2,6), 1e-10; loss + gradient in theta (64) and lambda",
                              **run_adjoint(sg, torch, device, args.adjoint_steps))

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cms, cits = oracle_steps(CPU_BASELINE_STEPS, 1)
        out["cpu_baseline"] = {"value": sum(cms) / len(cms), "unit": "ms/step", "cores": oracle_threads(),
                               "host_cores": os.cpu_count(), "kind": "oracle",
                               "cg_iters_per_step": sum(cits) / len(cits),
                               "sample": "FP64 numpy oracle, %d thread(s) of %d host cores: 1 untimed + %d timed "
                                         "complete steps of the same sequence (EXTRAP(2,8) guess, Jacobi-PCG to "
                                         "1e-10, history update), host clock per step"
                                         % (oracle_threads(), os.cpu_count() or 0, CPU_BASELINE_STEPS)}
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
