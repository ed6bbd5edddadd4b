#!/usr/bin/env python3
"""Benchmark: Jacobian solves per second at a relative residual of 1e-10 on the
3D unit cube with 128^3 nodes (2,097,152 complex unknowns), field mu = 1 along
(1,1,1)/sqrt(3), psi == 1 (the state of the paper's Sec. 4 experiments), random
complex-normal right-hand side (seed 5).

One step = one R_1-preconditioned MINRES solve of J(psi) x = b from x = 0 until
the FP64 true residual ||b - J x||_D / ||b||_D <= 1e-10.  The preconditioner is
set up once for psi before the timed region (setup-exclusive solves/s).  Two
mixed-precision forms are measured (GL_MIXED: FP32 inner MINRES solves with FP32
Jacobian applies and V-cycles inside FP64 defect correction; GL_MIXED_PRECOND:
FP32 V-cycle inside FP64 MINRES); the faster one is then measured again with
the learned warm start (a 4-layer, 64-channel graph network trained on the GPU
on eight other right-hand sides of the same state; every solve pays its
inference and the zero-guess fallback check), and the faster of the two is the
headline.  The FP64 form is timed beside it.  The AMG hierarchy stops coarsening at 4096 nodes
(--max-coarse), where the dense FP64 inverse takes over.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Multi-GPU (one rank per GPU via torch.distributed.run): every rank solves its
own copy of the workload (replicas, no exchange); value = solves of all ranks
divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gl_inputs as gi  # noqa: E402

METRIC = "Jacobian solves/s @1e-10 rel-res (3D 128^3): mixed+learned vs FP64 GPU; %HBM"
UNIT = "solves/s"


def max_over_ranks(x, dist=None, device="cpu"):
    """The largest of every rank's x (the slowest rank's time); x itself on one rank."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, seconds):
    """Units of work all ranks processed (replicas: the same on each) per second of
    the slowest rank."""
    return world * units_per_rank / seconds


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--N", type=int, default=128, help="nodes per side of the cube")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--max-coarse", type=int, default=4096, help="coarsest-level size bound of the AMG hierarchy")
    ap.add_argument("--no-learned", action="store_true", help="skip training and timing the learned warm start")
    ap.add_argument("--ws-steps", type=int, default=200, help="Adam steps of warm-start training")
    ap.add_argument("--no-extra", action="store_true", help="skip the batch64 and 2D workload measurements")
    ap.add_argument("--sweep-sync", type=int, default=0, choices=[0, 1, 2],
                    help="coarse-sweep synchronisation (options.sweep_sync; 0 = timed at setup)")
    ap.add_argument("--workload", default="cube", choices=["cube", "cube-continuation"],
                    help="cube: the headline solve; cube-continuation: the field-strength continuation with the "
                         "learned warm start (its own JSON line)")
    ap.add_argument("--cont-steps", type=int, default=64, help="continuation steps (cube-continuation)")
    ap.add_argument("--host-loop", action="store_true",
                    help="MINRES iterations replayed by the host instead of the device-side graph loop "
                         "(options.device_loop = 0; for launch lists of profilers that skip conditional graphs)")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi every 50 ms.  The
    sampler is started, and its first sample awaited, before the region; the
    summary keeps the samples that arrived inside the region (all of them if none
    did)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.rows = []
        self.proc = None
        self.t0 = self.t1 = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            deadline = time.perf_counter() + 5.0
            while not self.rows and time.perf_counter() < deadline and self.proc.poll() is None:
                time.sleep(0.01)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.perf_counter(), [x.strip() for x in line.split(",")]))

    def start(self):
        self.t0 = time.perf_counter()

    def stop(self):
        self.t1 = time.perf_counter()
        time.sleep(0.06)  # the sample taken at the end of the region

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        inside = [r for t, r in self.rows
                  if self.t0 is not None and self.t1 is not None and self.t0 <= t <= self.t1 + 0.06]
        rows = inside or [r for _, r in self.rows]
        sm = [float(r[1]) for r in rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, name in enumerate(names):
                if len(r) > 5 + k and "Active" in r[5 + k] and "Not" not in r[5 + k]:
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_in_region": len(inside),
                "interval_ms": 50}


def recorded_traffic(cls):
    """DRAM bytes per launch of kernel class `cls` from the committed ncu capture,
    or None when there is none or the kernel's sources changed since it."""
    import hashlib

    p = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        recs = json.load(f)
    rec = recs.get(cls)
    if not rec:
        return None
    h = hashlib.sha256()
    for s in rec["sources"]:
        with open(os.path.join(ROOT, s), "rb") as f:
            h.update(f.read())
    return rec["dram_bytes_per_launch"] if h.hexdigest() == rec["sources_sha256"] else None


def workload(N):
    dim, _, mu, bh = gi.WORKLOADS["cube128"]
    n = N ** 3
    return dim, mu, bh, n


def _oracle_solve_timed(oracle, N, b, max_coarse, threads):
    """One full FP64 R_1-MINRES solve of the oracle on `threads` host threads (0: all
    processors); returns (seconds of the solve, solution, info, threads used, setup s)."""
    dim, mu, bh, n = workload(N)
    used = oracle.set_threads(threads)
    t0 = time.perf_counter()
    m = oracle.Mesh(dim, N, mu, bh)
    psi = np.ones(n, complex)
    P = oracle.Precond(m, psi, max_coarse=max_coarse)
    t1 = time.perf_counter()
    x, info = P.minres(b)
    t2 = time.perf_counter()
    return t2 - t1, x, info, used, t1 - t0


def cpu_baseline(N, b, x_gpu, max_coarse):
    """The oracle's FP64 R_1-MINRES solve of the same system on the host (setup
    excluded, like the GPU number), on one thread and on all host processors (the
    oracle shares out only its row loops, so both give the same bits); also the
    GPU solution's error against it."""
    import oracle

    t1, x, info, _, setup1 = _oracle_solve_timed(oracle, N, b, max_coarse, 1)
    tall, xall, infoall, cores, _ = _oracle_solve_timed(oracle, N, b, max_coarse, 0)
    oracle.set_threads(1)
    err = float(np.linalg.norm(x_gpu - x) / np.linalg.norm(x)) if x_gpu is not None else None
    return {
        "value": 1.0 / tall, "unit": UNIT, "cores": cores, "kind": "oracle",
        "sample": f"one full FP64 R_1-MINRES solve of the {N}^3 cube system on {cores} host threads "
                  f"({infoall.iters} iterations, true relres {infoall.true_relres:.2e}; mesh+setup untimed)",
        "iters": infoall.iters, "same_bits_as_one_thread": bool(np.array_equal(x, xall)),
        "one_thread": {"value": 1.0 / t1, "unit": UNIT, "cores": 1, "seconds": t1,
                       "mesh_setup_s": setup1},
    }, err


def run_reference(args):
    """The oracle timed on the host processors, in the bench's metric and config:
    every step is one whole FP64 R_1-MINRES solve of the workload's system (setup
    once, untimed), on all host processors (the oracle's row loops; its sums stay
    serial, so the result does not depend on the thread count)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    N = args.N
    dim, mu, bh, n = workload(N)
    cores = oracle.set_threads(0)
    m = oracle.Mesh(dim, N, mu, bh)
    psi = np.ones(n, complex)
    b = gi.complex_normal(n, 5)
    P = oracle.Precond(m, psi, max_coarse=args.max_coarse)
    secs, iters = [], []
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _, info = P.minres(b)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            secs.append(dt)
            iters.append(info.iters)
    total = float(np.sum(secs))
    value = args.steps / total
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"cube{N}^3 mu=1 bhat=(1,1,1)/sqrt3 psi=1 b=CN(0,1) seed 5",
                   "n": n, "tol": 1e-10, "l2": "inputs larger than L2"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"one whole FP64 R_1-MINRES solve per step ({iters[0] if iters else 0} "
                                   f"iterations) on {cores} host threads, setup untimed"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def alu_roofline(pr, nsolves, peak_gbs, peak_gflops, kernel, peak_kind):
    """Roofline of a kernel class bounded by min(HBM, arithmetic pipe): the bound is
    whichever of bytes / HBM peak and flops / FMA peak takes longer."""
    sec = pr["ms"] / 1e3
    t_hbm = pr["bytes"] / (peak_gbs * 1e9)
    t_alu = pr["flops"] / (peak_gflops * 1e9) if pr["flops"] > 0 else 0.0
    alu = t_alu > t_hbm
    r = {
        "bound": "alu" if alu else "hbm", "kernel": kernel,
        "unit": "GFLOP/s" if alu else "GB/s",
        "achieved": (pr["flops"] / sec / 1e9) if alu else (pr["bytes"] / sec / 1e9),
        "peak": peak_gflops if alu else peak_gbs,
        "frac": max(t_hbm, t_alu) / sec, "frac_hbm": t_hbm / sec, "frac_alu": t_alu / sec,
        "alg_bytes_per_launch": pr["bytes"] / pr["timed"], "alg_flops_per_launch": pr["flops"] / pr["timed"],
        "launches_timed": pr["timed"], "avg_launch_us": 1e3 * pr["ms"] / pr["timed"],
        "ms_per_solve": pr["ms"] / nsolves, "peak_kind": peak_kind,
    }
    return r


def run_batch64(gl, torch, dev, steps=3):
    """The batched-continuation workload: 64 2D squares, N_s log-uniform in [32, 512]
    (seed 6), mu_s = 2 (s + 1) / 64, psi_s = 1 + 0.1 disk noise (seed 7 + s), b_s
    complex normal (seed 100 + s); one CUDA-graph launch per run."""
    sizes = gi.batch_sizes(64, seed=6)
    meshes, psis, bs = [], [], []
    for s_, N in enumerate(sizes):
        n = N * N
        meshes.append(gl.gl_mesh_create(2, N, 2.0 * (s_ + 1) / 64))
        psis.append(torch.from_numpy(gi.psi_noisy_one(n, 7 + s_)).to(dev))
        bs.append(torch.from_numpy(gi.complex_normal(n, 100 + s_)).to(dev))
    xs = [torch.zeros_like(b) for b in bs]
    out = {"instances": len(sizes), "unknowns": int(sum(N * N for N in sizes)),
           "sizes": f"{min(sizes)}^2..{max(sizes)}^2"}
    try:
        for name, prec in (("fp64", gl.GL_FP64), ("fp32_vcycle", gl.GL_MIXED_PRECOND)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            B = gl.gl_batch_create(meshes, psis, gl.options(precision=prec))
            torch.cuda.synchronize()
            setup = time.perf_counter() - t0
            try:
                st, infos = gl.gl_batch_run(B, bs, xs)
                ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                ev0.record()
                for _ in range(steps):
                    for x in xs:
                        x.zero_()
                    st, infos = gl.gl_batch_run(B, bs, xs)
                ev1.record()
                torch.cuda.synchronize()
                ms = ev0.elapsed_time(ev1) / steps
                out[name] = {"solves_per_s": 1e3 * len(sizes) / ms, "ms_per_batch": ms, "setup_s": setup,
                             "status": st, "all_converged": all(i.converged for i in infos),
                             "max_true_relres": max(i.true_relres for i in infos),
                             "iters_max": max(i.iters for i in infos)}
            finally:
                gl.gl_batch_destroy(B)
    finally:
        for m in meshes:
            gl.gl_mesh_destroy(m)
    return out


def run_square(gl, torch, dev, name, steps=5):
    """Solves/s on the 2D workloads: square64 (psi uniform in the unit disk, seed 1,
    b ~ CN(0,1) seed 1, FP64) and square1024 (the Newton system of the state from
    Newton at mu = 2 started at psi = 1, plus 0.1 disk noise seed 2; FP64 and the
    FP32 V-cycle)."""
    dim, N, mu, bh = gi.WORKLOADS[name]
    n = N * N
    m = gl.gl_mesh_create(dim, N, mu, bh)
    out = {"n": n}
    try:
        if name == "square64":
            psi = torch.from_numpy(gi.disk(n, 1)).to(dev)
            b = torch.from_numpy(gi.complex_normal(n, 1)).to(dev)
            forms = (("fp64", gl.GL_FP64),)
        else:
            psi = torch.ones(n, dtype=torch.complex128, device=dev)
            for _ in range(5):
                r = torch.zeros_like(psi)
                gl.gl_residual(m, psi, r)
                if float(torch.sqrt(torch.sum(torch.abs(r) ** 2))) / (N - 1) <= 1e-7:
                    break
                gl.gl_newton_step(m, psi, gl.options(max_coarse=512, tol=1e-8))
            psi += torch.from_numpy(0.1 * gi.disk(n, 2)).to(dev)
            r = torch.zeros_like(psi)
            gl.gl_residual(m, psi, r)
            b = -r
            forms = (("fp64", gl.GL_FP64), ("fp32_vcycle", gl.GL_MIXED_PRECOND))
        x = torch.zeros_like(psi)
        for fname, prec in forms:
            o = gl.options(precision=prec, max_coarse=512)
            P = gl.gl_precond_setup(m, psi, o)
            try:
                infos = []
                for rep in range(1 + steps):
                    if rep == 1:
                        torch.cuda.synchronize()
                        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                        ev0.record()
                    x.zero_()
                    st, info = gl.gl_jacobian_solve(m, psi, P, b, x, o)
                    infos.append(info)
                ev1.record()
                torch.cuda.synchronize()
                ms = ev0.elapsed_time(ev1) / steps
                out[fname] = {"solves_per_s": 1e3 / ms, "iters": infos[-1].iters,
                              "true_relres": max(i.true_relres for i in infos), "status": st}
            finally:
                gl.gl_precond_destroy(P)
    finally:
        gl.gl_mesh_destroy(m)
    return out


def run_continuation(args):
    """The continuation workload on the N^3 cube (the 256^3 configuration at --N 256):
    natural-parameter continuation in mu over [0, 1.5] in --cont-steps steps from
    psi = 1 (Sec. 4), Newton at every mu (J d = -GL(psi), FP32 V-cycle inside FP64
    MINRES, corrections to 1e-8, while ||GL||_R > 1e-7; the preconditioner of each
    Newton step takes over the previous one's symbolic part).  Every Newton system
    has a hint: the correction of the same Newton step at the previous mu.  The warm
    start is trained on the systems of the first half; on the second half every
    system is solved from zero, from the hint's minimal-residual multiple alone
    (no network: one FP64 Jacobian apply and three inner products) and from hint +
    network, with the same preconditioner; iterations and device time (the guess,
    inference and fallback check included) are summed."""
    import torch

    import paper_1204_5125_gb300 as gl

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    N, steps = args.N, args.cont_steps
    dim, _, _, bh = gi.WORKLOADS["cube128"]
    n = N ** 3
    mus = [1.5 * s / (steps - 1) for s in range(steps)]
    mesh = gl.gl_mesh_create(dim, N, mus[0], bh)
    psi = torch.ones(n, dtype=torch.complex128, device=dev)
    o = gl.options(precision=gl.GL_MIXED_PRECOND, max_coarse=args.max_coarse, tol=1e-8)
    t_start = time.perf_counter()
    train, held, prev, like = dict(psi=[], b=[], hint=[]), [], [], None
    newton_total = 0
    try:
        for s_, mu in enumerate(mus):
            if s_ > 0:
                gl.gl_mesh_set_mu(mesh, mu)
            cur = []
            for it in range(8):
                r = torch.zeros_like(psi)
                gl.gl_residual(mesh, psi, r)
                if float(torch.sqrt(torch.sum(torch.abs(r) ** 2))) / (N - 1) ** 1.5 <= 1e-7:
                    break
                b = -r
                P = gl.gl_precond_setup_like(mesh, psi, like, o) if like is not None else gl.gl_precond_setup(mesh, psi, o)
                if like is not None:
                    gl.gl_precond_destroy(like)
                like = P
                d = torch.zeros_like(psi)
                st, inf = gl.gl_jacobian_solve(mesh, psi, P, b, d, o)
                newton_total += 1
                hint = prev[it] if it < len(prev) else None
                if hint is not None:
                    if s_ < steps // 2:
                        train["psi"].append(psi.clone())
                        train["b"].append(b.clone())
                        train["hint"].append(hint)
                    else:
                        held.append((mu, psi.clone(), b.clone(), hint))
                cur.append(d.clone())
                psi = psi + d
            prev = cur
        gen_s = time.perf_counter() - t_start
        ws = gl.gl_warmstart_create(gi.warmstart_init(12))
        t0 = time.perf_counter()
        losses = gl.gl_warmstart_train(ws, [mesh] * len(train["b"]), train["psi"], train["b"], steps=args.ws_steps,
                                       batch=2, lr=2e-3, hints=train["hint"])
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        trained = gl.gl_warmstart_get_params(ws)
        forms = {"zero guess": None, "hint multiple": "hint", "hint + network": trained}
        res = {k: {"iters": 0, "ms": 0.0, "used": 0, "max_true_relres": 0.0} for k in forms}
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        for mu, p, b, hint in held:
            gl.gl_mesh_set_mu(mesh, mu)
            P = gl.gl_precond_setup_like(mesh, p, like, o)
            try:
                for k, params in forms.items():
                    oo = gl.options(precision=gl.GL_MIXED_PRECOND, max_coarse=args.max_coarse, tol=1e-8)
                    if params is not None:
                        oo.warmstart_hint = hint.data_ptr()
                    if params is not None and not isinstance(params, str):
                        gl.gl_warmstart_set_params(ws, params)
                        oo.warmstart = ws.value
                    x = torch.zeros_like(b)
                    ev0.record()
                    st, inf = gl.gl_jacobian_solve(mesh, p, P, b, x, oo)
                    ev1.record()
                    torch.cuda.synchronize()
                    res[k]["iters"] += inf.iters
                    res[k]["ms"] += ev0.elapsed_time(ev1)
                    res[k]["used"] += inf.warmstart_used
                    res[k]["max_true_relres"] = max(res[k]["max_true_relres"], inf.true_relres)
            finally:
                gl.gl_precond_destroy(P)
        gl.gl_warmstart_destroy(ws)
    finally:
        if like is not None:
            gl.gl_precond_destroy(like)
        gl.gl_mesh_destroy(mesh)
    z = res["zero guess"]
    line = {
        "metric": "MINRES iterations and ms on held-out continuation Newton systems: zero guess vs learned warm start",
        "workload": f"cube{N}^3 continuation mu in [0, 1.5], {steps} steps, bhat=(1,1,1)/sqrt3, Newton corrections "
                    f"to 1e-8, GL_MIXED_PRECOND",
        "newton_systems": newton_total, "training_systems": len(train["b"]), "held_out_systems": len(held),
        "generation_s": gen_s, "train_steps": args.ws_steps, "train_s": train_s,
        "train_loss_first": float(np.mean(losses[:10])), "train_loss_last": float(np.mean(losses[-10:])),
        "forms": res,
        "iterations_saved": {k: z["iters"] - v["iters"] for k, v in res.items()},
        "ms_saved": {k: z["ms"] - v["ms"] for k, v in res.items()},
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "cube-continuation":
        run_continuation(args)
        return
    import torch

    import paper_1204_5125_gb300 as gl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()

    N = args.N
    dim, mu, bh, n = workload(N)
    b_host = gi.complex_normal(n, 5)
    psi = torch.ones(n, dtype=torch.complex128, device=dev)
    b = torch.from_numpy(b_host).to(dev)
    x = torch.zeros_like(b)

    t0 = time.perf_counter()
    mesh = gl.gl_mesh_create(dim, N, mu, bh)
    t1 = time.perf_counter()
    dl = 0 if args.host_loop else 1
    opts_mixed = gl.options(precision=gl.GL_MIXED, max_coarse=args.max_coarse, sweep_sync=args.sweep_sync,
                            device_loop=dl)
    opts_fp64 = gl.options(precision=gl.GL_FP64, max_coarse=args.max_coarse, sweep_sync=args.sweep_sync,
                           device_loop=dl)
    prec = gl.gl_precond_setup(mesh, psi, opts_mixed)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    nlev = gl.gl_precond_levels(prec)
    levels = [gl.gl_precond_level_info(prec, l) for l in range(nlev)]

    def solve(opts):
        x.zero_()
        st, info = gl.gl_jacobian_solve(mesh, psi, prec, b, x, opts)
        if st != 0:
            raise RuntimeError(f"solve failed: status {st} {info.as_dict()}")
        return info

    def timed(opts, steps, warm, profile_class=None, count=False, clocks=None):
        """Times `steps` solves after `warm` untimed ones.  profile_class: time every
        launch of that kernel class with CUDA events; count: only count launches;
        clocks: the sampler whose window is the timed region."""
        profiling = bool(profile_class) or count
        if profiling:
            # before the warm-up, so graphs it makes the solver re-capture are captured there
            gl.gl_profile_begin(profile_class, 1 << 16 if profile_class else 0)
        for _ in range(warm):
            solve(opts)
        if profiling:
            gl.gl_profile_end()
            gl.gl_profile_begin(profile_class, 1 << 16 if profile_class else 0)
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if clocks:
            clocks.start()
        ev0.record(stream)
        infos = [solve(opts) for _ in range(steps)]
        ev1.record(stream)
        torch.cuda.synchronize()
        if clocks:
            clocks.stop()
        prof = gl.gl_profile_end() if profiling else None
        ms = max_over_ranks(ev0.elapsed_time(ev1), dist, dev)
        return ms, infos, prof

    # FP64 GPU form (context and the ratio the metric asks for)
    ms64, infos64, _ = timed(opts_fp64, max(1, args.steps // 2), max(1, args.warmup // 2))
    x64 = x.clone()
    # the two mixed forms: FP32 inner solves in FP64 defect correction, and an
    # FP32 V-cycle inside FP64 MINRES; the faster one is the headline
    forms = {"mixed_inner": opts_mixed, "mixed_precond": gl.options(precision=gl.GL_MIXED_PRECOND,
                                                                     max_coarse=args.max_coarse, device_loop=dl)}
    quick = {}
    for name, o in forms.items():
        q_ms, q_inf, _ = timed(o, 2, 1)
        quick[name] = {"solves_per_s": 2e3 / q_ms, "iters": [i.iters for i in q_inf],
                       "outer": [i.outer_iters for i in q_inf], "true_relres": max(i.true_relres for i in q_inf)}
    head = max(quick, key=lambda k: quick[k]["solves_per_s"])
    opts_head = forms[head]

    # learned warm start: trained on the GPU on eight other right-hand sides
    # (seeds 1000..1007) of the same state; the timed right-hand side is not among them
    learned = None
    wsh = None
    if not args.no_learned:
        wsh = gl.gl_warmstart_create(gi.warmstart_init(11))
        train_b = [torch.from_numpy(gi.complex_normal(n, 1000 + j)).to(dev) for j in range(8)]
        torch.cuda.synchronize()
        tt0 = time.perf_counter()
        losses = gl.gl_warmstart_train(wsh, [mesh] * 8, [psi] * 8, train_b, steps=args.ws_steps, batch=2, lr=2e-3)
        torch.cuda.synchronize()
        train_s = time.perf_counter() - tt0
        del train_b
        # relative true residual of the guess for the timed right-hand side
        x0 = torch.zeros_like(b)
        gl.gl_warmstart_predict(wsh, mesh, psi, b, x0)
        vol = torch.zeros(n, dtype=torch.float64, device=dev)
        gl.gl_mesh_info(mesh, vol)
        jx = torch.zeros_like(b)
        gl.gl_jacobian_apply(mesh, psi, x0, jx)
        guess_rel = float(torch.sqrt(torch.sum(vol * torch.abs(b - jx) ** 2) / torch.sum(vol * torch.abs(b) ** 2)))
        del x0, jx, vol
        opts_learned = gl.options(precision=opts_head.precision, max_coarse=args.max_coarse, device_loop=dl)
        opts_learned.warmstart = wsh.value
        q_ms, q_inf, _ = timed(opts_learned, 2, 1)
        wsf_ms, _, wsf_prof = timed(opts_learned, 2, 1, profile_class="wsf")
        learned = {
            "train_steps": args.ws_steps, "train_batch": 2, "train_s": train_s,
            "train_loss_first": float(np.mean(losses[:10])), "train_loss_last": float(np.mean(losses[-10:])),
            "guess_relres": guess_rel, "warmstart_used": [i.warmstart_used for i in q_inf],
            "solves_per_s": 2e3 / q_ms, "iters": [i.iters for i in q_inf],
            "true_relres": max(i.true_relres for i in q_inf),
            "forward_layer_us": 1e3 * wsf_prof["ms"] / wsf_prof["timed"] if wsf_prof["timed"] else None,
            "forward_layer_gbs": (wsf_prof["bytes"] / (wsf_prof["ms"] / 1e3) / 1e9) if wsf_prof["ms"] > 0 else None,
        }
    use_learned = learned is not None and learned["solves_per_s"] > quick[head]["solves_per_s"]
    opts_final = opts_learned if use_learned else opts_head
    form = head + ("+learned" if use_learned else "")
    if learned is not None:
        learned["headline"] = use_learned

    # headline: the chosen form, with the dominant kernel timed live by CUDA events
    # launches are counted during the timed solves; nothing is timed per kernel
    with Clocks(dev.index if world == 1 else local) as clk:
        ms, infos, count = timed(opts_final, args.steps, args.warmup, count=True, clocks=clk)
    x_mixed = x.clone()
    err_mixed_vs_fp64 = float(torch.linalg.norm(x_mixed - x64) / torch.linalg.norm(x64))

    # end to end through the C ABI with host buffers: H2D of b, solve, D2H of x
    e2e = None
    if not args.no_e2e:
        b_pin = torch.from_numpy(b_host).pin_memory()
        x_pin = torch.empty_like(b_pin).pin_memory()
        for _ in range(1):
            b.copy_(b_pin, non_blocking=True)
            solve(opts_final)
            x_pin.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        te0 = time.perf_counter()
        for _ in range(args.steps):
            b.copy_(b_pin, non_blocking=True)
            solve(opts_final)
            x_pin.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        te = max_over_ranks(time.perf_counter() - te0, dist, dev)
        e2e = {"value": whole_job_rate(args.steps, world, te), "unit": UNIT, "h2d_bytes_per_step": 16 * n,
               "d2h_bytes_per_step": 16 * n}

    value = whole_job_rate(args.steps, world, ms / 1e3)
    value64 = whole_job_rate(len(infos64), world, ms64 / 1e3)
    peak, peak_kind = peaks()

    # setup-inclusive rates: a preconditioner built from scratch (aggregation,
    # colouring, Galerkin products, the dense coarsest inverse, the setup-time
    # kernel timing, the FP32 copies) or taking over an earlier one's symbolic part
    torch.cuda.synchronize()
    ts0 = time.perf_counter()
    prec_like = gl.gl_precond_setup_like(mesh, psi, prec, opts_mixed)
    torch.cuda.synchronize()
    like_s = time.perf_counter() - ts0
    gl.gl_precond_destroy(prec_like)
    setup_inclusive = {
        "from_scratch": {"setup_s": t2 - t1, "solves_per_s": 1.0 / (t2 - t1 + ms / 1e3 / args.steps)},
        "setup_like": {"setup_s": like_s, "solves_per_s": 1.0 / (like_s + ms / 1e3 / args.steps)},
    }

    # measured arithmetic peaks of this GPU (own FMA kernel, CUDA events) and the
    # latencies that bound a phase of the coarse sweeps (own probe kernels)
    fp64_gflops = gl.gl_measure_fma_peak(gl.GL_FP64)
    fp32_gflops = gl.gl_measure_fma_peak(gl.GL_MIXED)
    sync_lat = gl.gl_measure_sync_latency()

    # live per-class timing (CUDA events around every launch of the class, on the
    # launching stream): the finest-level sweep from the headline run, then the
    # coarse-level sweeps and the Jacobian in two short runs of the same form
    KERNELS = {
        "gs0": (("k_gs_lat2 (Gauss-Seidel colour sweep, finest level, FP32, tabulated lattice stencil, two "
                 "positions per thread)" if N % 4 == 0 else
                 "k_gs_lat (Gauss-Seidel colour sweep, finest level, FP32, tabulated lattice stencil)")
                if infos[-1].lattice_stencil else "k_gs (Gauss-Seidel colour sweep, finest level, FP32)"),
        "gs": "k_sgs_flags / k_sgs_coop / k_sgs_cluster (symmetric Gauss-Seidel step, coarse levels, FP32)",
        "jz": ("k_jz_latdf (double-FP32 Jacobian apply fused with the Lanczos dot; SM-pipe bound)"
               if infos[-1].df_jacobian else "k_jz (Jacobian apply fused with the Lanczos dot, FP64)"),
        "coarse": "k_dense_mv_df (double-FP32 dense coarsest product)",
    }
    profs = {}
    for cls in ("gs0", "gs", "jz", "coarse"):
        _, _, pr = timed(opts_final, 2, 1, profile_class=cls)
        profs[cls] = (pr, 2)
    prof = profs["gs0"][0]
    rooflines = {}
    for cls, (pr, nsolves) in profs.items():
        if not pr or not pr["timed"] or pr["ms"] <= 0:
            continue
        rooflines[cls] = {
            "bound": "hbm", "kernel": KERNELS[cls], "unit": "GB/s", "peak": peak,
            "achieved": pr["bytes"] / (pr["ms"] / 1e3) / 1e9,
            "frac": pr["bytes"] / (pr["ms"] / 1e3) / 1e9 / peak,
            "traffic": recorded_traffic(cls), "alg_bytes_per_launch": pr["bytes"] / pr["timed"],
            "launches_timed": pr["timed"], "avg_launch_us": 1e3 * pr["ms"] / pr["timed"],
            "ms_per_solve": pr["ms"] / nsolves, "peak_kind": f"{peak_kind} hbm_gbs (copy)",
        }
    # the coarse sweep is a chain of dependent phases: each waits for a hand-off
    # from the CTAs it reads (release store -> acquiring poll), gathers the
    # neighbours' x from L2, and publishes its own writes behind a GPU-scope fence;
    # its floor per phase is the sum of those three measured latencies
    sweep_levels = [lv for lv in levels[1:-1]]
    if "gs" in rooflines and sweep_levels:
        phases = sum(2 * lv["ncolors"] - 1 for lv in sweep_levels)  # per pre- or post-smoothing
        us_phase = rooflines["gs"]["avg_launch_us"] * len(sweep_levels) / phases
        floor_us = (sync_lat["handoff_ns"] + sync_lat["l2_load_ns"] + sync_lat["fence_ns"]) / 1e3
        rooflines["gs"]["latency"] = {
            "bound": "latency", "phases_per_launch": phases / len(sweep_levels), "us_per_phase": us_phase,
            "floor_us_per_phase": floor_us, "frac": floor_us / us_phase, **sync_lat,
            "how": "floor = median one-way CTA hand-off + dependent L2 load + store and GPU-scope fence, "
                   "measured by gl_measure_sync_latency"}
    # the double-FP32 Jacobian is bounded by the FP32 pipe: its min(HBM, ALU) roofline
    if "jz" in rooflines and profs["jz"][0]["flops"] > 0 and infos[-1].df_jacobian:
        rooflines["jz"]["alu"] = alu_roofline(profs["jz"][0], 2, peak, fp32_gflops,
                                              KERNELS["jz"], "measured FP32 FMA peak (own kernel)")
    # the FP64 form's classes against min(HBM, FP64 ALU)
    rooflines_fp64 = {}
    KERNELS64 = {"gs0": "k_gs (Gauss-Seidel colour sweep, finest level, FP64)",
                 "gs": "k_sgs_flags / k_sgs_coop (symmetric Gauss-Seidel step, coarse levels, FP64)",
                 "jz": "k_jz (Jacobian apply fused with the Lanczos dot, FP64)"}
    for cls in ("gs0", "gs", "jz"):
        _, _, pr = timed(opts_fp64, 2, 1, profile_class=cls)
        if pr and pr["timed"] and pr["ms"] > 0:
            rooflines_fp64[cls] = alu_roofline(pr, 2, peak, fp64_gflops, KERNELS64[cls],
                                               f"{peak_kind} hbm_gbs (copy) / measured FP64 FMA peak (own kernel)")
    dominant = max(rooflines, key=lambda k: rooflines[k]["ms_per_solve"]) if rooflines else None
    roofline = dict(rooflines[dominant]) if dominant else None
    if roofline:
        roofline["class"] = dominant

    extra = None
    if rank == 0 and world == 1 and not args.no_extra:
        extra = {"batch64": run_batch64(gl, torch, dev), "square64": run_square(gl, torch, dev, "square64"),
                 "square1024": run_square(gl, torch, dev, "square1024")}

    cpu = None
    err_vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu, err_vs_oracle = cpu_baseline(N, b_host, x_mixed.cpu().numpy(), args.max_coarse)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c64/f64", "data": "synthetic",
            "config": {"workload": f"cube{N}^3 mu=1 bhat=(1,1,1)/sqrt3 psi=1 b=CN(0,1) seed 5",
                       "n": n, "tol": 1e-10, "form": form, "max_coarse": args.max_coarse,
                       "l2": "inputs larger than L2 (operators ~0.5 GB)", "levels": [lv["n"] for lv in levels],
                       "colors": [lv["ncolors"] for lv in levels], "parallelism": f"replicas x{world}",
                       "coarse_sweeps": {"fp32": gl.gl_precond_level_sweep(prec, 1, gl.GL_MIXED_PRECOND),
                                         "fp64": gl.gl_precond_level_sweep(prec, 1, gl.GL_FP64)}
                       if nlev > 2 else None},
            "iters_mixed": [i.iters for i in infos], "outer_mixed": [i.outer_iters for i in infos],
            "mixed_forms": quick, "learned": learned, "warmstart_used": [i.warmstart_used for i in infos],
            "true_relres_mixed": max(i.true_relres for i in infos),
            "fp64_value": value64, "iters_fp64": [i.iters for i in infos64],
            "true_relres_fp64": max(i.true_relres for i in infos64),
            "mixed_over_fp64": value / value64, "err_mixed_vs_fp64_gpu": err_mixed_vs_fp64,
            "err_mixed_vs_fp64_oracle": err_vs_oracle,
            "setup_s": {"mesh": t1 - t0, "precond": t2 - t1}, "setup_inclusive": setup_inclusive,
            "peaks": {"hbm_gbs": peak, "hbm_kind": peak_kind, "fp64_gflops_measured": fp64_gflops,
                      "fp32_gflops_measured": fp32_gflops, "sync_latency_ns": sync_lat},
            "roofline": roofline, "rooflines": rooflines, "rooflines_fp64": rooflines_fp64,
            "workloads": extra, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": count["launches"] if count else None, "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if wsh is not None:
        gl.gl_warmstart_destroy(wsh)
    gl.gl_precond_destroy(prec)
    gl.gl_mesh_destroy(mesh)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
