"""Benchmark of the online stage: batched reduced Newton solves per second on one GB300.

A step is one pass of the whole hot path (theta, Jacobian contraction, FP64 residual, LU,
update, every Newton iteration to convergence, pressure recovery) over one batch of synthetic
queries resident in HBM. Default workload: the n = 50 parameter sweep (4096 queries,
Q_a = Q_c = 6, Q_f = 3, pressure with M = 30).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                    [--workload sweep_n50|dense_n300|...] [--impl ours|reference]

Prints one JSON line (rank 0). Under torchrun each rank solves its own batch (weak scaling, no
collective on the data path). --impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

PREC = {"fp64": 0, "mixed": 1}
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sweep_n50", choices=sorted(synth.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=sorted(PREC))
    ap.add_argument("--batch", type=int, default=None)
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-recon", action="store_true",
                    help="skip the pressure-reconstruction comparison (combined basis)")
    ap.add_argument("--serve", action="store_true",
                    help="serving mode: saturation throughput of the continuous-batching server "
                         "and p50/p99 submit-to-completion latency under Poisson arrivals")
    ap.add_argument("--serve-burst", type=int, default=2048)
    ap.add_argument("--serve-seconds", type=float, default=4.0)
    ap.add_argument("--large", action=argparse.BooleanOptionalAction, default=True,
                    help="also measure the largest configuration (dense_n300: n = 300, Q = 24, "
                         "16384 queries) in the same run and report it as its own block")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def rank_queries(wl, batch, rank, world):
    """This rank's share of the job: queries [rank * batch, (rank + 1) * batch) of one seeded
    draw of world * batch queries (independent problems; no exchange between ranks)."""
    qall = synth.make_queries(wl, batch=batch * world)
    sl = slice(rank * batch, (rank + 1) * batch)
    return synth.QuerySet(qall.mu[sl].copy(), qall.n[sl].copy())


def max_over_ranks(value, device):
    """The largest value over the ranks of the default process group (the job's time)."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def run_reference(args, wl, rank, world):
    """The FP64 CPU oracle timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl, batch=args.batch)
    o = oracle.Oracle.from_set(ops)
    threads = oracle.max_threads()
    # size the per-step sample so that the whole run stays within a few minutes
    probe = max(threads, 16)
    t0 = time.perf_counter()
    o.solve(q.mu[:probe], q.n[:probe], threads=threads)
    per_q = (time.perf_counter() - t0) / probe
    budget = 150.0 / max(1, args.steps + args.warmup)
    sample = int(max(threads, min(len(q.mu), budget / max(per_q, 1e-9))))
    for _ in range(args.warmup):
        o.solve(q.mu[:threads], q.n[:threads], threads=threads)
    times = []
    for s in range(args.steps):
        off = (s * sample) % len(q.mu)
        idx = (np.arange(sample) + off) % len(q.mu)
        t0 = time.perf_counter()
        o.solve(q.mu[idx], q.n[idx], threads=threads)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = args.steps * sample / total
    line = {
        "impl": "reference", "metric": "reduced Newton solves/s", "value": value,
        "unit": "solves/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n_max, "q_a": wl.q_a, "q_c": wl.q_c,
                   "q_f": wl.q_f, "m": wl.m, "batch_per_gpu": len(q.mu), "precision": "fp64",
                   "l2": "host caches (CPU oracle)", "parallelism": f"replicas x{world}",
                   "sample_per_step": sample},
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": threads, "kind": "oracle",
                         "sample": f"{sample} queries of the {wl.name} workload per step"},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(wl, ops, q, seconds, idx=None):
    """Oracle (as is) on the host cores on a bounded sample; also returns its results. With
    `idx` the sample is those queries; otherwise evenly spaced queries, as many as about
    `seconds` of oracle time allows."""
    import oracle
    o = oracle.Oracle.from_set(ops)
    threads = oracle.max_threads()
    if idx is not None:
        t0 = time.perf_counter()
        u, p, info = o.solve(q.mu[idx], q.n[idx], threads=threads)
        dt = time.perf_counter() - t0
        return {"value": len(idx) / dt, "unit": "solves/s", "cores": threads, "kind": "oracle",
                "sample": f"{len(idx)} queries of the {len(q.mu)}-query {wl.name} batch (the 4 "
                          f"corners of the parameter box and queries stratified over alpha and "
                          f"log Re; {dt:.1f} s on {threads} threads)"}, idx, u, p, info
    probe = max(threads, 8)
    idx = np.linspace(0, len(q.mu) - 1, probe).astype(int)
    t0 = time.perf_counter()
    u, p, info = o.solve(q.mu[idx], q.n[idx], threads=threads)
    dt = time.perf_counter() - t0
    per_q = dt / probe
    sample = int(min(len(q.mu), max(probe, seconds / max(per_q, 1e-9))))
    if sample > probe and dt < 0.5 * seconds:  # the probe was short: time a larger sample
        idx = np.unique(np.linspace(0, len(q.mu) - 1, sample).astype(int))
        t0 = time.perf_counter()
        u, p, info = o.solve(q.mu[idx], q.n[idx], threads=threads)
        dt = time.perf_counter() - t0
    return {"value": len(idx) / dt, "unit": "solves/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(idx)} evenly spaced queries of the {len(q.mu)}-query {wl.name} batch "
                      f"({dt:.1f} s on {threads} threads)"}, idx, u, p, info


def main():
    args = parse()
    rank, world, local = dist_env()
    wl = synth.WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl, rank, world)
        return
    if args.serve:
        run_serve(args, wl, rank, world, local)
        return
    import torch
    from paper_1807_11866_gb300 import _build, rb

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if rank == 0:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    rb.library()

    line = measure(args, wl, args.batch or wl.batch, args.steps, args.warmup, rank, world, local,
                   dev, recon=not args.no_recon, cpu_seconds=args.cpu_seconds)
    if args.large and wl.name != LARGEST and world == 1:
        # the largest configuration of the metric's range, measured in the same run (its own
        # steps and warm-up; the operators of the first workload are freed by then)
        big = synth.WORKLOADS[LARGEST]
        sub = measure(args, big, big.batch, LARGE_STEPS, LARGE_WARMUP, 0, 1, local, dev,
                      recon=False, cpu_seconds=args.cpu_seconds, parity_sample=True)
        keep = ("value", "unit", "ms_per_step", "steps", "warmup", "dtype", "config",
                "latency_ms", "iters", "status_ok", "e2e", "gpu_launches", "kernels", "clocks",
                "roofline", "rooflines", "autotune", "plain_fp64", "speedup_vs_plain_fp64",
                "cpu_baseline", "rel_err_vs_oracle")
        line[LARGEST] = {k: sub[k] for k in keep if k in sub}
    if args.large and wl.name != SMALLEST and world == 1:
        # the plain single query (latency): one query of the n = 20 set solved to 1e-12
        small = synth.WORKLOADS[SMALLEST]
        sub = measure(args, small, 1, 50, 5, 0, 1, local, dev, recon=False, cpu_seconds=2.0)
        line[SMALLEST] = {k: sub[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup",
                                              "config", "latency_ms", "iters", "status_ok", "e2e",
                                              "gpu_launches", "kernels", "plain_fp64",
                                              "speedup_vs_plain_fp64", "cpu_baseline",
                                              "rel_err_vs_oracle") if k in sub}
        line[SMALLEST]["latency_us"] = 1e3 * sub["ms_per_step"]
    if args.large and world == 1:
        line["offline"] = offline_block(args, local)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def offline_block(args, local, steps=3):
    """The offline stage (Sec. 3.2, 3.5, 3.6) on the synthetic high-fidelity model: a 128 x 128
    periodic grid with two velocity components (N_h = 32768), K = 128 snapshots, n = 50 modes,
    two affine viscous matrices and forcing vectors, two convection forms of 8 quadrature terms
    each. One reduction = POD + projections + both tensors through the public calls (host
    buffers, synchronous); kernel times from the library's events; the tensor's triple
    contraction against the FP64 peak; the oracle on the host cores for the POD, projections and
    the first tensor (the CPU baseline), which also checks the GPU's operators."""
    from paper_1807_11866_gb300 import rb
    from synth import hf
    m = hf.make_hf_model(G=128, K=128, R=60, decay=0.85, q_c=2)
    n = 50
    ctx = rb.Context(rb.RB_PREC_FP64, device=local)

    def reduction():
        lam, V = ctx.rb_offline_pod(m.S, m.Z, n)
        A = [ctx.rb_offline_project(V, M) for M in m.A]
        f = [ctx.rb_offline_project_vector(V, fq) for fq in m.f]
        C = [ctx.rb_offline_tensor(V, t) for t in m.terms]
        return lam, V, A, f, C

    reduction()  # warm-up
    ctx.rb_profile(True)
    t0 = time.perf_counter()
    for _ in range(steps):
        lam, V, A, f, C = reduction()
    wall = (time.perf_counter() - t0) / steps
    kprof = ctx.rb_profile_read()
    ctx.rb_profile(False)
    ctx.close()
    pts = [t[0].shape[0] for t in m.terms[0]]
    flop = float(sum(2.0 * n ** 3 * p for tq in m.terms for p in [t[0].shape[0] for t in tq]))
    ten_ms = kprof["k_offline_tensor"][0] / steps
    ach = flop / (ten_ms * 1e-3) / 1e12
    out = {
        "metric": "offline reductions/s (POD + projections + tensors)", "value": 1.0 / wall,
        "unit": "reductions/s", "ms_per_reduction": 1e3 * wall, "steps": steps, "warmup": 1,
        "config": {"grid": "128 x 128 periodic, 2 components", "N_h": m.N, "snapshots": 128,
                   "modes": n, "q_a": 2, "q_f": 2, "q_c": 2, "terms_per_form": len(pts),
                   "points": pts[0]},
        "kernels": {k: {"ms_per_reduction": v[0] / steps, "launches": v[1]}
                    for k, v in kprof.items() if v[1]},
        "roofline": {"bound": "alu", "kernel": "k_offline_tensor (triple contraction)",
                     "achieved": ach, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": ach / FP64_PEAK_TFLOPS, "traffic": None, "work": "algorithmic",
                     "peak_source": "FP64 FMA throughput of a probe kernel of this project"},
    }
    if not args.no_cpu:
        from oracle import offline
        t0 = time.perf_counter()
        lam_o, V_o = offline.pod(m.S, m.Z, n)
        A_o = [offline.project(V_o, M) for M in m.A]
        t1 = time.perf_counter()
        C_o = offline.tensor(V_o, m.terms[0])
        t2 = time.perf_counter()
        full = (t1 - t0) + len(m.terms) * (t2 - t1)  # every tensor costs as much as the first
        s = np.sign(np.einsum("jn,jn->j", V, (m.Z @ V_o.T).T))
        rel = lambda a, b: float(np.abs(a - b).max() / np.abs(b).max())
        out["cpu_baseline"] = {"value": 1.0 / full, "unit": "reductions/s",
                               "cores": os.cpu_count(), "kind": "oracle",
                               "sample": f"POD, both projections ({t1 - t0:.1f} s) and the first "
                                         f"of {len(m.terms)} tensors ({t2 - t1:.1f} s), the rate "
                                         f"counting the other tensors at the first one's time"}
        out["rel_err_vs_oracle"] = {
            "lambda": rel(lam[:n], lam_o[:n]),
            "A": max(rel(Ag, Ao * np.outer(s, s)) for Ag, Ao in zip(A, A_o)),
            "C0": rel(C[0], C_o * np.einsum("j,l,k->jlk", s, s, s))}
    return out


LARGEST = "dense_n300"        # the largest configuration of the metric's range (n = 300)
SMALLEST = "single_n20"       # the plain single query (latency)
LARGE_STEPS, LARGE_WARMUP = 3, 3


def measure(args, wl, batch, steps, warmup, rank, world, local, dev, recon, cpu_seconds,
            parity_sample=False):
    """One workload: `warmup` untimed and `steps` timed solves of the batch resident in HBM,
    L2 flushed between steps; a kernel-by-kernel pass for the per-kernel breakdown and the
    roofline; the same solves end to end through rb_solve with pinned host buffers; the plain
    FP64 GPU path and the oracle on the host cores (rank 0, N = 1). Returns the JSON dict."""
    import torch
    from paper_1807_11866_gb300 import rb

    ops = synth.make_operators(wl)
    q = rank_queries(wl, batch, rank, world)
    if parity_sample:  # the corners of the parameter box take the last four queries
        q.mu[-4:] = synth.corner_queries(wl)
    prec = PREC[args.precision]
    tol_res = 1e-12 if wl.manufactured else None  # the single query is solved to 1e-12
    ctx = rb.Context(precision=prec, device=local, theta_family=wl.theta_family, tol_res=tol_res)
    ctx.load_set(ops)
    m = ctx.m
    stream = torch.cuda.Stream(device=dev)
    d_mu = torch.from_numpy(q.mu).to(dev)
    d_n = torch.from_numpy(q.n).to(dev)
    d_u = torch.empty((batch, wl.n_max), dtype=torch.float64, device=dev)
    d_p = torch.empty((batch, max(m, 1)), dtype=torch.float64, device=dev) if m else None
    d_info = torch.empty((batch, 4), dtype=torch.float64, device=dev)  # 32 B per query
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def step(s):
        ctx.rb_solve_device(d_mu, batch, d_n, d_u, d_p, d_info, s.cuda_stream)

    with torch.cuda.stream(stream):
        for _ in range(warmup):
            step(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.zero_()  # write > L2 between timed steps
            starts[i].record(stream)
            step(stream)
            ends[i].record(stream)
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # per-kernel breakdown: the same steps again with the library's per-launch CUDA events on the
    # launching stream (these launch kernel by kernel instead of replaying the solve graph)
    ctx.rb_profile(True)
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.zero_()
            step(stream)
    torch.cuda.synchronize()
    kprof = ctx.rb_profile_read()
    issued = ctx.rb_profile_issued()
    ctx.rb_profile(False)
    t_dev = sum(step_ms) / 1e3
    if world > 1:
        t_dev = max_over_ranks(t_dev, dev)
    value = batch * world * steps / t_dev

    info = d_info.cpu().numpy().view(rb.INFO_DTYPE).reshape(batch)
    u_gpu = d_u.cpu().numpy()
    p_gpu = d_p.cpu().numpy() if d_p is not None else None
    # kernels of one step: those the profiled pass counted plus the graph's loop-condition kernel
    # (one per Newton iteration of the batch)
    launches_total = sum(v[1] for v in kprof.values()) + steps * int(info["iters"].max())

    # end-to-end through the public host-buffer API, pinned host memory
    h_mu = torch.from_numpy(q.mu).pin_memory()
    h_n = torch.from_numpy(q.n).pin_memory()
    h_u = torch.empty((batch, wl.n_max), dtype=torch.float64).pin_memory()
    h_p = torch.empty((batch, max(m, 1)), dtype=torch.float64).pin_memory() if m else None
    h_info = torch.empty((batch, 4), dtype=torch.float64).pin_memory()
    L = rb.library()
    e2e_t = []
    for i in range(warmup + steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = L.rb_solve(ctx.h, h_mu.data_ptr(), batch, h_n.data_ptr(), h_u.data_ptr(),
                        h_p.data_ptr() if h_p is not None else None, h_info.data_ptr())
        t1 = time.perf_counter()
        assert rc == 0, ctx.last_error()
        if i >= warmup:
            e2e_t.append(t1 - t0)
    e2e_val = batch * world * len(e2e_t) / sum(e2e_t)
    h2d = q.mu.nbytes + q.n.nbytes
    d2h = batch * wl.n_max * 8 + (batch * m * 8 if m else 0) + batch * 32

    # roofline of the dominant kernel, measured live with events on the launching stream
    chord = chord_queries(prec, wl, q, ctx.rb_tuning())
    roof, roofs, kernels = kernel_rooflines(prec, wl, q, info, kprof, steps, chord, issued)

    line = {
        "metric": "reduced Newton solves/s", "value": value, "unit": "solves/s",
        "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": 1e3 * t_dev / steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16+f32+f64" if prec == 1 else "f64",
        "data": "synthetic",
        "config": {"workload": wl.name, "n": wl.n_max, "q_a": wl.q_a, "q_c": wl.q_c,
                   "q_f": wl.q_f, "m": m, "c_storage": wl.c_dtype, "batch_per_gpu": batch,
                   "precision": args.precision,
                   "l2": "flushed between timed steps (512 MiB write)",
                   "parallelism": f"replicas x{world}"},
        "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
        "iters": {"mean": float(info["iters"].mean()), "max": int(info["iters"].max())},
        "status_ok": int((info["status"] == 0).sum()),
        "e2e": {"value": e2e_val, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches_total),
        "kernels": kernels,
        "clocks": clk,
        "wall_s": wall,
    }
    line["roofline"] = roof
    line["rooflines"] = roofs
    line["autotune"] = ctx.rb_tuning()
    if rank == 0 and m and recon:
        line["pressure_reconstruction"] = pressure_reconstruction(
            rb, ctx, wl, batch, d_u, d_n, p_gpu, kprof, stream, flush, args, steps, warmup)
    ctx.close()
    del d_mu, d_n, d_u, d_p, d_info
    if rank == 0 and not args.no_plain and prec != 0:
        line["plain_fp64"] = plain_fp64(rb, ops, q, batch, dev, flush, steps, tol_res)
        line["speedup_vs_plain_fp64"] = value / line["plain_fp64"]["value"]
    del flush
    torch.cuda.empty_cache()
    if rank == 0 and world == 1 and not args.no_cpu:  # the CPU baseline at N = 1 only
        if parity_sample:  # 4 corners and 12 queries stratified over the parameter box
            idx = np.concatenate([synth.stratified_indices(wl, q.mu[:-4], cells=(3, 4)),
                                  np.arange(batch - 4, batch)])
            cb, idx, u_ref, p_ref, inf_ref = cpu_baseline(wl, ops, q, cpu_seconds, idx=idx)
        else:
            cb, idx, u_ref, p_ref, inf_ref = cpu_baseline(wl, ops, q, cpu_seconds)
        line["cpu_baseline"] = cb
        err = np.linalg.norm(u_gpu[idx] - u_ref, axis=1) / np.linalg.norm(u_ref, axis=1)
        line["rel_err_vs_oracle"] = {"u_max": float(err.max()), "u_mean": float(err.mean()),
                                     "queries": int(len(idx)),
                                     "sample": "corners + stratified over alpha, log Re" if parity_sample
                                     else "evenly spaced over the batch"}
        sizes = q.n[idx]
        if len(np.unique(sizes)) > 1:  # per reduced size (nested truncations)
            line["rel_err_vs_oracle"]["u_max_per_n"] = {
                int(v): float(err[sizes == v].max()) for v in np.unique(sizes)}
        if p_gpu is not None and p_ref is not None:
            perr = np.linalg.norm(p_gpu[idx] - p_ref, axis=1) / np.linalg.norm(p_ref, axis=1)
            line["rel_err_vs_oracle"]["p_max"] = float(perr.max())
    return line


FP64_PEAK_TFLOPS = 1.196  # FP64 FMA throughput measured on GB300 (152 SMs at 2070 MHz)
# FP32 FMA peak from the unit counts and the clock: 152 SMs x 128 FP32 lanes x 2 FLOP x 2.07 GHz
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the kernels as they
# stand, from ncu captures of this bench command on the n = 50 sweep (4096 queries) and on the
# n = 300 dense regime; a kernel changed since its capture has no entry.
NCU_TRAFFIC = {
    # DRAM read + write bytes per launch of each timed kernel kind, averaged as the bench counts
    # its launches (the residual GEMM: full product and increment; the assembly: rungs 0-3 with
    # the gated refresh launch; the elimination: three factorisations and a chord solve), from
    # one ncu capture of the same bench command. Workloads without a capture of the current
    # kernels report null.
    "sweep_n50": {
        "k_tc_gemm<sliced>": 16.14e6,
        "k_tc_gemm<plain>": 7.46e6,
        "k_tc_gemm<sliced,pressure>": 20.73e6,
        "k_newton_system": 113.9e6,
        "k_lu_mixed": 42.54e6,
        "k_prep": 21.20e6,
    },
}


def chord_queries(prec, wl, q, tuning):
    """Queries whose Newton iterations from the fourth on were chord steps: every query of the
    mixed path (each elimination kernel keeps its factors), unless RB_CHORD=0."""
    on = prec != 0 and os.environ.get("RB_CHORD", "") != "0"
    return np.full(len(q.n), on, bool)


def kernel_rooflines(prec, wl, q, info, kprof, steps, chord, issued=None):
    """Roofline of every timed kernel kind, and of the one with the largest device time.

    `achieved` counts the method's ALGORITHMIC work only (the multiply-adds of the contraction
    the kernel stands for, per active query-iteration of size n, padding excluded), so `frac`
    says how close the kernel comes to the time that work alone would take at the peak:
      fused FP64 Newton: 2 (Q_c n^3 + Q_a n^2) (Jacobian) + 2 Q_c n^3 (residual)
        + 2 n^3 / 3 + 2 n^2 (LU and solves) FLOP per iteration (FP64 ALU);
      Jacobian GEMM: 2 Q_c n^3 FLOP per new Jacobian (the iterations after the first, up to the
        third for queries on chord steps) (tensor);
      sliced residual GEMM: 2 Q_c n^3 FLOP per FP64-accurate residual (from the third iteration
        on) (tensor);
      sliced pressure GEMM: 2 Q_c n^2 m FLOP per query (tensor; where the library folds
        As(mu) u into it, large Q_a, its 2 Q_a n m FLOP are left out: a lower bound);
      elimination: 2 n^3 / 3 + 2 n^2 FLOP in FP32 per factorisation, 2 n^2 per chord solve (ALU);
      system assembly: 8 n^2 (A(mu)) + 4 n^2 (J^c, iterations with a new Jacobian after the
        first) bytes read and 4 n (n + 1) bytes written; a chord step reads A(mu) and writes the
        right-hand side, 8 n^2 + 4 n (HBM);
      per-query preparation: 8 n^2 bytes of A(mu) written, once per query (HBM).
    The tensor kernels ISSUE more products than that: the Jacobian GEMM 3 split-BF16 products
    (hi hi, hi lo, lo hi) and the sliced GEMMs up to P = S (S + 1) / 2 digit-pair products for an
    FP64-accurate result (fewer for the chord steps' increments), over padded tiles;
    `issued_tflops` / `issued_frac` report that rate (how busy the tensor pipe is), separately
    from `frac`, from the FLOPs of the MMAs the kernels executed, counted on the device
    (`issued`: kernel -> FLOPs over the profiled steps)."""
    peaks, kind = measured_peaks()
    n = q.n.astype(np.float64)
    it = info["iters"].astype(np.float64)
    full = np.where(chord, np.minimum(it, 3), it)   # iterations that factor a new Jacobian
    chs = it - full                                 # chord steps
    jac = np.maximum(full - 1, 0)                   # Jacobian contractions
    res = np.maximum(it - 2, 0)                     # FP64-accurate (sliced) residuals
    tot_ms = sum(v[0] for v in kprof.values()) or 1.0
    kernels = {k: {"ms_per_step": v[0] / steps, "launches_per_step": v[1] / steps,
                   "share": v[0] / tot_ms} for k, v in kprof.items() if v[1]}
    bf16 = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    hbm = peaks.get("hbm_gbs")
    bf16_src = f"bf16 sustained, {kind} (MEASURED_PEAKS.json)"
    hbm_src = f"HBM copy, {kind} (MEASURED_PEAKS.json)"
    work = {  # kernel -> (bound, algorithmic units per step, tensor kernel, peak, unit, src)
        "k_newton_fp64": ("alu", float(np.sum(it * (2 * (2 * wl.q_c * n ** 3 + wl.q_a * n ** 2)
                                                     + 2 * n ** 3 / 3 + 2 * n ** 2))), None,
                          FP64_PEAK_TFLOPS, "TFLOP/s",
                          "FP64 FMA throughput of a probe kernel of this project on GB300 (152 SMs, "
                          "2070 MHz); not a MEASURED_PEAKS.json figure"),
        "k_tc_gemm<plain>": ("tensor", float(np.sum(jac * 2.0 * wl.q_c * n ** 3)), True,
                             bf16, "TFLOP/s", bf16_src),
        "k_tc_gemm<sliced>": ("tensor", float(np.sum(res * 2.0 * wl.q_c * n ** 3)), True,
                              bf16, "TFLOP/s", bf16_src),
        "k_tc_gemm<sliced,pressure>": ("tensor", float(np.sum(2.0 * (wl.m or 0) * wl.q_c * n ** 2)),
                                       True, bf16, "TFLOP/s", bf16_src),
        "k_lu_mixed": ("alu", float(np.sum(full * (2 * n ** 3 / 3 + 2 * n ** 2) + chs * 2 * n ** 2)),
                       None, FP32_PEAK_TFLOPS, "TFLOP/s",
                       "FP32 FMA peak from unit counts and clock (152 x 128 x 2 x 2.07 GHz)"),
        "k_newton_system": ("hbm", float(np.sum(full * (8 * n ** 2 + 4 * n * (n + 1)) + jac * 4 * n ** 2
                                                + chs * (8 * n ** 2 + 4 * n))), None,
                            hbm, "GB/s", hbm_src),
        "k_prep": ("hbm", float(np.sum(8 * n ** 2)), None, hbm, "GB/s", hbm_src),
    }
    rl = {}
    for k, (ms, launches) in kprof.items():
        if not launches or k not in work:
            continue
        bound, units, tensor, peak, unit, src = work[k]
        scale = 1e12 if unit == "TFLOP/s" else 1e9
        ach = steps * units / (ms * 1e-3) / scale
        traffic = NCU_TRAFFIC.get(wl.name, {}).get(k)
        rl[k] = {"bound": bound, "kernel": k, "achieved": ach, "peak": peak, "unit": unit,
                 "frac": ach / peak, "traffic": traffic, "peak_source": src,
                 "work": "algorithmic", "launches": launches}
        flops = (issued or {}).get(k, 0.0)
        if tensor and flops > 0:
            # the MMAs the launches executed (digit or split products, padding tiles), counted
            # on the device over the same profiled steps
            rl[k]["issued_tflops"] = flops / (ms * 1e-3) / 1e12
            rl[k]["issued_frac"] = rl[k]["issued_tflops"] / peak
            rl[k]["issued_per_algorithmic"] = flops / (steps * units) if units else None
    dom = max(kprof, key=lambda k: kprof[k][0])
    return rl.get(dom), rl, kernels


def run_serve(args, wl, rank, world, local):
    """Serving: the server takes queries one by one through the public C API (rb_serve_submit /
    rb_serve_poll, host buffers), each of its own size n. (1) Saturation: a burst of
    --serve-burst queries, throughput = queries / time to the last completion. (2) Load points at
    25%, 50% and 80% of saturation: Poisson arrivals for --serve-seconds, with the server's own
    submit-to-completion p50 / p99. Every rank serves its own stream (replicas); rank 0 prints
    the sum of the ranks' saturation rates and its own latencies."""
    import torch
    from paper_1807_11866_gb300 import _build, rb
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        dist.barrier()
    ops = synth.make_operators(wl)
    q = synth.make_queries(wl, batch=wl.batch)
    ctx = rb.Context(precision=PREC[args.precision], device=local, theta_family=wl.theta_family)
    ctx.load_set(ops)
    B = len(q.mu)

    def point(rate, count, seed):
        ctx.rb_serve_start()
        g = np.random.default_rng(seed)
        pending = []
        t0 = time.perf_counter()
        nxt = t0
        for i in range(count):
            if rate:
                nxt += g.exponential(1.0 / rate)
                while True:
                    d = nxt - time.perf_counter()
                    if d <= 0:
                        break
                    time.sleep(min(d, 1e-3))
            pending.append(ctx.rb_serve_submit(q.mu[i % B], n=int(q.n[i % B])))
        status = []
        while pending:
            left = []
            for t in pending:
                r = ctx.rb_serve_poll(t)
                if r is None:
                    left.append(t)
                else:
                    status.append(int(r[2]["status"]))
            pending = left
            if pending:
                time.sleep(2e-4)
        t1 = time.perf_counter()
        p50, p99, sps = ctx.rb_serve_stats()
        ctx.rb_serve_stop(True)
        return {"offered_per_s": rate, "queries": count, "served_per_s": count / (t1 - t0),
                "server_solves_per_s": sps, "p50_ms": 1e3 * p50, "p99_ms": 1e3 * p99,
                "ok": int(sum(1 for s in status if s == 0))}

    # warm-up: one burst of the measured size (layouts, slot tables, each size bucket's scratch
    # grown to its working size), as a server in steady state has seen
    point(None, args.serve_burst, 1)
    clocks = ClockSampler(local)
    clocks.start()
    ctx.rb_profile(True)  # counts the server's launches (events on its stream, read after stop)
    sat = point(None, args.serve_burst, 2)
    kprof = ctx.rb_profile_read()
    ctx.rb_profile(False)
    launches = int(sum(v[1] for v in kprof.values()))
    kernels = {k: {"ms": v[0], "launches": v[1]} for k, v in kprof.items() if v[1]}
    loads = []
    for frac in (0.25, 0.5, 0.8):
        rate = frac * sat["served_per_s"]
        loads.append(point(rate, max(64, int(rate * args.serve_seconds)), 3 + len(loads)))
    clk = clocks.stop()
    value = sat["served_per_s"]
    if world > 1:
        t = torch.tensor([value], device="cuda")
        torch.distributed.all_reduce(t)
        value = float(t.item())
    slots = None
    if rank == 0:
        m = ctx.m
        line = {
            "metric": "served reduced Newton solves/s (saturation) and p99 latency", "value": value,
            "unit": "solves/s", "n_gpus": world, "steps": 1, "warmup": 1,
            "ms_per_step": 1e3 * args.serve_burst / sat["served_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "bf16+f32+f64" if PREC[args.precision] == 1 else "f64", "data": "synthetic",
            "config": {"workload": wl.name, "n": f"U[{wl.size_range[0]},{wl.size_range[1]}]" if wl.size_range else wl.n_max,
                       "q_a": wl.q_a, "q_c": wl.q_c, "q_f": wl.q_f, "m": wl.m,
                       "precision": args.precision, "burst": args.serve_burst,
                       "parallelism": f"replicas x{world}",
                       "l2": "not flushed (serving: operators stay resident by design)"},
            "latency_ms": {"p50": loads[-1]["p50_ms"], "p99": loads[-1]["p99_ms"],
                           "at_offered_per_s": loads[-1]["offered_per_s"]},
            "saturation": sat, "load_points": loads,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 20 * args.serve_burst,
                    "d2h_bytes_per_step": (8 * (wl.n_max + m) + 32) * args.serve_burst},
            "gpu_launches": launches, "kernels": kernels, "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def combined_pressure_modes(U, Pp, rtol=1e-10):
    """Pressure data of the velocity basis by the second construction of Sec. 4.2: POD of the
    velocity snapshots U [K][n] by the method of snapshots (eigenvectors of U U^T scaled to
    orthonormal modes psi_j = sum_i v^j_i u_i, the modes with eigenvalue below rtol times the
    largest dropped), pressure functions p^_j = sum_i v^j_i p_i from their pressures Pp [K][m]
    with the same coefficients. Returned in the coordinates of the reduced velocity basis the
    solver uses, P_hat [m][n] with p = P_hat u, and the number of POD modes kept."""
    n = U.shape[1]
    lam, W = np.linalg.eigh(U @ U.T)
    order = np.argsort(lam)[::-1][:n]
    keep = order[lam[order] > rtol * lam[order[0]]]
    V = W[:, keep] / np.sqrt(lam[keep])[None, :]
    Psi = U.T @ V          # [n][r] orthonormal POD modes in reduced coordinates
    return (Pp.T @ V) @ Psi.T, len(keep)


def pressure_reconstruction(rb, ctx, wl, batch, d_u, d_n, p_rec, kprof, stream, flush, args,
                            steps, warmup):
    """Pressure reconstruction (Sec. 4.2) against recovery on the same batch: the modes fitted
    from training queries of the same workload (solved, pressure recovered), then p = P_hat u for
    the timed batch's velocities; kernel time by CUDA events, error against recovery."""
    import torch
    K = 1024
    qt = synth.make_queries(wl, batch=batch * max(1, int(os.environ.get("WORLD_SIZE", "1"))) + K)
    mu_t, n_t = qt.mu[-K:], qt.n[-K:]
    full = n_t == wl.n_max
    U, Pp, info = ctx.rb_solve(mu_t[full], n_t[full])
    good = info["status"] == 0
    P_hat, r = combined_pressure_modes(U[good], Pp[good])
    ctx.rb_load_pressure_modes(P_hat)
    d_pr = torch.empty((batch, P_hat.shape[0]), dtype=torch.float64, device=d_u.device)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(warmup + steps)]
    with torch.cuda.stream(stream):
        for a, b in ev:
            flush.zero_()
            a.record(stream)
            ctx.rb_reconstruct_pressure_device(d_u, batch, d_n, d_pr, stream.cuda_stream)
            b.record(stream)
    torch.cuda.synchronize()
    t = [a.elapsed_time(b) for a, b in ev[warmup:]]
    p_r = d_pr.cpu().numpy()
    err = np.linalg.norm(p_r - p_rec, axis=1) / np.linalg.norm(p_rec, axis=1)
    rec_ms = sum(kprof.get(k, (0.0, 0))[0] for k in ("k_pressure", "k_tc_gemm<sliced,pressure>"))
    rec_ms /= steps
    return {"ms_per_step": float(np.mean(t)), "recovery_ms_per_step": rec_ms,
            "rel_err_vs_recovery": {"median": float(np.median(err)), "max": float(err.max())},
            "modes": f"m_r = {P_hat.shape[0]}, {r} POD modes (eigenvalues above 1e-10 of the "
                     f"largest) of {int(good.sum())} training queries of the workload (combined "
                     "basis, second construction of Sec. 4.2)"}


def plain_fp64(rb, ops, q, batch, dev, flush, steps, tol_res=None):
    """The plain FP64 GPU path (one CTA per query, every step in FP64) on the same batch, or on
    its first two waves (2 x 152 queries) when one FP64 query-iteration exceeds 1 GFLOP."""
    import torch
    wl = ops.wl
    if 2.0 * wl.q_c * wl.n_max ** 3 > 1e9:
        batch = min(batch, 304)
        q = synth.QuerySet(q.mu[:batch].copy(), q.n[:batch].copy())
    ctx = rb.Context(precision=rb.RB_PREC_FP64, device=dev.index, theta_family=wl.theta_family,
                     tol_res=tol_res)
    ctx.load_set(ops)
    stream = torch.cuda.Stream(device=dev)
    d_mu = torch.from_numpy(q.mu).to(dev)
    d_n = torch.from_numpy(q.n).to(dev)
    d_u = torch.empty((batch, ctx.n_max), dtype=torch.float64, device=dev)
    d_p = torch.empty((batch, max(ctx.m, 1)), dtype=torch.float64, device=dev) if ctx.m else None
    d_info = torch.empty((batch, 4), dtype=torch.float64, device=dev)
    steps = max(2, min(steps, 3))
    with torch.cuda.stream(stream):
        ctx.rb_solve_device(d_mu, batch, d_n, d_u, d_p, d_info, stream.cuda_stream)
        ev = []
        for _ in range(steps):
            flush.zero_()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            ctx.rb_solve_device(d_mu, batch, d_n, d_u, d_p, d_info, stream.cuda_stream)
            e.record(stream)
            ev.append((s, e))
    torch.cuda.synchronize()
    ms = [s.elapsed_time(e) for s, e in ev]
    ctx.close()
    return {"value": batch * len(ms) / (sum(ms) / 1e3), "unit": "solves/s",
            "ms_per_step": float(np.mean(ms)), "queries_per_step": int(batch)}


if __name__ == "__main__":
    main()
