#!/usr/bin/env python3
"""Benchmark of the fused FP32 bounce map on 2048^2 resonators.

Workload: two 2048 x 2048 complex64 resonators, Fresnel number 1000,
g0 in {0.1, 0.3}, T1 = 1e4 bounces, R = 0.9, super-Gaussian pump (order 10,
radius 0.8), 8-pixel absorbing edge, seeded noise start.  One step = B
bounces (default 500, one captured CUDA graph per resonator) of each
resonator; the default 20 timed steps are the full 1e4 round trips.  The two
resonators run concurrently on their own streams (independent resonators
overlap on the device; each keeps its state resident).

Prints one JSON line.  `value` is resonator round trips per second over the
timed steps with the state resident on the device (CUDA events, L2 flushed
between steps).  Alongside: per-kernel event timing and the HBM roofline of
the dominant sweep, the same metric end to end through the C ABI from pinned
host buffers, the one-stream (sequential) rate, the batched 256-resonator
parameter sweep, the plain FP64 GPU path and a cuFFT + PyTorch pointwise form
on the same GPU (comparisons only), the error against the FP64 oracle after
one bounce, and the oracle's own rate on the host cores.

`--impl reference` times the FP64 CPU oracle on the same workload instead
(bounded samples of the same resonators per step).
Under torchrun each rank runs its own pair of resonators (weak scaling).
"""
from __future__ import annotations

import argparse
import csv
import dataclasses
import hashlib
import io
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1410_2855_gb300 import workloads as wl  # noqa: E402

METRIC = "round trips/s at 2048² FP32 vs FP64, % HBM peak; serve p50/p99 latency"
UNIT = "round trips/s"
COL_BYTES_PER_PT = 16   # column sweep: read and write the complex64 field
ROW_BYTES_PER_PT = 24   # row sweep: field (8+8) and inversion (4+4)
KERNEL_SOURCES = ["fft_core.cuh", "sweep.cuh", "sweep_tma.cuh", "tma.cuh", "launch.cuh", "k_fp32_col.cu",
                  "k_fp32_row.cu"]


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--bounces-per-step", type=int, default=500)
    ap.add_argument("--no-comparisons", action="store_true", help="skip the comparison legs")
    ap.add_argument("--col-tile", type=int, default=0, help="fixed column-sweep tile width (0: autotune)")
    ap.add_argument("--col-order", type=int, default=0, help="radix order with a fixed --col-tile")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests of the 50 req/s serving replay (the first arrivals of the seeded trace)")
    ap.add_argument("--serve-capacity-requests", type=int, default=100,
                    help="requests of the serving replay at a sustainable rate")
    ap.add_argument("--serve-capacity-rate", type=float, default=2.0, help="its arrival rate, requests/s")
    ap.add_argument("--sweep-case", default="",
                    help="small case for a profiler: KIND:N[:TILE[:ORDER]] runs --steps sweeps (KIND col or row) "
                         "of one seeded n x n resonator after --warmup sweeps, prints one line and exits")
    ap.add_argument("--batch-case", action="store_true",
                    help="small case for a profiler: --warmup then --steps bounces of the 256-resonator sweep")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def workload(rank: int):
    return [wl.Resonator(n=c.n, fresnel=c.fresnel, g0=c.g0, T1=c.T1, R=c.R, seed=c.seed + 1000 * rank)
            for c in wl.C3]


def config_block():
    """The workload, the same in both arms (the bounce count per step of each
    arm is reported beside it)."""
    c = wl.C3[0]
    return {"workload": "two 2048x2048 complex64 resonators, N_F=1000, g0 in {0.1,0.3}, T1=1e4, R=0.9, "
                        "super-Gaussian pump (order 10, r=0.8), 8 px edge, 1e4 round trips per resonator",
            "grid": c.n, "resonators": len(wl.C3), "fresnel": c.fresnel, "g0": [r.g0 for r in wl.C3],
            "T1": c.T1, "R": c.R,
            "l2": "GPU arm: L2 flushed between steps (256 MiB write), each resonator's 48 MiB state L2-resident "
                  "within a step; host arm: not applicable"}


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples (200 ms) of SM clock and throttle reasons."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = ""

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        rows = [r for r in csv.reader(io.StringIO(self.out or "")) if len(r) >= 9]
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------ helpers

def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def kernel_source_sha():
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_1410_2855_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, n: int):
    """DRAM bytes per launch from the committed ncu summary of this kernel, or
    None when the summary is missing or the kernel source changed since."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{n}.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if ":" in line and line.strip().startswith(("traffic_bytes_per_launch", "kernel_source_sha",
                                                    "- traffic_bytes_per_launch", "- kernel_source_sha")):
            k, v = line.split(":", 1)
            vals[k.strip(" -*`")] = v.strip(" `")
    if vals.get("kernel_source_sha") != kernel_source_sha():
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def oracle_params(p):
    import oracle as orc
    return orc.make_params(p.n, orc.alpha_from_fresnel(p.fresnel, p.d_over_w), p.g0, p.T1, p.R, Isat=p.Isat,
                           edge=p.edge, pump_order=p.pump_order, pump_radius=p.pump_radius)


def oracle_setup_s(params_list, E0s, N0s, threads):
    """Seconds the oracle spends per call before its first bounce (pump,
    phase table in long double, buffers): the median of three calls of zero
    bounces, per resonator."""
    import oracle as orc
    out = []
    for p, E, N in zip(params_list, E0s, N0s):
        ts = []
        for _ in range(3):
            t0 = time.perf_counter()
            orc.run(p, E, N, 0, nthreads=threads, history=False)
            ts.append(time.perf_counter() - t0)
        out.append(statistics.median(ts))
    return out


def oracle_rate(params_list, E0s, N0s, budget_s=12.0, horizons=(1, 20)):
    """Bounces/s of the FP64 oracle on the host cores (bounded sample), and
    its fields after each of `horizons` bounces from the starting state
    (those runs are part of the timed sample).  Every call pays the oracle's
    set-up, which is timed separately and taken out, so the rate is bounces
    over bounce time."""
    import oracle as orc
    threads = orc.threads_available(os.cpu_count() or 1)
    setup = oracle_setup_s(params_list, E0s, N0s, threads)
    done, t_total = 0, 0.0
    fields = {}

    def timed_run(i, nb):
        nonlocal done, t_total
        t0 = time.perf_counter()
        E, _, _ = orc.run(params_list[i], E0s[i], N0s[i], nb, nthreads=threads, history=False)
        t_total += max(time.perf_counter() - t0 - setup[i], 1e-9)
        done += nb
        return E

    for h in horizons:
        for i in range(len(params_list)):
            fields[(i, h)] = timed_run(i, h)
    while t_total < budget_s and done < 64:
        for i in range(len(params_list)):
            timed_run(i, 4)
    return done / t_total, threads, done, fields, statistics.mean(setup)


def radix_passes(n: int, order: int) -> str:
    """The radix sequence of a column transform of side n in radix order
    `order` (16s with the small pass last, first or second), e.g. "16.16.8"."""
    logn = n.bit_length() - 1
    p = [16] * (logn // 4)
    if logn % 4:
        p.insert(len(p) if order == 0 else (0 if order == 1 or len(p) < 2 else 1), 1 << (logn % 4))
    return ".".join(map(str, p))


def multi_stream_rate(rt, torch, params, B, steps=3):
    """Round trips/s of len(params) resonators, each on its own stream with
    graphs of B bounces, stepped together; L2 flushed before each timed step."""
    main = torch.cuda.Stream()
    streams = [torch.cuda.Stream() for _ in params]
    res = [rt.Resonator.from_params(p, cuda_stream=s.cuda_stream, chunk=B) for p, s in zip(params, streams)]
    fork = Fork(torch, main, streams)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def step():
        fork.begin()
        for r in res:
            rt.rt_step(r.h, B)
        fork.end()

    with torch.cuda.stream(main):
        step()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(main)
            step()
            b.record(main)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    for r in res:
        r.sync()
        r.close()
    return len(params) * B * steps / (sum(ms) / 1e3)


def graph_sweep_ms(rt, torch, r, stream, kind, reps=100):
    """Average duration of one sweep of `kind`: a CUDA graph of reps back-to-back
    launches on the resonator's stream, events around a replay."""
    for _ in range(3):
        rt.rt_sweep(r.h, kind)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        for _ in range(reps):
            rt.rt_sweep(r.h, kind)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        g.replay()
        a.record(stream)
        g.replay()
        b.record(stream)
    torch.cuda.synchronize()
    del g
    return a.elapsed_time(b) / reps


def rel_l2(a, b):
    return float(np.linalg.norm(np.asarray(a, np.complex128) - b) / np.linalg.norm(b))


def batch_slot_errors(rt, orc, threads, stream):
    """Relative L2 against the FP64 oracle after 1 and 20 bounces of one
    sampled resonator per grid size of the batched sweep (the first of each
    size among the 256), run in a batch through the batched kernels, the
    oracle started from the slot's own initial field and its own pump."""
    jobs = wl.batch_sweep(count=256, sides=(256, 512, 1024))
    first = {}
    for i, j in enumerate(jobs):
        first.setdefault(j.n, i)
    picks = [jobs[i] for i in sorted(first.values())]
    out = []
    with rt.Batch(picks, chunk=0, cuda_stream=stream.cuda_stream) as bt:
        E0 = [bt.field(i) for i in range(len(picks))]
        bt.step(1)
        E1 = [bt.field(i) for i in range(len(picks))]
        bt.step(19)
        E20 = [bt.field(i) for i in range(len(picks))]
    for k, j in enumerate(picks):
        q = oracle_params(j)
        N0 = orc.pump(q)
        o1, _, _ = orc.run(q, E0[k], N0, 1, nthreads=threads, history=False)
        o20, _, _ = orc.run(q, E0[k], N0, 20, nthreads=threads, history=False)
        out.append({"slot": jobs.index(j), "n": j.n, "fresnel": j.fresnel, "bounce1_rel_l2": rel_l2(E1[k], o1),
                    "bounce20_rel_l2": rel_l2(E20[k], o20)})
    return out


def served_request_errors(rt, orc, threads, stream):
    """Relative L2 against the FP64 oracle of served results: the first
    request of each grid size of the serving trace, submitted for 1 and for
    20 bounces together (they share rounds), each compared with the oracle
    run from the same seeded noise start (the oracle's own generator,
    rounded to complex64 as the library rounds it) and its own pump."""
    trace = wl.serve_trace(count=200, rate_hz=50.0)
    first = {}
    for q in trace:
        first.setdefault(q.job.n, q.job)
    picks = [first[n] for n in sorted(first)]
    outs = {}
    with rt.Server(chunk=500, budget_bytes=8 << 30, cuda_stream=stream.cuda_stream) as srv:
        for j in picks:
            for nb in (1, 20):
                buf = np.zeros((j.n, j.n), np.complex64)
                srv.submit(j, nb, buf)
                outs[(j.n, nb)] = buf
        srv.drain(600.0)
        res = srv.poll(64)
    assert all(r.status == 0 for r in res)
    out = []
    for j in picks:
        q = oracle_params(j)
        E0, N0 = orc.init_state(q, j.seed, j.noise_amp)
        E0 = E0.astype(np.complex64).astype(np.complex128)
        o1, _, _ = orc.run(q, E0, N0, 1, nthreads=threads, history=False)
        o20, _, _ = orc.run(q, E0, N0, 20, nthreads=threads, history=False)
        out.append({"n": j.n, "fresnel": j.fresnel, "bounce1_rel_l2": rel_l2(outs[(j.n, 1)], o1),
                    "bounce20_rel_l2": rel_l2(outs[(j.n, 20)], o20)})
    return out


# ---------------------------------------------------------------- reference

REF_BOUNCES_PER_STEP = 4


def run_reference(args):
    rank, local_rank, world = dist_env()
    if rank != 0:
        return
    import oracle as orc
    orc.build()
    res = workload(0)
    params = [oracle_params(p) for p in res]
    init = [orc.init_state(p, r.seed, r.noise_amp) for p, r in zip(params, res)]
    threads = orc.threads_available(os.cpu_count() or 1)
    setup = oracle_setup_s(params, [E for E, _ in init], [N for _, N in init], threads)
    k = REF_BOUNCES_PER_STEP
    # each step: k bounces of each resonator from its start (a bounded sample
    # of the workload); the oracle's per-call set-up is taken out of each call
    for _ in range(args.warmup):
        for p, (E, N) in zip(params, init):
            orc.run(p, E, N, k, nthreads=threads, history=False)
    step_s = []
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        t = 0.0
        for i, (p, (E, N)) in enumerate(zip(params, init)):
            t0 = time.perf_counter()
            orc.run(p, E, N, k, nthreads=threads, history=False)
            t += max(time.perf_counter() - t0 - setup[i], 1e-9)
        step_s.append(t)
    wall = time.perf_counter() - t_wall
    dt = sum(step_s)
    value = args.steps * k * len(params) / dt
    sample = (f"{args.steps} steps x {k} bounces of each of the {len(params)} 2048^2 resonators (FP64 oracle, "
              f"{threads} threads); the oracle's set-up before the first bounce of each call "
              f"({statistics.mean(setup):.3f} s: pump, phase table, buffers) is timed separately and not counted")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_block(),
        "bounces_per_step": k, "oracle_setup_s_per_call": statistics.mean(setup), "wall_s_with_setup": wall,
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ---------------------------------------------------------------------- ours

class Fork:
    """Run work on several streams as one step: the streams wait for an
    event on `main` before the work and `main` waits for all of them after."""

    def __init__(self, torch, main, streams):
        self.torch, self.main, self.streams = torch, main, streams

    def begin(self):
        e = self.torch.cuda.Event()
        e.record(self.main)
        for s in self.streams:
            s.wait_event(e)

    def end(self):
        for s in self.streams:
            e = self.torch.cuda.Event()
            e.record(s)
            self.main.wait_event(e)


def torch_cufft_rate(p, steps=100):
    """Comparison only: the same bounce with cuFFT (torch.fft) and PyTorch
    pointwise kernels in FP32."""
    import torch
    n = p.n
    dev = torch.device("cuda")
    m = torch.fft.fftfreq(n, d=1.0 / n, device=dev).to(torch.float64)
    alpha = p.d_over_w ** 2 / p.fresnel
    ph = torch.remainder(alpha * (m[None, :] ** 2 + m[:, None] ** 2), 2.0)
    H = torch.polar(torch.ones_like(ph), -math.pi * ph).to(torch.complex64)
    x = (torch.arange(n, device=dev, dtype=torch.float32) - n // 2) / (n // 2)
    r2 = x[None, :] ** 2 + x[:, None] ** 2
    N0 = (p.g0 * torch.exp(-(r2 / p.pump_radius ** 2) ** (p.pump_order / 2))).float()
    A = torch.zeros(n, device=dev)
    A[p.edge:n - p.edge] = 1
    A2 = (A[None, :] * A[:, None]) * math.sqrt(p.R)
    E = (torch.randn(n, n, device=dev, dtype=torch.complex64) * 1e-6)
    N = N0.clone()

    def bounce(E, N):
        Ep = torch.fft.ifft2(torch.fft.fft2(E) * H)
        inten = Ep.real ** 2 + Ep.imag ** 2
        E = Ep * (A2 * torch.exp(0.5 * N))
        N = N + (N0 - N * (1 + inten / p.Isat)) / p.T1
        return E, N

    for _ in range(5):
        E, N = bounce(E, N)
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record()
    for _ in range(steps):
        E, N = bounce(E, N)
    e.record()
    torch.cuda.synchronize()
    return steps / (s.elapsed_time(e) / 1e3)


def weak_scaling_rate(local_ms, local_units, world, device=None):
    """Whole-job rate of a weak-scaling run: every rank processed local_units
    in its own local_ms; the job took the slowest rank's time.  Returns
    (units per second over all ranks, max ms)."""
    total_ms = float(local_ms)
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return world * local_units / (total_ms / 1e3), total_ms


def _pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))] if xs else None


def serve_replay(rt, stream, count=1000, rate_hz=50.0, policy=0, round_points=0):
    """Replay the first `count` requests of the seeded Poisson stream (mean
    rate_hz; sides 128..2048, bounces log-uniform in [1e3, 1e5]) against a
    server with 500-bounce rounds and an 8 GiB budget; latency is completion
    minus submission on the server clock, split into queueing (admission
    minus submission) and service (completion minus admission).  policy: the
    server's scheduling policy (0 first come first served, 1 shortest
    remaining work first)."""
    trace = wl.serve_trace(count=count, rate_hz=rate_hz)
    t_wall = time.perf_counter()
    with rt.Server(chunk=500, budget_bytes=8 << 30, cuda_stream=stream.cuda_stream, policy=policy,
                   round_points=round_points) as srv:
        t0 = time.perf_counter()
        for req in trace:
            delay = t0 + req.arrival_s - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            srv.submit(req.job, req.bounces)
        srv.drain(3600.0)
        res = srv.poll(4 * count)
        st = srv.stats()
    lat = [r.finish_s - r.submit_s for r in res]
    work = sum(float(r.n) ** 2 * r.bounces for r in res)
    span = max(r.finish_s for r in res) - min(r.submit_s for r in res)
    arrivals_s = max(trace[-1].arrival_s, 1e-9)
    offered = sum(float(q.job.n) ** 2 * q.bounces for q in trace) / arrivals_s
    return {"workload": f"first {count} requests of a Poisson stream at {rate_hz:g} req/s, sides uniform over "
                        "{128,...,2048}, bounces log-uniform in [1e3,1e5]; 500-bounce rounds, 8 GiB budget",
            "policy": "shortest remaining work first" if policy else "every resident request every round",
            "requests": len(res), "failed": sum(1 for r in res if r.status != 0),
            "p50_latency_s": _pct(lat, 0.5), "p99_latency_s": _pct(lat, 0.99),
            "p50_queue_s": _pct([r.admit_s - r.submit_s for r in res], 0.5),
            "p99_queue_s": _pct([r.admit_s - r.submit_s for r in res], 0.99),
            "p50_service_s": _pct([r.finish_s - r.admit_s for r in res], 0.5),
            "p99_service_s": _pct([r.finish_s - r.admit_s for r in res], 0.99),
            "round_trips_per_s": sum(r.bounces for r in res) / span,
            "offered_req_per_s": len(trace) / arrivals_s, "served_req_per_s": len(res) / span,
            "served_point_bounces_per_s": work / span, "offered_point_bounces_per_s": offered,
            "offered_over_served": offered / (work / span), "rounds": st.rounds,
            "peak_resident_bytes": st.peak_resident_bytes, "round_points": round_points or (1 << 23),
            "wall_s": time.perf_counter() - t_wall}


def run_ours(args):
    import torch
    from paper_1410_2855_gb300 import build, rt

    rank, local_rank, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local_rank)
    build.build()
    dev = torch.device("cuda", local_rank)
    main = torch.cuda.Stream(device=dev)
    B, K, W = args.bounces_per_step, args.steps, args.warmup
    params = workload(rank)
    from paper_1410_2855_gb300 import tune
    if args.col_tile:
        tune.rt_tune_set(params[0].n, args.col_tile)
        tune.rt_tune_set_order(params[0].n, args.col_order)
        col_tile, tile_source = args.col_tile, "fixed on the command line"
    else:
        # column-sweep tile width and radix order for this GPU (2048^2 and the larger-than-L2 4096^2)
        # first the sweep alone, then whole bounces of the resonators as this
        # run steps them (one stream each), which decides: a tile that is
        # fastest alone can hold shared memory the other stream's sweeps need
        kernel_pick = tune.rt_autotune(params[0].n, reps=50)[0], tune.rt_tune_get_order(params[0].n)[0]
        col_tile, order_pick, _ = tune.rt_autotune_concurrent(params[0].n, len(params), bounces=100, reps=3)
        tune.rt_autotune(4096, reps=20)
        tune.rt_autotune_concurrent(4096, 2, bounces=20, reps=3)
        tile_source = (f"autotuned at start-up on whole bounces of the {len(params)} resonators on their streams "
                       f"(the column sweep alone picked tile {kernel_pick[0]}, order {kernel_pick[1]})")
    col_order = tune.rt_tune_get_order(params[0].n)[0]
    streams = [torch.cuda.Stream(device=dev) for _ in params]
    res = [rt.Resonator.from_params(p, precision=rt.RT_FP32, cuda_stream=s.cuda_stream, chunk=B)
           for p, s in zip(params, streams)]
    fork = Fork(torch, main, streams)
    P = params[0].n ** 2
    E0 = [r.field() for r in res]
    N0 = [r.inversion() for r in res]
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def step():
        fork.begin()
        for r in res:
            rt.rt_step(r.h, B)
        fork.end()

    with torch.cuda.stream(main):
        for _ in range(W):
            step()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        barrier()
        torch.cuda.synchronize()
        with ClockSampler(local_rank) as clk:
            for k in range(K):
                flush.fill_(float(k))
                evs[k][0].record(main)
                step()
                evs[k][1].record(main)
            torch.cuda.synchronize()
            barrier()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        value, total_ms = weak_scaling_rate(sum(step_ms), K * B * len(res), world, dev)
        for r in res:
            r.sync()

        # per-kernel durations on the launching stream, one resonator at a time
        # (the kernels alone on the GPU): first with events around each sweep
        reps = 200
        r, st = res[0], streams[0]
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3 * reps)]
        for i in range(reps):
            e[3 * i].record(st)
            rt.rt_sweep(r.h, rt.RT_SWEEP_COLUMNS)
            e[3 * i + 1].record(st)
            rt.rt_sweep(r.h, rt.RT_SWEEP_ROWS)
            e[3 * i + 2].record(st)
        torch.cuda.synchronize()
        col_ev_ms = statistics.mean(e[3 * i].elapsed_time(e[3 * i + 1]) for i in range(reps))
        row_ev_ms = statistics.mean(e[3 * i + 1].elapsed_time(e[3 * i + 2]) for i in range(reps))

        # the same sweeps back to back, as the bounce loop runs them: `reps`
        # launches of one kind captured in one CUDA graph on the resonator's
        # stream, events around a replay (no event between launches; the row
        # sweeps alone keep the state finite: saturable gain).  Direct
        # back-to-back launches if the capture is refused.
        b2b, b2b_how = {}, "a CUDA graph of"
        for kind in (rt.RT_SWEEP_COLUMNS, rt.RT_SWEEP_ROWS):
            for _ in range(5):
                rt.rt_sweep(r.h, kind)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            try:
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=st):
                    for _ in range(reps):
                        rt.rt_sweep(r.h, kind)
                with torch.cuda.stream(st):
                    g.replay()
                    a.record(st)
                    g.replay()
                    b.record(st)
                torch.cuda.synchronize()
                del g
            except RuntimeError:
                torch.cuda.synchronize()
                b2b_how = "direct"
                a.record(st)
                for _ in range(reps):
                    rt.rt_sweep(r.h, kind)
                b.record(st)
                torch.cuda.synchronize()
            b2b[kind] = a.elapsed_time(b) / reps
        col_ms, row_ms = b2b[rt.RT_SWEEP_COLUMNS], b2b[rt.RT_SWEEP_ROWS]

    peak, peak_kind = measured_peak()
    col_gbs = COL_BYTES_PER_PT * P / (col_ms / 1e3) / 1e9
    row_gbs = ROW_BYTES_PER_PT * P / (row_ms / 1e3) / 1e9
    if row_ms >= col_ms:
        dom, dom_bytes, dom_gbs, dom_ms = "row_sweep", ROW_BYTES_PER_PT * P, row_gbs, row_ms
    else:
        dom, dom_bytes, dom_gbs, dom_ms = "column_sweep", COL_BYTES_PER_PT * P, col_gbs, col_ms
    bounce_gbs = (COL_BYTES_PER_PT + ROW_BYTES_PER_PT) * P * value / world / 1e9

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": total_ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": config_block(),
        "bounces_per_step": B,
        "launch": {"graph": f"one CUDA graph per {B} bounces per resonator",
                   "streams": "one per resonator, concurrent", "col_tile": col_tile, "col_tile_source": tile_source,
                   "col_radix_order": col_order,
                   "col_radix_passes": radix_passes(params[0].n, col_order),
                   "batch_launch": "autotuned in the batch_sweep leg"},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": dom_gbs, "peak": peak, "unit": "GB/s",
                     "frac": dom_gbs / peak, "peak_kind": f"of {peak_kind}",
                     "traffic": profiled_traffic(dom, params[0].n),
                     "algorithmic_bytes_per_launch": dom_bytes, "avg_launch_ms": dom_ms,
                     "timing": f"CUDA events around {b2b_how} {reps} back-to-back launches on the kernel's stream, "
                               "kernel alone on the GPU",
                     "avg_launch_ms_events_around_each": col_ev_ms if dom == "column_sweep" else row_ev_ms},
        "kernels": {"column_sweep": {"avg_ms": col_ms, "gbs": col_gbs, "bytes_per_launch": COL_BYTES_PER_PT * P,
                                     "avg_ms_events_around_each": col_ev_ms},
                    "row_sweep": {"avg_ms": row_ms, "gbs": row_gbs, "bytes_per_launch": ROW_BYTES_PER_PT * P,
                                  "avg_ms_events_around_each": row_ev_ms}},
        "bounce_hbm": {"bytes_per_point": COL_BYTES_PER_PT + ROW_BYTES_PER_PT, "achieved_gbs": bounce_gbs,
                       "frac": bounce_gbs / peak, "peak_kind": f"of {peak_kind}"},
        "gpu_launches": 2 * K * B * len(res),
        "clocks": clk.summary(),
    }

    # the comparison legs (larger-than-L2, batch, serving, FP64 and cuFFT
    # forms, the oracle on the host) run at N = 1 only: a multi-GPU run
    # measures the scaling of the headline step
    if not args.no_comparisons and world == 1:
        out.update(comparisons(args, rt, torch, main, streams, params, res, E0, N0, rank, world))
        big = out["larger_than_l2"]["two_4096"]
        # the case whose state really streams through HBM, as a second roofline entry
        out["roofline"]["larger_than_l2"] = {
            "bound": "hbm", "kernel": "bounce (column + row sweep) of two 4096^2 resonators on two streams",
            "achieved": big["bounce_gbs"], "peak": peak, "unit": "GB/s", "frac": big["bounce_hbm_frac"],
            "peak_kind": f"of {peak_kind}", "algorithmic_bytes_per_bounce": 40 * 4096 ** 2, "traffic": None,
            "timing": "CUDA events around steps of 100 bounces per resonator, L2 flushed before each step"}
    if world > 1:
        torch.distributed.barrier()
    for r in res:
        r.close()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def comparisons(args, rt, torch, main, streams, params, res, E0, N0, rank, world):
    from paper_1410_2855_gb300 import tune
    B = args.bounces_per_step
    extra = {}
    P = params[0].n ** 2
    fork = Fork(torch, main, streams)
    # ---- end to end through the C ABI from pinned host buffers
    hostE = [torch.from_numpy(e.view(np.float32).copy()).pin_memory() for e in E0]
    hostN = [torch.from_numpy(nv.copy()).pin_memory() for nv in N0]
    outE = [torch.empty(P * 2, dtype=torch.float32).pin_memory() for _ in res]
    K2 = max(2, min(args.steps, 6))

    def e2e_step():
        fork.begin()
        for r, e, nv in zip(res, hostE, hostN):
            rt.rt_write_field(r.h, e)
            rt.rt_write_inversion(r.h, nv)
            rt.rt_step(r.h, B)
        for r, o in zip(res, outE):
            rt.rt_read_field(r.h, o)     # blocks until that resonator's step is done
        fork.end()

    with torch.cuda.stream(main):
        e2e_step()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(K2):
            e2e_step()
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
    extra["e2e"] = {"value": world * K2 * B * len(res) / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": len(res) * 12 * P, "d2h_bytes_per_step": len(res) * 8 * P,
                    "steps": K2, "timing": "host wall clock around the steps"}

    # ---- the same resonators one after the other on a single stream
    with torch.cuda.stream(main):
        one = [rt.Resonator.from_params(p, cuda_stream=main.cuda_stream, chunk=B) for p in params]
        for r in one:
            r.step(B)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(main)
        for _ in range(4):
            for r in one:
                r.step(B)
        e.record(main)
        torch.cuda.synchronize()
        for r in one:
            r.close()
    extra["one_stream"] = {"value": 4 * B * len(params) / (s.elapsed_time(e) / 1e3), "unit": UNIT}

    # ---- curved and rough mirror (aperture phase in the row sweep), one resonator on one stream
    extra["curved_mirror"] = {}
    flat = dataclasses.replace(wl.CURVED, z_over_F=0.0, roughness_rms=0.0)
    lens = dataclasses.replace(wl.CURVED, roughness_rms=0.0)
    for name, q in (("flat", flat), ("lens", lens), ("lens_roughness", wl.CURVED)):
        with torch.cuda.stream(main):
            with rt.Resonator.from_params(q, cuda_stream=main.cuda_stream, chunk=B) as r:
                r.step(B)
                torch.cuda.synchronize()
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(main)
                r.step(2 * B)
                e.record(main)
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(51)]
                for i in range(50):
                    ev[i].record(main)
                    rt.rt_sweep(r.h, rt.RT_SWEEP_ROWS)
                ev[50].record(main)
                torch.cuda.synchronize()
                r.sync()
                extra["curved_mirror"][name] = {
                    "round_trips_per_s": 2 * B / (s.elapsed_time(e) / 1e3),
                    "row_sweep_ms": ev[0].elapsed_time(ev[50]) / 50}
    extra["curved_mirror"]["workload"] = ("2048^2, N_F 1000, g0 0.3, R 0.9; z/F 0.16 (50 mm mirror, L 2 mm); "
                                          "roughness 0.05 rad rms; one stream, graphs of %d bounces" % B)

    # ---- the other extensions of the map on the same 2048^2 resonator, one stream
    base = params[1]
    variants = {"slices_4": (base, dict(slices=4)),
                "taper16_exact_relax": (dataclasses.replace(base, taper_px=16, relax=rt.RT_RELAX_EXACT), {})}
    extra["extensions"] = {}
    for name, (q, kw) in variants.items():
        with torch.cuda.stream(main):
            with rt.Resonator.from_params(q, cuda_stream=main.cuda_stream, chunk=100, **kw) as r:
                r.step(100)
                torch.cuda.synchronize()
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(main)
                r.step(400)
                e.record(main)
                torch.cuda.synchronize()
                r.sync()
                extra["extensions"][name] = {"round_trips_per_s": 400 / (s.elapsed_time(e) / 1e3)}
    with rt.Resonator.from_params(base, cuda_stream=main.cuda_stream, chunk=0) as r:
        buf = np.empty((base.n, base.n), np.complex64)
        r.field_at(0.5)
        t0 = time.perf_counter()
        for _ in range(5):
            rt.rt_read_field_at(r.h, 0.5, buf)
        extra["extensions"]["field_at_ms"] = (time.perf_counter() - t0) / 5 * 1e3
        r.set_pattern(rt.RT_PATTERN_VORTEX_ARRAY, 0.01, periods=64, out_of_phase=True, envelope=0.6)
        t0 = time.perf_counter()
        for _ in range(5):
            r.set_pattern(rt.RT_PATTERN_VORTEX_ARRAY, 0.01, periods=64, out_of_phase=True, envelope=0.6)
        extra["extensions"]["vortex_pattern_ms"] = (time.perf_counter() - t0) / 5 * 1e3
    extra["extensions"]["workload"] = ("2048^2, N_F 1000, g0 0.3, R 0.9, one stream; field_at and the pattern "
                                       "include the host copy / synchronisation (wall clock)")

    # ---- state larger than L2 (126 MB): the bounce streams its state through HBM
    peak, peak_kind = measured_peak()
    big = [dataclasses.replace(base, n=4096, fresnel=4000.0, seed=base.seed + 100 + i) for i in range(2)]
    four = [dataclasses.replace(base, seed=base.seed + 200 + i) for i in range(4)]
    rate_big = multi_stream_rate(rt, torch, big, 100)
    rate_one = multi_stream_rate(rt, torch, big[:1], 100)
    rate_four = multi_stream_rate(rt, torch, four, B // 5)
    st = torch.cuda.Stream()
    with rt.Resonator.from_params(big[0], cuda_stream=st.cuda_stream, chunk=0) as r:
        col4 = graph_sweep_ms(rt, torch, r, st, rt.RT_SWEEP_COLUMNS)
        row4 = graph_sweep_ms(rt, torch, r, st, rt.RT_SWEEP_ROWS)
    P4 = 4096 ** 2
    extra["larger_than_l2"] = {
        "two_4096": {"workload": "two 4096^2 resonators (N_F 4000, g0 0.3, R 0.9) on two streams: 384 MiB of "
                                 "state against a 126 MB L2; graphs of 100 bounces",
                     "round_trips_per_s": rate_big, "bounce_gbs": 40 * P4 * rate_big / 1e9,
                     "bounce_hbm_frac": 40 * P4 * rate_big / 1e9 / peak},
        "one_4096": {"round_trips_per_s": rate_one, "bounce_hbm_frac": 40 * P4 * rate_one / 1e9 / peak},
        "four_2048": {"workload": "four 2048^2 resonators on four streams (192 MiB of state), graphs of "
                                  f"{B // 5} bounces", "round_trips_per_s": rate_four,
                      "bounce_hbm_frac": 40 * P * rate_four / 1e9 / peak},
        "sweeps_4096": {"column_ms": col4, "column_frac": COL_BYTES_PER_PT * P4 / (col4 / 1e3) / 1e9 / peak,
                        "row_ms": row4, "row_frac": ROW_BYTES_PER_PT * P4 / (row4 / 1e3) / 1e9 / peak,
                        "col_tile": tune.rt_tune_get(4096)[0], "timing": "graph of 100 back-to-back launches"},
        "peak_kind": f"of {peak_kind}"}

    # ---- batched parameter sweep: 256 resonators of side 256/512/1024 in one graph per 100 bounces;
    # the launch form (one launch per sweep across sizes, or one per size class) and the graph chains
    # per class autotuned first
    jobs = wl.batch_sweep(count=256, sides=(256, 512, 1024))
    form = tune.autotune_batch(jobs, bounces=100, cuda_stream=main.cuda_stream)
    with torch.cuda.stream(main):
        with rt.Batch(jobs, chunk=100, history_cap=128, cuda_stream=main.cuda_stream) as bt:
            bt.step(100)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(main)
            bt.step(200)
            e.record(main)
            torch.cuda.synchronize()
            bt.sync()
            secs = s.elapsed_time(e) / 1e3
            Pb = sum(j.n ** 2 for j in jobs)
            peak, _ = measured_peak()
            extra["batch_sweep"] = {
                "workload": "256 resonators, sides uniform over {256,512,1024}, N_F log-uniform [100,1000], "
                            "g0 U[0.1,0.3], T1 U[1e3,1e4], R=0.95; one CUDA graph per 100 bounces",
                "round_trips_per_s": len(jobs) * 200 / secs, "point_bounces_per_s": Pb * 200 / secs,
                "hbm_frac": 40 * Pb * 200 / secs / 1e9 / peak, "footprint_bytes": bt.footprint(),
                "launch_form": (f"one launch per sweep across sizes ({form['split']} graph chains)" if form["mixed"]
                                else f"one launch per sweep and size class ({form['split']} graph chains per class)"),
                "autotune_round_trips_per_s": form["round_trips_per_s"]}

    # ---- serving: the first requests of the seeded 50 req/s Poisson stream
    # (several times what the GPU can serve: latency there is the backlog),
    # then a replay at a rate the GPU sustains (latency is service plus
    # modest queueing), each under both scheduling policies
    # (shortest-first advances only the least-work requests each round, so with hundreds resident it
    # runs many small rounds: its overload replay takes the first 300 arrivals and 32M-point rounds)
    extra["serve_overload"] = {
        "fifo": serve_replay(rt, main, count=args.serve_requests, rate_hz=50.0),
        "shortest_first": serve_replay(rt, main, count=min(args.serve_requests, 300), rate_hz=50.0,
                                       policy=rt.RT_SERVE_SHORTEST_FIRST, round_points=32 << 20)}
    extra["serve_capacity_rate"] = {
        "fifo": serve_replay(rt, main, count=args.serve_capacity_requests, rate_hz=args.serve_capacity_rate),
        "shortest_first": serve_replay(rt, main, count=args.serve_capacity_requests,
                                       rate_hz=args.serve_capacity_rate, policy=rt.RT_SERVE_SHORTEST_FIRST)}

    # ---- plain FP64 GPU path on the same GPU (unfused, six sweeps per bounce)
    p = params[1]
    with rt.Resonator.from_params(p, precision=rt.RT_FP64, cuda_stream=main.cuda_stream, chunk=50) as r64:
        with torch.cuda.stream(main):
            rt.rt_step(r64.h, 50)
            torch.cuda.synchronize()
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(main)
            rt.rt_step(r64.h, 200)
            e.record(main)
            torch.cuda.synchronize()
        r64.sync()
        fp64 = 200 / (s.elapsed_time(e) / 1e3)
    extra["fp64_plain"] = {"value": fp64, "unit": UNIT, "resonators": 1, "bounces": 200}
    extra["torch_cufft_fp32"] = {"value": torch_cufft_rate(p), "unit": UNIT, "resonators": 1,
                                 "note": "comparison only: cuFFT C2C + PyTorch pointwise kernels"}
    if rank == 0:
        # ---- error after one bounce against the FP64 oracle, and the oracle's rate
        import oracle as orc
        orc.build()
        oparams = [oracle_params(q) for q in params]
        E0w = [x.astype(np.complex128) for x in E0]
        N0o = [orc.pump(q) for q in oparams]
        rate, threads, done, fields, setup_s = oracle_rate(oparams, E0w, N0o)

        err1, err20 = [], []
        for i, (q, e0) in enumerate(zip(params, E0)):
            with rt.Resonator.from_params(q, precision=rt.RT_FP32, chunk=0) as r1:
                r1.set_field(e0)
                r1.step(1)
                err1.append(rel_l2(r1.field(), fields[(i, 1)]))
                r1.step(19)
                err20.append(rel_l2(r1.field(), fields[(i, 20)]))
        extra["error_vs_oracle"] = {"bounce1_rel_l2": err1, "bounce20_rel_l2": err20,
                                    "bar": {"bounce1": 1e-5, "bounce20": 1e-3},
                                    "resonators": "the two 2048^2 resonators, same start as the oracle",
                                    "batch_slots": batch_slot_errors(rt, orc, threads, main),
                                    "served_requests": served_request_errors(rt, orc, threads, main)}
        extra["cpu_baseline"] = {"value": rate, "unit": UNIT, "cores": threads, "kind": "oracle",
                                 "sample": f"{done} oracle bounces over the two 2048^2 resonators, runs of 1, 20 and 4 bounces "
                                           f"(FP64, {threads} threads); the set-up before the first bounce of each "
                                           f"call ({setup_s:.3f} s) is timed separately and not counted"}
    return extra


def run_case(args):
    """A small, fixed case for kernel captures (no timing, no JSON line)."""
    import torch
    from paper_1410_2855_gb300 import build, rt
    build.build()
    st = torch.cuda.Stream()
    if args.batch_case:
        jobs = wl.batch_sweep(count=256, sides=(256, 512, 1024))
        with rt.Batch(jobs, chunk=0, cuda_stream=st.cuda_stream) as b:
            b.step(args.warmup)
            b.step(args.steps)
            b.sync()
        print(f"batch case: 256 resonators, {args.warmup} + {args.steps} bounces")
        return
    from paper_1410_2855_gb300 import tune
    kind, n, *rest = args.sweep_case.split(":")
    n = int(n)
    tile, order = (int(rest[0]) if rest else 0), (int(rest[1]) if len(rest) > 1 else 0)
    if tile:
        tune.rt_tune_set(n, tile)
    tune.rt_tune_set_order(n, order)
    p = wl.Resonator(n=n, fresnel=1000.0 * n / 2048, g0=0.3, T1=1e4, R=0.9)
    with rt.Resonator.from_params(p, cuda_stream=st.cuda_stream, chunk=0) as r:
        r.set_field(wl.smooth_field(n, 3, 1.0, dtype=np.complex64))
        which = rt.RT_SWEEP_COLUMNS if kind == "col" else rt.RT_SWEEP_ROWS
        for _ in range(args.warmup + args.steps):
            rt.rt_sweep(r.h, which)
        r.sync()
    print(f"sweep case: {kind} sweeps of one {n}x{n} resonator, {args.warmup} + {args.steps}")


def main():
    args = parse_args()
    if args.sweep_case or args.batch_case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
