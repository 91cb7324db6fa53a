#!/usr/bin/env python
"""Throughput of the stochastic-ETD pseudo-spectral step on GB300.

Workload (one bench step = one SETD step of every replica): Model B (conserved
scalar field), d = 2, 1024 x 1024 periodic lattice, dx = 1, Gamma = 1, r = -1,
u = 1, T = 0.1, SETD1, h = 0.05, 2/3 dealiasing, R replicas per GPU started
from seeded iid N(0, 0.01^2) fields, with the shell-averaged structure factor
S(k, t) taken every 100 steps inside the timed region (at least once per timed
region).  Inputs are synthetic.

Prints one JSON line (rank 0).  Multi-GPU runs (torchrun, one rank per GPU)
shard replicas: every rank advances its own R replicas (disjoint Philox
replica counters), no data-path collective; timing is the max over ranks.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
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

import sft_inputs as W  # noqa: E402

METRIC = "Gsite-steps/s per GB300 + % HBM roofline, batched FP32 vs plain, at stated error"
UNIT = "Gsite-steps/s"
OBS_EVERY = 100
L2_BYTES = 129 * 1024 * 1024


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=32)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--replicas", type=int, default=64)
    ap.add_argument("--scheme", type=int, default=1)
    ap.add_argument("--h", type=float, default=0.05)
    ap.add_argument("--n", type=int, default=1024)
    ap.add_argument("--quick", action="store_true", help="skip the secondary measurements")
    ap.add_argument("--precision", type=int, default=0,
                    help="cgl_2048: 1 runs the split-BF16x3 tensor-core transforms of the precision study")
    ap.add_argument("--workload", default="model_b_1024",
                    choices=["model_b_1024", "model_a_64", "kpz_ensemble", "cgl_2048", "model_a_128_3d",
                             "model_a_128_3d_tangent", "sde0d", "dynamics", "model_b_1024_phase_shift",
                             "model_b_1024_real_space_noise", "model_b_768"],
                    help="model_b_1024 is the headline; the others print their own line for the other workloads")
    return ap.parse_args()


def workload(args):
    return W.model_b_1024(n=[args.n, args.n], scheme=args.scheme, h=args.h, replicas=args.replicas)


def scheme_name(s):
    return {0: "SETD-EM", 1: "SETD1", 2: "SETD2"}[s]


def observations(K):
    """S(k) calls inside a timed region of K steps: one after every OBS_EVERY
    steps, and one after all K steps when K < OBS_EVERY.  Returns (calls,
    steps between calls)."""
    return max(1, K // OBS_EVERY), min(OBS_EVERY, K)


def headline_config(w, R, ws, K):
    """The `config` of the headline line, shared by the GPU arm and the
    reference arm (the same workload, whichever arm times it)."""
    n_obs, obs_every = observations(K)
    return {"workload": "model_b_1024_%s_h%g" % (scheme_name(w.scheme), w.h), "field": "Model B (conserved)",
            "lattice": "%dx%d" % (w.n[0], w.n[1]), "replicas_per_gpu": R, "global_batch": R * ws,
            "scheme": scheme_name(w.scheme), "h": w.h, "observe_every": obs_every,
            "observations_timed": n_obs,
            "setup": "schedule autotuned and step graph captured before the warm-up (sft_prepare)",
            "parallelism": "replicas x%d" % ws,
            "l2": "working set %.0f MB > 129 MB L2, no flush" % (R * (w.n[0] // 2 + 1) * w.n[1] * 8 * 3 / 1e6)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist, device="cuda"):
    """The largest value of x over the ranks of the process group (x itself
    when there is none): the whole job takes as long as its slowest rank."""
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_replica0(rank, replicas_per_rank):
    """Global index of a rank's first replica: ranks take disjoint Philox
    replica counters, so N ranks of R replicas run one ensemble of N R."""
    return rank * replicas_per_rank


def algorithmic_bytes(w, scheme, ncols):
    """Algorithmic HBM bytes per replica of each kernel of one step of the
    two-pass design (x-major spectra, dealiased intermediates with ncols of the
    nx/2+1 x-columns):
      row pass:    read P, write Q                     (ncols * ny complex each)
      column pass: read Q, read + write phi, write P   (phi: (nx/2+1) * ny complex)
                   SETD2 adds read + write of F_prev on the ncols columns."""
    nx, ny = w.n[0], w.n[1]
    hx = nx // 2 + 1
    c8 = 8
    rows = 2 * ncols * ny * c8
    cols = (2 * ncols + 2 * hx) * ny * c8
    if scheme == 2:
        cols += 2 * ncols * ny * c8
    return rows, cols


def algorithmic_bytes_complex(nx, ny, scheme, dealias):
    """The same counts per replica for the complex 2-D step (CGL): the spectrum
    holds every a_x (nx columns); the intermediates carry the a_x with
    3 |a_x| < nx in compact order (2 ((nx - 1) // 3) + 1 columns) under 2/3
    truncation, all nx without it."""
    mx = 2 * ((nx - 1) // 3) + 1 if dealias == 1 else nx
    rows = 2 * mx * ny * 8
    cols = (2 * mx + 2 * nx) * ny * 8
    if scheme == 2:
        cols += 2 * mx * ny * 8
    return rows, cols


def hbm_roofline(kernel, alg_bytes, launch_ms):
    """Roofline entry of one kernel against the measured HBM copy bandwidth."""
    peak, src = measured_peak()
    achieved = alg_bytes / (launch_ms * 1e-3) / 1e9
    return {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "alg_bytes_per_launch": alg_bytes, "launch_ms": launch_ms,
            "peak_source": src}


# sources each recorded kernel is compiled from: its translation unit and the headers it includes
KERNEL_SOURCES = {
    "k2_cols_real": ["sft_k2d_cols.cu", "sft_k2d_cols_large.cu", "sft_k2d_cols.cuh", "sft_step_common.cuh", "sft_device.cuh", "sft_async.cuh",
                     "sft_internal.h"],
    "k2_rows_real": ["sft_k2d.cu", "sft_k2d_large.cu", "sft_k2d.cuh", "sft_step_common.cuh", "sft_device.cuh", "sft_async.cuh",
                     "sft_internal.h"],
    "k2_rows_pair": ["sft_k2d_pair.cu", "sft_warpfft.cuh", "sft_step_common.cuh", "sft_device.cuh", "sft_async.cuh",
                     "sft_internal.h"],
    "k2_cols_warp": ["sft_k2d_colwarp.cu", "sft_warpfft.cuh", "sft_step_common.cuh", "sft_device.cuh",
                     "sft_async.cuh", "sft_internal.h"],
    "k2_cols_pipe": ["sft_k2d_pipe.cu", "sft_step_common.cuh", "sft_device.cuh", "sft_async.cuh", "sft_internal.h"],
}


def source_hash(kernel):
    """Hash of the sources a kernel is built from (a record taken on other sources is stale)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2511_22510_gb300", "csrc")
    for f in sorted(KERNEL_SOURCES[kernel]):
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(kernel_tag):
    """DRAM bytes per launch recorded by the ncu summary under profiles/, if it
    was taken on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        rec = json.load(open(path))
    except Exception:
        return None
    ent = rec.get(kernel_tag)
    if not ent or ent.get("source_hash") != source_hash(kernel_tag.split("_model")[0]):
        return None
    return ent.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                               parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        return float(json.load(open(path))["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------- oracle
ERR_STEPS = 100
ERR_R = 2


def oracle_threads(w, R, nsteps):
    """FP64 oracle on replicas 0..R-1 of the workload, one thread (one host core)
    per replica: returns (final fields, the seconds one replica took, the FP32
    initial fields).  ctypes releases the GIL inside the C oracle."""
    import oracle
    oracle.build()
    f0 = W.initial_fields(w, replicas=R).astype(np.float32)
    out, secs = [None] * R, [0.0] * R

    def one(r):
        o = oracle.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, replica0=r)
        o.set_field(0, f0[r].astype(np.float64))
        t0 = time.perf_counter()
        o.step(nsteps)
        secs[r] = time.perf_counter() - t0
        out[r] = o.field(0)

    th = [threading.Thread(target=one, args=(r,)) for r in range(R)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    return out, max(secs), f0


def _oracle_worker(job):
    """One host process of the all-core oracle run: steps one replica of the
    workload (replica offset `rep`), timed after a shared barrier."""
    (cfg, rep, nsteps, barrier) = job
    import oracle
    w = W.model_b_1024(**cfg)
    f0 = W.initial_fields(w, replicas=1, seed_offset=rep)[0].astype(np.float64)
    o = oracle.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias, replica0=rep)
    o.set_field(0, f0)
    barrier.wait()
    t0 = time.perf_counter()
    o.step(nsteps)
    return time.perf_counter() - t0


def host_cpu():
    """Model name and logical core count of this host."""
    model = ""
    try:
        with open("/proc/cpuinfo") as fh:
            for line in fh:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"model": model or "unknown", "logical_cores": os.cpu_count()}


def oracle_all_cores(w, nsteps=2):
    """The oracle as it stands on every host core: one spawned process per core,
    each stepping its own replica of the workload (independent replicas, so the
    cores share no work); throughput = all site-steps / the slowest process."""
    import multiprocessing as mp
    import oracle
    oracle.build()
    n = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    cfg = dict(n=list(w.n), scheme=w.scheme, h=w.h)
    with ctx.Manager() as man:
        bar = man.Barrier(n)
        with ctx.Pool(n) as pool:
            times = pool.map(_oracle_worker, [(cfg, r, nsteps, bar) for r in range(n)])
    el = max(times)
    return {"value": w.sites * n * nsteps / el / 1e9, "unit": UNIT, "cores": n, "kind": "oracle",
            "sample": "FP64 oracle, %d processes (one per host core), each %d steps of its own %dx%d replica"
                      % (n, nsteps, w.n[0], w.n[1]), "host": host_cpu()}


def cufft_comparison(w, R, K, stream):
    """Comparison column (not the product path): the same SETD1 step written
    with torch.fft (cuFFT R2C/C2R) and elementwise torch ops, noise from
    torch.randn without the Hermitian fix-up, on R replicas; Gsite-steps/s over K
    steps with CUDA events."""
    import torch
    nx, ny = w.n
    G, r, u, T = w.p[:4]
    dev = "cuda"
    kx = 2 * math.pi * torch.fft.rfftfreq(nx, d=w.dx[0], device=dev, dtype=torch.float64)
    ky = 2 * math.pi * torch.fft.fftfreq(ny, d=w.dx[1], device=dev, dtype=torch.float64)
    k2 = ky[:, None] ** 2 + kx[None, :] ** 2
    ix = torch.arange(nx // 2 + 1, device=dev)[None, :]
    iy = torch.fft.fftfreq(ny, d=1.0 / ny, device=dev).abs()[:, None]
    mask = ((3 * ix < nx) & (3 * iy < ny)).to(torch.float32)
    c = -G * k2 * (r + k2)
    ch = c * w.h
    f1 = torch.exp(ch)
    A = torch.where(c != 0, torch.expm1(ch) / torch.where(c != 0, c, torch.ones_like(c)), torch.full_like(c, w.h))
    D = G * T * k2
    two = 2 * ch
    phi1 = torch.where(two != 0, torch.expm1(two) / torch.where(two != 0, two, torch.ones_like(two)),
                       torch.ones_like(two))
    g = (nx * ny / (nx * w.dx[0])) ** 1.0 * torch.sqrt(2 * D * w.h * phi1)
    s_nl = (-G * u * k2).to(torch.float32) * mask
    f1, A, g = f1.to(torch.float32), A.to(torch.float32), (g / math.sqrt(2)).to(torch.float32)
    with torch.cuda.stream(stream):
        gen = torch.Generator(device=dev)
        gen.manual_seed(w.seed)
        phi = torch.fft.rfft2(0.01 * torch.randn(R, ny, nx, device=dev, generator=gen))

        def step(phi):
            psi = torch.fft.irfft2(phi * mask, s=(ny, nx))
            F = s_nl * torch.fft.rfft2(psi * psi * psi)
            eta = torch.complex(torch.randn(phi.shape, device=dev, generator=gen),
                                torch.randn(phi.shape, device=dev, generator=gen))
            return f1 * phi + A * F + g * eta

        for _ in range(5):
            phi = step(phi)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(K):
            phi = step(phi)
        b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    return {"value": w.sites * R * K / (ms * 1e-3) / 1e9, "unit": UNIT, "replicas": R, "steps": K,
            "form": "torch.fft (cuFFT R2C/C2R) + elementwise torch ops, torch.randn noise; comparison only"}


def run_reference(args):
    """The oracle as it stands, on the host cores: each timed step is one FP64
    SETD step of one replica of the workload (a bounded sample), as many as fit
    in about a minute, with the S(k) observations the GPU arm takes in its
    timed region (one per OBS_EVERY steps, at least one)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build()
    w = workload(args)
    K = max(1, args.steps)
    n_obs, obs_every = observations(K)
    f0 = W.initial_fields(w, replicas=1)[0].astype(np.float32)
    o = oracle.Oracle(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias)
    o.set_field(0, f0.astype(np.float64))
    warm = 0
    t_warm = time.perf_counter()
    while warm < args.warmup and time.perf_counter() - t_warm < 30.0:  # warm-up steps, at most ~30 s
        o.step(1)
        warm += 1
    o.shells()
    times = []
    obs_done = 0
    t_start = time.perf_counter()
    for i in range(K):
        t0 = time.perf_counter()
        o.step(1)
        if (i + 1) % obs_every == 0 and obs_done < n_obs:
            o.shells()
            obs_done += 1
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > 60.0:
            break
    el = sum(times)
    value = w.sites * len(times) / el / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0, "steps": len(times),
        "warmup": warm, "ms_per_step": 1e3 * el / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(w, args.replicas, ws, K),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "FP64 serial oracle, %d single steps of one %dx%d replica with %d S(k) "
                                   "observations (the GPU arm runs %d replicas per step)"
                                   % (len(times), args.n, args.n, obs_done, args.replicas)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    import paper_2511_22510_gb300 as sft

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    w = workload(args)
    R = args.replicas
    stream = torch.cuda.Stream()
    g = sft.Stepper(w.d, w.n, w.dx, R, w.model, w.p, w.scheme, w.h, w.seed, stream=stream.cuda_stream,
                    replica0=rank_replica0(rank, R))
    f0 = W.initial_fields(w, replicas=R, seed_offset=rank).astype(np.float32)
    g.set_field(f0)
    ncols = sum(1 for c in range(w.n[0] // 2 + 1) if 3 * c < w.n[0])
    rows_b, cols_b = algorithmic_bytes(w, w.scheme, ncols)
    step_bytes_site = (rows_b + cols_b) / w.sites

    # one-time set-up, not a step: the schedule is autotuned and the step graph captured (state untouched);
    # then exactly the requested warm-up steps and one observation
    g.prepare()
    warm = max(args.warmup, 0)
    g.step(warm)
    g.observe(sft.SFT_OBS_SK)
    g.sync()
    K = max(args.steps, 1)
    # S(k) every OBS_EVERY steps inside the timed region, and at least once per timed region
    n_obs, obs_every = observations(K)
    l0 = sft.sft_kernel_launches(g.ctx)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        ev0.record(stream)
        done = obs_done = 0
        while done < K:
            n = min(obs_every, K - done)
            g.step(n)
            done += n
            if n == obs_every and obs_done < n_obs:
                g.observe(sft.SFT_OBS_SK)
                obs_done += 1
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    launches = sft.sft_kernel_launches(g.ctx) - l0
    ms_max = max_over_ranks(ms, dist)
    units = w.sites * R * K * ws
    value = units / (ms_max * 1e-3) / 1e9
    clocks = clk.summary()

    # per-kernel durations on the same stream (CUDA events around every launch)
    prof = sft.sft_profile(g.ctx, 50)
    plan = sft.sft_get_plan(g.ctx)
    row_kernel = "k2_rows_pair" if plan[0] == 3 else "k2_rows_real"
    col_kernel = "k2_cols_pipe" if plan[3] else ("k2_cols_warp" if plan[1] == 3 else "k2_cols_real")
    kern = [(row_kernel, prof[0], rows_b * R), (col_kernel, prof[1], cols_b * R)]
    dom = max(kern, key=lambda k: k[1])
    peak, peak_kind = measured_peak()
    achieved = dom[2] / (dom[1] * 1e-3) / 1e9
    tag = "%s_model_b_%d_R%d_%s" % (dom[0], w.n[0], R, scheme_name(w.scheme))
    traffic = profile_traffic(tag)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": dom[0], "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)",
                "alg_bytes_per_launch": dom[2], "launch_ms": dom[1],
                "kernels_ms": {k[0]: k[1] for k in kern}}
    step_achieved = step_bytes_site * value  # GB/s over the whole step
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": warm,
        "ms_per_step": ms_max / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic (seeded iid N(0, 0.01^2) fields, Philox noise)",
        "config": headline_config(w, R, ws, K),
        "roofline": roofline,
        "plan": dict(zip(("row_shape", "col_shape", "replicas_per_col_block", "pipelined_cols"), plan)),
        "step_roofline": {"bytes_per_site_step": step_bytes_site, "achieved_GBps": step_achieved,
                          "frac": step_achieved / peak,
                          "frac_at_24B_per_site": 24.0 * value / peak},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if rank == 0 and ws == 1 and not args.quick:
        # plain unbatched form: one replica, host-launched kernels, no graph
        p1 = sft.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, stream=stream.cuda_stream)
        p1.set_field(f0[:1])
        p1.step_plain(10)
        p1.sync()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        p1.step_plain(200)
        b.record(stream)
        torch.cuda.synchronize()
        plain = w.sites * 200 / (a.elapsed_time(b) * 1e-3) / 1e9
        p1.close()
        # the stated error of both forms: ERR_STEPS steps of ERR_R replicas against the FP64 oracle (one
        # oracle thread per replica; the serial oracle's time on one core is the CPU baseline)
        ofields, osec, of0 = oracle_threads(w, ERR_R, ERR_STEPS)
        errs = {}
        for form in ("batched", "plain"):
            chk = sft.Stepper(w.d, w.n, w.dx, ERR_R, w.model, w.p, w.scheme, w.h, w.seed, stream=stream.cuda_stream)
            chk.set_field(of0)
            (chk.step if form == "batched" else chk.step_plain)(ERR_STEPS)
            got = chk.field()
            chk.close()
            errs[form] = max(float(np.linalg.norm(got[r] - ofields[r]) / np.linalg.norm(ofields[r]))
                             for r in range(ERR_R))
        line["plain"] = {"value": plain, "unit": UNIT, "replicas": 1, "graph": False,
                         "batched_speedup": value / plain, "rel_l2_vs_fp64": errs["plain"]}
        line["cpu_baseline"] = {"value": w.sites * ERR_STEPS / osec / 1e9, "unit": UNIT, "cores": 1,
                                "kind": "oracle",
                                "sample": "FP64 serial oracle, %d steps of one %dx%d replica on one core (another "
                                          "replica on a second core at the same time)" % (ERR_STEPS, w.n[0], w.n[1])}
        line["error_vs_fp64"] = {"rel_l2_field": errs["batched"], "rel_l2_field_plain": errs["plain"],
                                 "steps": ERR_STEPS, "replicas": ERR_R, "tolerance": 1e-5,
                                 "note": "largest per-replica relative L2 of the real-space field"}
        line["cpu_baseline_all_cores"] = oracle_all_cores(w)
        # the batched path at other replica counts (R = 1: the state fits in L2)
        sweep = {}
        for Rs in (1, 16):
            gs = sft.Stepper(w.d, w.n, w.dx, Rs, w.model, w.p, w.scheme, w.h, w.seed, stream=stream.cuda_stream)
            gs.set_field(f0[:Rs])
            gs.step(64)
            gs.sync()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            gs.step(400)
            b.record(stream)
            torch.cuda.synchronize()
            sweep[str(Rs)] = w.sites * Rs * 400 / (a.elapsed_time(b) * 1e-3) / 1e9
            gs.close()
        sweep[str(R)] = value
        line["replica_sweep"] = {"unit": UNIT, "values": sweep,
                                 "note": "batched graph path, 400 steps without S(k); R = 1 is L2-resident"}
        line["cufft_comparison"] = cufft_comparison(w, R, 50, stream)
    # end to end through the public API with host buffers (every rank)
    pin = torch.from_numpy(f0).pin_memory()
    host_in = pin.numpy()
    chunks = 3
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    a.record(stream)
    for _ in range(chunks):
        sft.sft_set_field(g.ctx, -1, host_in)
        g.step(OBS_EVERY)
        sk = g.observe(sft.SFT_OBS_SK)
    b.record(stream)
    barrier()
    te = max_over_ranks(a.elapsed_time(b), dist)
    e2e_val = w.sites * R * ws * OBS_EVERY * chunks / (te * 1e-3) / 1e9
    line["e2e"] = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": f0.nbytes / OBS_EVERY,
                   "d2h_bytes_per_step": sk.nbytes / OBS_EVERY,
                   "note": "per chunk of 100 steps: set_field of all R fields from pinned host memory, "
                           "the steps, S(k) back to the host"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.close()
    if dist is not None:
        dist.destroy_process_group()


def run_other(args):
    """Throughput of the other workloads (one GPU): batched/graph path against the
    plain form (one replica or one member at a time, host-launched, no graph)."""
    import torch
    import paper_2511_22510_gb300 as sft
    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    K = max(args.steps // 10, 20)

    def timed(fn):
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b)

    line = {"metric": METRIC, "unit": UNIT, "n_gpus": 1, "steps": K, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic", "vs_baseline": None}
    if args.workload == "sde0d":
        # 0-d SDE ensemble of Sec. III: GBM (lambda = 2, mu = 1, delta = 1), SETD-Milstein, h = 2^-8, FP64
        S, p, h = 1 << 22, [2.0, 1.0, 1.0], 2.0 ** -8
        u = torch.ones(S, dtype=torch.float64, device="cuda")
        sft.sft_sde0d(1, p, sft.SFT_SDE_SETD_MILSTEIN, h, 16, u.data_ptr(), S, seed=9, stream=stream.cuda_stream)
        ms = timed(lambda: sft.sft_sde0d(1, p, sft.SFT_SDE_SETD_MILSTEIN, h, K, u.data_ptr(), S, seed=9, step0=16,
                                         stream=stream.cuda_stream))
        line.update({"metric": "Gpath-steps/s, 0-d SDE ensemble", "unit": "Gpath-steps/s", "dtype": "f64",
                     "value": S * K / (ms * 1e-3) / 1e9, "ms_per_step": ms / K,
                     "config": {"workload": "sde0d", "problem": "GBM lambda=2 mu=1 delta=1", "scheme": "SETD-Milstein",
                                "paths": S, "h": h}})
        print(json.dumps(line), flush=True)
        return
    if args.workload == "dynamics":
        # C(k, omega), chi(k, omega) and the FDT deviation (App. C) on Model A 256^2 x 64 (the paper's FDT set-up)
        import time
        w = W.model_a_64(n=[256, 256], replicas=64, h=0.01)
        g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, stream=stream.cuda_stream)
        g.init_random(0.1)
        g.step(64)
        g.sync()
        ms_plain = timed(lambda: g.step(256))
        M = 256
        sft.sft_dyn_start(g.ctx, M, 1)
        ms_rec = timed(lambda: g.step(M))
        nm = (w.n[0] // 2 + 1) * w.n[1]
        t0 = time.perf_counter()
        _, _, dbar = sft.sft_dyn_result(g.ctx, nm, M)
        ms_res = (time.perf_counter() - t0) * 1e3
        g.close()
        sites = w.sites * w.replicas
        line.update({"value": sites * M / (ms_rec * 1e-3) / 1e9, "ms_per_step": ms_rec / M, "steps": M,
                     "config": {"workload": "dynamics", "lattice": "256x256", "replicas": w.replicas, "M": M,
                                "every": 1, "model": "Model A"},
                     "plain": {"value": sites * 256 / (ms_plain * 1e-3) / 1e9, "unit": UNIT,
                               "form": "the same stepper without recording"},
                     "result_ms": ms_res, "fdt_dbar": dbar})
        print(json.dumps(line), flush=True)
        return
    if args.workload == "kpz_ensemble":
        lengths = W.kpz_ensemble_lengths()
        counts = {L: lengths.count(L) for L in sorted(set(lengths))}
        members = [W.kpz_1d(L, replicas=c) for L, c in counts.items()] + [W.kpz_2d(replicas=64)]
        cfgs = [sft.make_config(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, w.dealias,
                                stream=stream.cuda_stream) for w in members]
        sites = sum(w.sites * w.replicas for w in members)
        batch = sft.Batch(cfgs)
        batch.step(32)
        batch.sync()
        ms = timed(lambda: batch.step(K))
        value = sites * K / (ms * 1e-3) / 1e9
        prof = sft.sft_profile(batch.ctx, 10)
        batch.close()
        singles = [sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed,
                               stream=stream.cuda_stream) for w in members]
        for g in singles:
            g.step_plain(2)
        Kp = max(K // 4, 5)

        def plain_all():
            for g in singles:
                g.step_plain(Kp)
        msp = timed(plain_all)
        plain = sites * Kp / (msp * 1e-3) / 1e9
        for g in singles:
            g.close()
        line.update({"value": value, "ms_per_step": ms / K,
                     "config": {"workload": "kpz_ensemble", "members": {str(L): c for L, c in counts.items()},
                                "plus": "64 x 256^2", "note": "lines up to 16384 points in one persistent launch; 32768 and 65536 points and the 2-D members each on a parallel graph branch"},
                     "batched_kernels_ms": {"k1_batch": prof[0], "other_members": prof[1]},
                     "plain": {"value": plain, "unit": UNIT, "batched_speedup": value / plain,
                               "form": "each member's own kernels launched from the host, no graph"}})
    else:
        noise_space = 0
        if args.workload == "model_a_64":
            w = W.model_a_64(replicas=1024)
        elif args.workload == "model_b_1024_phase_shift":
            w = W.model_b_1024(replicas=64, dealias=2)
        elif args.workload == "model_b_768":
            w = W.model_b_1024(n=[768, 768], replicas=64)
        elif args.workload == "model_b_1024_real_space_noise":
            w = W.model_b_1024(replicas=64)
            noise_space = 1
        elif args.workload == "cgl_2048":
            w = W.cgl_2048(replicas=4)
        else:
            w = W.model_a_128_3d(replicas=32)
        prec = args.precision if args.workload == "cgl_2048" else 0
        g = sft.Stepper(w.d, w.n, w.dx, w.replicas, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                        stream=stream.cuda_stream, noise_space=noise_space, precision=prec)
        g.init_random(max(w.sigma0, 0.1))
        if args.workload == "model_a_128_3d_tangent":
            seed = torch.zeros((w.replicas,) + w.shape, dtype=torch.float32, device="cuda")
            seed[..., 1] = 1.0
            torch.cuda.synchronize()
            sft.sft_tangent_step(g.ctx, seed.data_ptr(), 4, None)
            ms = timed(lambda: sft.sft_tangent_step(g.ctx, None, K, None))
        else:
            g.step(32)
            g.sync()
            ms = timed(lambda: g.step(K))
        value = w.sites * w.replicas * K / (ms * 1e-3) / 1e9
        prof = sft.sft_profile(g.ctx, 10)
        g.close()
        p1 = sft.Stepper(w.d, w.n, w.dx, 1, w.model, w.p, w.scheme, w.h, w.seed, dealias=w.dealias,
                         stream=stream.cuda_stream, noise_space=noise_space, precision=prec)
        p1.init_random(0.1)
        p1.step_plain(2)
        msp = timed(lambda: p1.step_plain(K))
        plain = w.sites * K / (msp * 1e-3) / 1e9
        p1.close()
        line.update({"value": value, "ms_per_step": ms / K,
                     "config": {"workload": args.workload, "lattice": "x".join(str(n) for n in w.n),
                                "replicas": w.replicas, "scheme": scheme_name(w.scheme), "h": w.h,
                                "dealias": {0: "none", 1: "2/3 truncation", 2: "phase shifts"}[w.dealias],
                                "noise": "real space + FFT" if noise_space else "Fourier space",
                                "transforms": "split-BF16x3 tensor cores (precision study)" if prec else "FP32"},
                     "kernels_ms": list(map(float, prof)),
                     "plain": {"value": plain, "unit": UNIT, "replicas": 1, "graph": False,
                               "batched_speedup": value / plain}})
        if args.workload == "cgl_2048" and not prec and w.n[0] in (1024, 2048) and w.dealias == 1:
            # the warp row and column passes (both lines of 1024 or 2048 points under 2/3 truncation)
            rb, cb = algorithmic_bytes_complex(w.n[0], w.n[1], w.scheme, w.dealias)
            line["roofline"] = hbm_roofline("k2c_cols_warp", cb * w.replicas, float(prof[1]))
            line["roofline"]["traffic"] = None
            line["roofline_row_pass"] = hbm_roofline("k2c_rows_warp", rb * w.replicas, float(prof[0]))
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "model_b_1024":
        run_other(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
