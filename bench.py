#!/usr/bin/env python3
"""Benchmark of the GP-MPPI rollout (one "step" = one mppi_step: every
sample's rollout, costs, weights and the control update) on the K=4096, T=50,
N=500, 16-obstacle figure-eight workload.

Prints ONE JSON line (rank 0).  Metric: rollout sample-steps/s (K*T per
mppi_step) with the p50 mppi_step latency alongside.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (launched by torchrun) every rank runs an independent replica of
the controller with its own seed (the method has no exchange step between
controllers); value = all ranks' sample-steps / the slowest rank's time.
--impl reference times the FP64 oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import shutil
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "rollout sample-steps/s and p50 mppi_step latency vs plain FP32 GPU path"
WORKLOAD = "cfg2"
L2_FLUSH_BYTES = 512 << 20
CSRC = os.path.join(ROOT, "paper_2411_03289_gb300", "csrc")
PROFILES = os.path.join(ROOT, "profiles")


def rollout_flops_per_sample_step(N, O, S):
    """Algorithmic FP32 flops of one sample-step (exps counted separately):
    triangular quadratic form N(N+1) (N(N+1)/2 multiply-adds), 16N for the
    kernel row (4 differences, 4 squares-and-adds), the two means and the
    sum of squares, 15 per obstacle, 10 per lane segment, 150 for the
    dynamics, covariance and stage cost."""
    return N * (N + 1) + 16 * N + 15 * O + 10 * S + 150


def fp32_peak_tflops(sm_mhz=2070.0, n_sm=152):
    """FP32 FMA pipe from unit counts: 128 lanes per SM, 2 flops per FMA (the
    fallback when the probe cannot run)."""
    return n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12


def measure_alu_peaks(gp, dev, stream):
    """Measured throughput of the FP32 FMA pipe (scalar and packed f32x2 FMA)
    and of the SFU's ex2 on this GPU: the library's probe kernels, timed
    with CUDA events on the launch stream after a warm-up launch, with the
    SM clock sampled while they run."""
    import torch
    n_sm = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks = 8 * n_sm
    out = torch.empty(blocks * 256, dtype=torch.float32, device=dev)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    res = {}
    clocks.begin()
    for kind, name, iters in ((0, "fma", 600_000), (1, "fma_x2", 600_000), (2, "ex2", 60_000)):
        gp.gpmppi_alu_probe(kind, blocks, 1000, out, stream)       # warm-up
        ms = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gp.gpmppi_alu_probe(kind, blocks, iters, out, stream)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        ops = blocks * 256 * iters * 16
        res[name] = ops / (min(ms) / 1e3)
    clocks.end()
    clk = clocks.stop()
    fma = max(res["fma"], res["fma_x2"])
    return {"fp32_tflops": 2.0 * fma / 1e12,
            "fp32_scalar_tflops": 2.0 * res["fma"] / 1e12,
            "fp32_packed_x2_tflops": 2.0 * res["fma_x2"] / 1e12,
            "ex2_gops": res["ex2"] / 1e9,
            "sm_mhz": clk["sm_mhz"] if clk else None,
            "how": f"probe kernels ({blocks} CTAs x 256 threads x 16 independent chains), best of 3, "
                   "CUDA events; FMA counted as 2 flops"}


def alu_roof(achieved, peaks, kernel, traffic, note_extra=""):
    """Roofline entry for a kernel bound by the FP32 FMA pipe."""
    if peaks:
        peak, note = peaks["fp32_tflops"], "measured FP32 FMA probe (faster of scalar and packed f32x2)"
    else:
        peak, note = fp32_peak_tflops(2070.0), "FP32 FMA pipe 152 SM x 128 lanes x 2 flops x 2070 MHz (derived)"
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "kernel": kernel, "traffic": traffic, "peak_note": note + note_extra}


PRECISIONS = {"fp32": 0, "bf16split": 1, "fp16split": 2, "bf16split3": 3}


def measured_tensor_peak():
    """Dense 16-bit tensor peak: the measured BF16 burst figure (FP16 has the
    same nominal rate), else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            v = float(json.load(fh)["bf16_tflops"])
        return v, "measured BF16 dense burst (cuBLAS), same nominal rate for FP16"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s BF16 dense"


def describe(sc):
    P = sc.params
    prec = {v: k for k, v in PRECISIONS.items()}[P.precision]
    return {"workload": f"{sc.name}: K={P.K} T={P.T} N={sc.N} obstacles={sc.obstacles.shape[0]} "
                        f"path={sc.meta.get('path')} ({sc.path.shape[0]} vertices), {prec}",
            "K": P.K, "T": P.T, "N": sc.N, "obstacles": int(sc.obstacles.shape[0]),
            "path_vertices": int(sc.path.shape[0]), "precision": prec,
            "variance_mode": "per_sample",
            "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"}


# ---------------------------------------------------------------------------
# distributed plumbing
# ---------------------------------------------------------------------------

def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def slowest_rank(*values):
    """Element-wise maximum over all ranks of this rank's per-rank figures
    (times): the replicas are independent, so the job takes as long as its
    slowest rank.  Without a process group the values come back unchanged.
    Under NCCL the reduction runs on the current CUDA device, under gloo on
    the CPU."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return tuple(float(v) for v in values)
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return tuple(float(x) for x in t.tolist())


def replica_throughput(units_per_rank, seconds_per_rank):
    """Whole-job throughput of independent replicas (no data-path
    collective): the units all ranks processed over the slowest rank's time.
    Returns (throughput, slowest time)."""
    import torch.distributed as dist
    ws = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    (t,) = slowest_rank(seconds_per_rank)
    return units_per_rank * ws / t, t


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock and throttle-reason samples, each stamped with the host
    time at which it was read, so that the rows of the timed region can be
    picked out.  start() waits (bounded) until the first row arrives: the tool
    takes a while to come up, longer than a short timed region lasts."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.rows = []
        self.window = None
        self._thread = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append((time.perf_counter(), parts))

    def start(self, wait_s=5.0):
        import threading
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True, bufsize=1)
        except Exception:
            self.proc = None
            return
        self._thread = threading.Thread(target=self._read, daemon=True)
        self._thread.start()
        t0 = time.perf_counter()
        while not self.rows and time.perf_counter() - t0 < wait_s and self.proc.poll() is None:
            time.sleep(0.01)

    def begin(self):
        self.window = [time.perf_counter(), None]

    def end(self):
        if self.window is not None:
            self.window[1] = time.perf_counter()

    def in_window(self):
        if self.window is None or self.window[1] is None:
            return 0
        return sum(1 for t, _ in self.rows if self.window[0] <= t <= self.window[1])

    def stop(self, extra=None):
        """Statistics of the rows inside the timed window; with fewer than 3
        there, also those of `extra` = (t0, t1), a stretch of the same
        untimed work run right after it.  None without nvidia-smi."""
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self._thread is not None:
            self._thread.join(timeout=2)
        w0, w1 = self.window if self.window else (0.0, float("inf"))
        timed = [r for t, r in self.rows if w0 <= t <= w1]
        rows, where = timed, "timed region"
        if len(timed) < 3 and extra is not None:
            rows = timed + [r for t, r in self.rows if extra[0] <= t <= extra[1]]
            where = "timed region and the same steps run untimed right after it"
        if not rows:
            return None

        def num(v):
            try:
                return float(v)
            except ValueError:
                return None
        sm = [x for x in (num(r[1]) for r in rows) if x is not None]
        mx = [x for x in (num(r[2]) for r in rows) if x is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows),
                "samples_in_timed_region": len(timed), "window": where,
                "period_ms": self.PERIOD_MS}


# ---------------------------------------------------------------------------
# measured DRAM traffic of the rollout kernel (from the committed ncu summary)
# ---------------------------------------------------------------------------

def committed_traffic(kernel="rollout_fp32", workload=WORKLOAD):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if it was taken on the current sources: the summary records the
    sha256 of the kernel's .cu file and of every other source it names, and
    each must match the file as it is now; else None."""
    try:
        txt = open(os.path.join(PROFILES, f"{kernel}_{workload}_ncu.md")).read()
    except OSError:
        return None
    shas = dict(re.findall(r"^([A-Za-z0-9_.]+\.(?:cu|cuh)) sha256:\s*([0-9a-f]{64})", txt, re.M))
    if f"{kernel}.cu" not in shas:
        return None
    for name, want in shas.items():
        try:
            have = hashlib.sha256(open(os.path.join(CSRC, name), "rb").read()).hexdigest()
        except OSError:
            return None
        if have != want:
            return None
    m_tr = re.search(r"dram bytes per launch \(full workload\):\s*([0-9.eE+]+)", txt)
    return float(m_tr.group(1)) if m_tr else None


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, in a spawned process
# ---------------------------------------------------------------------------

CPU_SAMPLE_ROWS = 512


def _cpu_child(rows, reps, workload=WORKLOAD):
    import numpy as np  # noqa: F401
    import oracle as O
    import scenarios as S
    if workload.endswith("-terrain3"):
        sc = S.terrain_scenario(workload[:-len("-terrain3")], M=3)
    else:
        sc = S.scenario(workload)
    fits = O.fit_scenario(sc)
    samples = list(range(rows))
    t0 = time.perf_counter()
    for r in range(reps):
        O.rollout(sc, fits, sc.x0, sc.U0, r, samples=samples)
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "sample_steps": rows * sc.params.T * reps, "T": sc.params.T}))


def cpu_baseline(rows=CPU_SAMPLE_ROWS, reps=8, workload=WORKLOAD, threads=None, single_core=True):
    """The oracle on the host cores (BLAS threads = all cores, or `threads`),
    in a spawned process; with single_core, also a smaller sample on one
    BLAS thread (taskset to one core where available)."""
    cores = threads or os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    env.pop("CUDA_VISIBLE_DEVICES", None)
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-child", str(rows), str(reps), workload]
    if threads == 1 and shutil.which("taskset"):
        cmd = ["taskset", "-c", "0"] + cmd
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    if out.returncode != 0 or not line:
        return {"value": None, "unit": "sample-steps/s", "cores": cores, "kind": "oracle",
                "sample": f"failed: {out.stderr.strip()[-200:]}"}
    d = json.loads(line[-1])
    res = {"value": d["sample_steps"] / d["seconds"], "unit": "sample-steps/s", "cores": cores,
           "kind": "oracle",
           "sample": f"FP64 numpy oracle, {rows} of the K samples x T={d['T']} steps x {reps} iterations "
                     f"({d['seconds']:.1f} s), BLAS threads = {cores}"}
    if single_core and threads is None:
        one = cpu_baseline(rows=max(16, rows // 8), reps=2, workload=workload, threads=1, single_core=False)
        res["single_core"] = {k: one[k] for k in ("value", "unit", "cores", "sample")}
    return res


# ---------------------------------------------------------------------------
# the reference arm: the oracle, timed as it stands
# ---------------------------------------------------------------------------

def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle as O
    import scenarios as S
    sc = S.scenario(WORKLOAD)
    fits = O.gp_fit(sc.X, sc.Y, sc.hyper)
    rows = list(range(args.ref_rows))
    for w in range(args.warmup):
        O.rollout(sc, fits, sc.x0, sc.U0, w, samples=rows)
    times = []
    for s in range(args.steps):
        t0 = time.perf_counter()
        ro = O.rollout(sc, fits, sc.x0, sc.U0, args.warmup + s, samples=rows)
        O.mppi_update(sc.U0, ro["u_tilde"], O.mppi_weights(ro["costs"], sc.params.lam))
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.ref_rows * sc.params.T * args.steps / tot
    cores = os.cpu_count() or 1
    cfg = describe(sc)
    line = {"metric": METRIC, "value": value, "unit": "sample-steps/s", "impl": "reference",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "p50_ms": 1e3 * statistics.median(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": "sample-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.ref_rows} of K={sc.params.K} samples per step, full T and N"},
            "e2e": {"value": value, "unit": "sample-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------

def timed_steps(gp, ctrl, x0, U, U_new, w, c, flush, stream, steps, warmup, barrier, clocks=None):
    """W warm-up steps, then `steps` mppi_steps each bracketed by CUDA events on
    the launch stream, with an L2 flush (untimed) between them.  The library's
    per-kernel profiling is off in the timed loop (its events would sit
    between the rollout and the update, and reading them synchronises every
    step); a second pass of min(steps, 100) steps with profiling on, after the
    timed loop, gives the rollout and update kernel times."""
    import torch
    gp.mppi_set_profiling(ctrl, False)
    if clocks is not None:
        clocks.start()
    for _ in range(warmup):
        gp.mppi_step(ctrl, x0, U, U_new, w, c)
        flush.fill_(1.0)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    barrier()
    torch.cuda.synchronize()
    if clocks is not None:
        clocks.begin()
    t_wall = time.perf_counter()
    for i in range(steps):
        starts[i].record(stream)
        gp.mppi_step(ctrl, x0, U, U_new, w, c)
        ends[i].record(stream)
        flush.fill_(float(i))
    torch.cuda.synchronize()
    barrier()
    t_wall = time.perf_counter() - t_wall
    clk = None
    if clocks is not None:
        clocks.end()
        extra = None
        if clocks.in_window() < 3:
            # a timed region shorter than a few sampling periods: keep the same
            # steps running (untimed) until three more samples came in
            t0 = time.perf_counter()
            n0 = len(clocks.rows)
            while len(clocks.rows) < n0 + 3 and time.perf_counter() - t0 < 3.0:
                for _ in range(20):
                    gp.mppi_step(ctrl, x0, U, U_new, w, c)
                    flush.fill_(1.0)
                torch.cuda.synchronize()
            extra = (t0, time.perf_counter())
        clk = clocks.stop(extra)
    gp.mppi_device_status(ctrl)
    step_ms = [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)]
    # per-kernel times (events the library records around its launches)
    gp.mppi_set_profiling(ctrl, True)
    rollout_ms, update_ms = [], []
    for i in range(min(steps, 100)):
        gp.mppi_step(ctrl, x0, U, U_new, w, c)
        r_ms, u_ms = gp.mppi_last_profile(ctrl)
        rollout_ms.append(r_ms)
        update_ms.append(u_ms)
        flush.fill_(float(i))
    gp.mppi_set_profiling(ctrl, False)
    gp.mppi_device_status(ctrl)
    return step_ms, rollout_ms, update_ms, t_wall, clk


def fp32_path(args, gp, S, dev, flush, stream, barrier, peaks=None):
    """The plain FP32 CUDA-core path on the same workload, for comparison."""
    import numpy as np
    import torch
    sc = S.scenario(args.workload, seed=1, precision=0)
    g = gp.gp_fit(sc.X, sc.Y, sc.hyper)
    ctrl = gp.mppi_create(sc.params, sc.obstacles, sc.path, g)
    U = torch.tensor(sc.U0, dtype=torch.float32, device=dev)
    U_new = torch.empty_like(U)
    w = torch.empty(sc.params.K, dtype=torch.float32, device=dev)
    c = torch.empty_like(w)
    gp.mppi_set_profiling(ctrl, True)
    steps = max(10, args.steps // 4)
    step_ms, rollout_ms, _, _, _ = timed_steps(gp, ctrl, sc.x0.astype(np.float32), U, U_new, w, c, flush,
                                               stream, steps, args.warmup, barrier)
    P = sc.params
    S_seg = max(sc.path.shape[0] - 1, 1)
    flops = rollout_flops_per_sample_step(sc.N, sc.obstacles.shape[0], S_seg) * P.K * P.T
    r_avg = sum(rollout_ms) / len(rollout_ms)
    ach = flops / (r_avg / 1e3) / 1e12
    roof = alu_roof(ach, peaks, "k_rollout_fp32", committed_traffic("rollout_fp32", args.workload))
    if peaks:
        # the kernel rows' exponentials: N per sample-step on the SFU
        ex2 = sc.N * P.K * P.T / (r_avg / 1e3) / 1e9
        roof["sfu"] = {"achieved_gops": ex2, "peak_gops": peaks["ex2_gops"], "frac": ex2 / peaks["ex2_gops"]}
    return {"value": P.K * P.T * steps / (sum(step_ms) / 1e3), "unit": "sample-steps/s",
            "p50_ms": statistics.median(step_ms), "steps": steps, "rollout_ms": r_avg,
            "roofline": roof}


def _tc_leg(args, gp, dev, flush, stream, barrier, sc, ctrl, flops, profile_key, steps):
    """A few timed mppi_steps of a tensor-core workload: the leg's entry of the
    bench line (throughput, latency, kernel times, tensor roofline)."""
    import numpy as np
    import torch
    P = sc.params
    U = torch.tensor(sc.U0, dtype=torch.float32, device=dev)
    U_new = torch.empty_like(U)
    w = torch.empty(P.K, dtype=torch.float32, device=dev)
    c = torch.empty_like(w)
    gp.mppi_set_profiling(ctrl, True)
    step_ms, rollout_ms, update_ms, _, _ = timed_steps(gp, ctrl, sc.x0.astype(np.float32), U, U_new, w, c,
                                                       flush, stream, steps, 3, barrier)
    r_avg = sum(rollout_ms) / len(rollout_ms)
    ach = flops / (r_avg / 1e3) / 1e12
    peak, note = measured_tensor_peak()
    kind = gp.mppi_rollout_kind(ctrl)
    return {"value": P.K * P.T * steps / (sum(step_ms) / 1e3),
            "unit": "sample-steps/s", "steps": steps, "warmup": 3, "p50_ms": statistics.median(step_ms),
            "kernel_ms": {"rollout_avg": r_avg, "update_avg": sum(update_ms) / len(update_ms)},
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                         "frac": ach / peak, "peak_note": note,
                         "kernel": "k_rollout_mma" if kind == gp.GPMPPI_KERNEL_TC_STREAM else str(kind),
                         "traffic": committed_traffic("rollout_mma", profile_key)}}


def cfg3_leg(args, gp, S, dev, flush, stream, barrier, precision="fp16split"):
    """Secondary leg: the K=16384, T=100, N=2048, 64-obstacle workload on the
    streaming tensor-core rollout (FP16 split, or the three-term BF16 split),
    a few timed mppi_steps."""
    sc = S.scenario("cfg3", seed=1, precision=PRECISIONS[precision])
    g = gp.gp_fit(sc.X, sc.Y, sc.hyper)
    ctrl = gp.mppi_create(sc.params, sc.obstacles, sc.path, g)
    S_seg = max(sc.path.shape[0] - 1, 1)
    flops = rollout_flops_per_sample_step(sc.N, sc.obstacles.shape[0], S_seg) * sc.params.K * sc.params.T
    leg = _tc_leg(args, gp, dev, flush, stream, barrier, sc, ctrl, flops,
                  "cfg3" if precision == "fp16split" else f"cfg3-{precision}", max(5, args.steps // 40))
    return {"workload": describe(sc)["workload"], **leg}


def terrain_leg(args, gp, S, dev, flush, stream, barrier):
    """Secondary leg: cfg2 with three terrain GPs of N = 500 mixed by Eq. 3, on
    the streaming tensor-core rollout over the GPs' stacked factors (FP16
    split), a few timed mppi_steps; flops summed over the GPs."""
    sc = S.terrain_scenario("cfg2", M=3, seed=1, precision=PRECISIONS["fp16split"])
    gps = [gp.gp_fit(X, Y, h) for X, Y, h in sc.terrains]
    ctrl = gp.mppi_create_ensemble(sc.params, sc.obstacles, sc.path, gps, sc.terrain_w)
    S_seg = max(sc.path.shape[0] - 1, 1)
    flops = sum(rollout_flops_per_sample_step(X.shape[0], sc.obstacles.shape[0], S_seg)
                for X, _, _ in sc.terrains) * sc.params.K * sc.params.T
    leg = _tc_leg(args, gp, dev, flush, stream, barrier, sc, ctrl, flops, "cfg2-terrain3", max(10, args.steps // 5))
    return {"workload": f"cfg2-terrain3: K={sc.params.K} T={sc.params.T} three terrain GPs of N=500 mixed by "
                        f"Eq. 3 (w={sc.terrain_w}), fp16split", **leg}


def cfg5_leg(args, gp, S, dev):
    """Secondary leg: 64 independent controllers (K 1024..16384, T 20..100,
    N 200..4096, FP16 split) advanced by one CUDA-graph replay of the batched
    step (one persistent rollout launch over the work queue, one update
    launch), after the per-shape autotuner; a few timed replays."""
    import torch
    scs = S.batched_scenarios(64)
    for sc in scs:
        sc.params.precision = PRECISIONS["fp16split"]
    t_fit = time.perf_counter()
    gps = [gp.gp_fit(sc.X, sc.Y, sc.hyper) for sc in scs]
    ctrls = [gp.mppi_create(sc.params, sc.obstacles, sc.path, g) for sc, g in zip(scs, gps)]
    batch = gp.mppi_batch_create(ctrls)
    for i, sc in enumerate(scs):
        batch.state[i].copy_(torch.tensor(sc.x0, dtype=torch.float32))
        batch.U_nom[i].copy_(torch.tensor(sc.U0, dtype=torch.float32))
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t_fit
    stream = torch.cuda.Stream()
    t_tune = time.perf_counter()
    gp.mppi_batch_autotune(batch, stream)
    t_tune = time.perf_counter() - t_tune
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    steps = 3
    with torch.cuda.stream(stream):
        for _ in range(2):
            gp.mppi_batch_graph(batch, stream)
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        for i in range(steps):
            starts[i].record(stream)
            gp.mppi_batch_graph(batch, stream)
            ends[i].record(stream)
            flush.fill_(float(i))
        stream.synchronize()
    step_ms = [a.elapsed_time(b_) for a, b_ in zip(starts, ends)]
    units = sum(sc.params.K * sc.params.T for sc in scs)
    flops = sum(rollout_flops_per_sample_step(sc.N, sc.obstacles.shape[0], max(sc.path.shape[0] - 1, 1))
                * sc.params.K * sc.params.T for sc in scs)
    peak, note = measured_tensor_peak()
    ach = flops / (statistics.median(step_ms) / 1e3) / 1e12
    layouts = [gp.mppi_batch_layout(batch, i)[0] for i in range(len(scs))]
    return {"workload": f"cfg5: 64 controllers, K {min(s.params.K for s in scs)}..{max(s.params.K for s in scs)}, "
                        f"T {min(s.params.T for s in scs)}..{max(s.params.T for s in scs)}, "
                        f"N {min(s.N for s in scs)}..{max(s.N for s in scs)}, fp16split, one graph replay per step",
            "value": units * steps / (sum(step_ms) / 1e3), "unit": "sample-steps/s", "steps": steps, "warmup": 2,
            "p50_ms": statistics.median(step_ms), "sample_steps_per_step": units,
            "threads_per_sample_chosen": {str(r): layouts.count(r) for r in sorted(set(layouts))},
            "fit_and_create_s": t_fit, "autotune_s": t_tune,
            "roofline": {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "kernel": "k_rollout_persistent", "traffic": None,
                         "peak_note": note + "; algorithmic flops of all controllers over the whole step"}}


def run_ours(args):
    import numpy as np
    import torch

    import paper_2411_03289_gb300 as gp
    import scenarios as S
    from paper_2411_03289_gb300 import build as B

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    terrain = args.workload.endswith("-terrain3")
    if terrain:
        # the terrain ensemble of Eq. 3 (three GPs mixed per step): the FP32
        # ensemble rollout, or in the split precisions the streaming
        # tensor-core rollout over the GPs' stacked factors
        sc = S.terrain_scenario(args.workload[:-len("-terrain3")], M=3, seed=1 + rank,
                                precision=PRECISIONS[args.precision])
        P = sc.params
        gps = [gp.gp_fit(X, Y, h) for X, Y, h in sc.terrains]
        ctrl = gp.mppi_create_ensemble(P, sc.obstacles, sc.path, gps, sc.terrain_w)
    else:
        kw = {"T": args.horizon} if args.horizon else {}
        if args.samples:
            kw["K"] = args.samples
        sc = S.scenario(args.workload, seed=1 + rank, precision=PRECISIONS[args.precision], **kw)
        P = sc.params
        g = gp.gp_fit(sc.X, sc.Y, sc.hyper)
        ctrl = gp.mppi_create(P, sc.obstacles, sc.path, g)
    U = torch.tensor(sc.U0, dtype=torch.float32, device=dev)
    U_new = torch.empty_like(U)
    w = torch.empty(P.K, dtype=torch.float32, device=dev)
    c = torch.empty_like(w)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    x0 = sc.x0.astype(np.float32)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    gp.mppi_set_profiling(ctrl, True)
    clocks = ClockSampler(torch.cuda.current_device())
    step_ms, rollout_ms, update_ms, t_wall, clk = timed_steps(gp, ctrl, x0, U, U_new, w, c, flush, stream,
                                                             args.steps, args.warmup, barrier, clocks)
    # whole-job throughput: every rank's sample-steps over the slowest rank's time
    value, tot_s = replica_throughput(P.K * P.T * args.steps, sum(step_ms) / 1e3)
    tot_ms = 1e3 * tot_s
    gp.mppi_set_profiling(ctrl, False)

    # ---- end to end through the ABI with host buffers -----------------------
    # mppi_step_host: U in from pinned host memory, the step, U_new back to the
    # host, one call that returns once U_new is there (the controller needs
    # U_new[0] on the host)
    U_host = torch.tensor(sc.U0, dtype=torch.float32).pin_memory()
    out_host = torch.empty_like(U_host).pin_memory()
    for _ in range(3):
        gp.mppi_step_host(ctrl, x0, U_host, out_host, stream=stream)
    barrier()
    e2e_s = 0.0
    for i in range(args.steps):
        flush.fill_(float(i))                # same cold-L2 condition as the device-timed loop
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gp.mppi_step_host(ctrl, x0, U_host, out_host, stream=stream)
        e2e_s += time.perf_counter() - t0
    (e2e_s,) = slowest_rank(e2e_s)
    h2d = U_host.numel() * 4 + 5 * 4
    d2h = out_host.numel() * 4

    S_seg = max(sc.path.shape[0] - 1, 1)
    if terrain:
        flops = sum(rollout_flops_per_sample_step(X.shape[0], sc.obstacles.shape[0], S_seg)
                    for X, _, _ in sc.terrains) * P.K * P.T
    else:
        flops = rollout_flops_per_sample_step(sc.N, sc.obstacles.shape[0], S_seg) * P.K * P.T
    r_avg = sum(rollout_ms) / len(rollout_ms)
    achieved = flops / (r_avg / 1e3) / 1e12
    kind = gp.mppi_rollout_kind(ctrl)
    src, kname = {gp.GPMPPI_KERNEL_FP32: ("rollout_fp32", "k_rollout_fp32"),
                  gp.GPMPPI_KERNEL_TC_STREAM: ("rollout_mma", "k_rollout_mma"),
                  gp.GPMPPI_KERNEL_TC_CLUSTER: ("rollout_cluster", "k_rollout_cl"),
                  gp.GPMPPI_KERNEL_ENSEMBLE: ("ensemble", "k_rollout_ens")}[kind]
    traffic = committed_traffic(src, args.workload)
    peaks = measure_alu_peaks(gp, dev, stream) if not args.no_alu_peaks else None
    if terrain and P.precision == 0:
        roof = alu_roof(achieved, peaks, "k_rollout_ens", traffic, "; flops summed over the three terrain GPs")
    elif P.precision == 0:
        roof = alu_roof(achieved, peaks, "k_rollout_fp32", traffic)
    else:
        peak, note = measured_tensor_peak()
        if terrain:
            note += "; flops summed over the three terrain GPs"
        roof = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "traffic": traffic, "kernel": kname, "peak_note": note}
        roof["frac"] = roof["achieved"] / roof["peak"]
    fp32 = None
    if P.precision != 0 and not terrain and not args.no_fp32_path:
        fp32 = fp32_path(args, gp, S, dev, flush, stream, barrier, peaks)
    legs = {}
    if args.workload == WORKLOAD and not terrain and not args.no_legs:
        legs["cfg3"] = cfg3_leg(args, gp, S, dev, flush, stream, barrier)
        legs["cfg3_bf16split3"] = cfg3_leg(args, gp, S, dev, flush, stream, barrier, "bf16split3")
        legs["cfg5"] = cfg5_leg(args, gp, S, dev)
        legs["cfg2_terrain3"] = terrain_leg(args, gp, S, dev, flush, stream, barrier)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "sample-steps/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "p50_ms": statistics.median(step_ms), "p90_ms": sorted(step_ms)[int(0.9 * (len(step_ms) - 1))],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f32", 1: "f32+bf16split", 2: "f32+f16split", 3: "f32+bf16split3"}[P.precision],
        "data": "synthetic (seeded GP training set, obstacles and figure-eight path)",
        "config": describe(sc) if not terrain else {
            **describe(sc), "workload": f"{sc.name}: K={P.K} T={P.T} three terrain GPs of N={sc.terrains[0][0].shape[0]} "
                                        f"mixed by Eq. 3 (w={sc.terrain_w}), obstacles={sc.obstacles.shape[0]}, "
                                        f"figure-eight, {args.precision}", "terrains": 3},
        "gpu_launches": 2 * args.steps,
        "kernel_ms": {"rollout_avg": r_avg, "update_avg": sum(update_ms) / len(update_ms)},
        "roofline": roof,
        "cpu_baseline": cpu_baseline(workload=args.workload) if (rank == 0 and ws == 1 and not args.no_cpu) else None,
        "e2e": {"value": P.K * P.T * args.steps * ws / e2e_s, "unit": "sample-steps/s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "clocks": clk,
        "fp32_path": fp32,
        "vs_plain_fp32_path": (value / (fp32["value"] * ws)) if fp32 else None,
        "alu_peaks": peaks,
        **legs,
        "wall_s_timed_region": t_wall,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


GRAD_SLOPE = 20.0
GRAD_CPU_ROWS = 4


def grad_flops_per_sample_step(N, O, S):
    """Algorithmic FP32 flops of the adjoint kernel per sample-step: the
    forward rollout (as above), the second triangular product b = L^-T v
    (N(N+1)), 60N for the GP adjoint row (kernel row, weights, z and
    lengthscale accumulators, the (dK/dl) alpha terms), 10 per lane segment
    and 30 per obstacle for the cost adjoint, 400 for the covariance and mean
    adjoints.  The recomputation of each checkpointed segment is not counted."""
    return rollout_flops_per_sample_step(N, O, S) + N * (N + 1) + 60 * N + 10 * S + 30 * O + 400


def _grad_cpu_child(rows):
    import numpy as np
    import oracle as O
    import scenarios as S
    sc = S.scenario("cfg4")
    U = sc.U0.copy()
    U[:, 1] = 0.4 * np.sin(np.arange(sc.params.T) / 6.0)
    t0 = time.perf_counter()
    O.fd_gradient(sc, sc.hyper, sc.x0, U, 0, list(range(rows)), GRAD_SLOPE, h_u=1e-3, h_l=1e-3)
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "sample_steps": rows * sc.params.T}))


def grad_cpu_baseline(rows=GRAD_CPU_ROWS):
    cores = os.cpu_count() or 1
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[k] = str(cores)
    cmd = [sys.executable, os.path.abspath(__file__), "--grad-cpu-child", str(rows)]
    out = subprocess.run(cmd, capture_output=True, text=True, env=env, cwd=ROOT, timeout=900)
    line = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    if out.returncode != 0 or not line:
        return {"value": None, "unit": "sample-steps/s", "cores": cores, "kind": "oracle",
                "sample": f"failed: {out.stderr.strip()[-200:]}"}
    d = json.loads(line[-1])
    return {"value": d["sample_steps"] / d["seconds"], "unit": "sample-steps/s", "cores": cores,
            "kind": "oracle",
            "sample": f"FP64 oracle gradient (central differences, h=1e-3, all 100 control and 8 "
                      f"lengthscale components) of the objective over {rows} of the K samples x T=50 "
                      f"({d['seconds']:.1f} s), BLAS threads = {cores}"}


def run_grad(args):
    """cfg4: one step = one mppi_grad call (smoothed cost J, dJ/dU (T x 2) and
    dJ/dl (2 x 4)) over all K samples."""
    import numpy as np
    import torch

    import paper_2411_03289_gb300 as gp
    import scenarios as S
    from paper_2411_03289_gb300 import build as B

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    kw = {"T": args.horizon} if args.horizon else {}
    if args.samples:
        kw["K"] = args.samples
    sc = S.scenario("cfg4", seed=1 + rank, **kw)
    P = sc.params
    g = gp.gp_fit(sc.X, sc.Y, sc.hyper)
    ctrl = gp.mppi_create(P, sc.obstacles, sc.path, g)
    U0 = sc.U0.copy()
    U0[:, 1] = 0.4 * np.sin(np.arange(P.T) / 6.0)
    U = torch.tensor(U0, dtype=torch.float32, device=dev)
    J = torch.empty(1, dtype=torch.float32, device=dev)
    dU = torch.empty(P.T, 2, dtype=torch.float32, device=dev)
    dl = torch.empty(2, 4, dtype=torch.float32, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    x0 = sc.x0.astype(np.float32)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def one():
        gp.mppi_grad(ctrl, x0, U, GRAD_SLOPE, None, J, dU, dl)

    for _ in range(args.warmup):
        one()
        flush.fill_(1.0)
    gp.mppi_set_profiling(ctrl, True)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    adj_ms, rest_ms = [], []
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        starts[i].record(stream)
        one()
        ends[i].record(stream)
        a_ms, r_ms = gp.mppi_last_profile(ctrl)
        adj_ms.append(a_ms)
        rest_ms.append(r_ms)
        flush.fill_(float(i))
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    gp.mppi_set_profiling(ctrl, False)
    step_ms = [a.elapsed_time(b_) for a, b_ in zip(starts, ends)]
    tot_ms = sum(step_ms)
    # end to end: controls in from pinned host memory, J and both gradients out
    U_host = torch.tensor(U0, dtype=torch.float32).pin_memory()
    out_host = torch.empty(1 + 2 * P.T + 8, dtype=torch.float32).pin_memory()
    e2e_s = 0.0
    for i in range(max(3, args.steps // 4) + 3):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        U.copy_(U_host, non_blocking=True)
        one()
        out_host[:1].copy_(J, non_blocking=True)
        out_host[1:1 + 2 * P.T].copy_(dU.view(-1), non_blocking=True)
        out_host[1 + 2 * P.T:].copy_(dl.view(-1), non_blocking=True)
        torch.cuda.synchronize()
        if i >= 3:
            e2e_s += time.perf_counter() - t0
    n_e2e = max(3, args.steps // 4)
    tot_ms, e2e_s = slowest_rank(tot_ms, e2e_s)
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    S_seg = max(sc.path.shape[0] - 1, 1)
    flops = grad_flops_per_sample_step(sc.N, sc.obstacles.shape[0], S_seg) * P.K * P.T
    a_avg = sum(adj_ms) / len(adj_ms)
    achieved = flops / (a_avg / 1e3) / 1e12
    peaks = measure_alu_peaks(gp, dev, stream) if not args.no_alu_peaks else None
    units = P.K * P.T
    line = {
        "metric": METRIC, "value": units * args.steps * ws / (tot_ms / 1e3), "unit": "sample-steps/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
        "p50_ms": statistics.median(step_ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded GP training set, obstacles, figure-eight path)",
        "config": {"workload": f"cfg4: K={P.K} T={P.T} N={sc.N} obstacles={sc.obstacles.shape[0]} figure-eight, "
                               f"gradient of the sigmoid-smoothed cost (slope {GRAD_SLOPE:g}) in U and the "
                               f"lengthscales, checkpoints every ceil(sqrt(T)) steps",
                   "K": P.K, "T": P.T, "N": sc.N, "obstacles": int(sc.obstacles.shape[0]),
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)"},
        "gpu_launches": 3 * args.steps,
        "kernel_ms": {"adjoint_avg": a_avg, "gram_trace_and_reduce_avg": sum(rest_ms) / len(rest_ms)},
        "roofline": alu_roof(achieved, peaks, "k_grad", committed_traffic("adjoint", "cfg4")),
        "alu_peaks": peaks,
        "cpu_baseline": grad_cpu_baseline() if (ws == 1 and not args.no_cpu) else None,
        "e2e": {"value": units * n_e2e * ws / e2e_s, "unit": "sample-steps/s",
                "h2d_bytes_per_step": U_host.numel() * 4 + 20, "d2h_bytes_per_step": out_host.numel() * 4},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_batched(args):
    """cfg5: 64 independent controllers (K, T, N, obstacles and paths all
    different) advanced together, one CUDA-graph replay per step."""
    import numpy as np
    import torch

    import paper_2411_03289_gb300 as gp
    import scenarios as S
    from paper_2411_03289_gb300 import build as B

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    B.build()
    dev = torch.device("cuda", torch.cuda.current_device())
    prec = PRECISIONS[args.precision]
    scs = S.batched_scenarios(args.batch, first_seed=args.batch * rank)
    for sc in scs:
        sc.params.precision = prec
    t_fit = time.perf_counter()
    gps = [gp.gp_fit(sc.X, sc.Y, sc.hyper) for sc in scs]
    ctrls = [gp.mppi_create(sc.params, sc.obstacles, sc.path, g) for sc, g in zip(scs, gps)]
    torch.cuda.synchronize()
    t_fit = time.perf_counter() - t_fit
    batch = gp.mppi_batch_create(ctrls)
    host_state = [torch.tensor(sc.x0, dtype=torch.float32).pin_memory() for sc in scs]
    host_U = [torch.tensor(sc.U0, dtype=torch.float32).pin_memory() for sc in scs]
    for i in range(len(scs)):
        batch.state[i].copy_(host_state[i])
        batch.U_nom[i].copy_(host_U[i])
    stream = torch.cuda.Stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    chosen = gp.mppi_batch_autotune(batch, stream)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            gp.mppi_batch_graph(batch, stream)
        stream.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        barrier()
        for i in range(args.steps):
            starts[i].record(stream)
            gp.mppi_batch_graph(batch, stream)
            ends[i].record(stream)
            flush.fill_(float(i))
        stream.synchronize()
        barrier()
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b_) for a, b_ in zip(starts, ends)]
        # end to end: every controller's state and controls in, results out
        outs = [torch.empty_like(u).pin_memory() for u in host_U]
        e2e_s = 0.0
        for i in range(args.steps):
            flush.fill_(float(i))
            stream.synchronize()
            t0 = time.perf_counter()
            for j in range(len(scs)):
                batch.state[j].copy_(host_state[j], non_blocking=True)
                batch.U_nom[j].copy_(host_U[j], non_blocking=True)
            gp.mppi_batch_graph(batch, stream)
            for j in range(len(scs)):
                outs[j].copy_(batch.U_new[j], non_blocking=True)
            stream.synchronize()
            e2e_s += time.perf_counter() - t0
    tot_ms = sum(step_ms)
    tot_ms, e2e_s = slowest_rank(tot_ms, e2e_s)
    units_step = sum(sc.params.K * sc.params.T for sc in scs)
    flops_step = sum(rollout_flops_per_sample_step(sc.N, sc.obstacles.shape[0], max(sc.path.shape[0] - 1, 1))
                     * sc.params.K * sc.params.T for sc in scs)
    value = units_step * args.steps * ws / (tot_ms / 1e3)
    peak, note = measured_tensor_peak()
    achieved = flops_step / (tot_ms / args.steps / 1e3) / 1e12
    if rank != 0:
        if ws > 1:
            torch.distributed.destroy_process_group()
        return
    line = {
        "metric": METRIC, "value": value, "unit": "sample-steps/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "p50_ms": statistics.median(step_ms),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {0: "f32", 1: "f32+bf16split", 2: "f32+f16split", 3: "f32+bf16split3"}[prec],
        "data": "synthetic (64 seeded controllers)",
        "config": {"workload": f"cfg5: {len(scs)} controllers, K {min(s.params.K for s in scs)}..{max(s.params.K for s in scs)}, "
                               f"T {min(s.params.T for s in scs)}..{max(s.params.T for s in scs)}, "
                               f"N {min(s.N for s in scs)}..{max(s.N for s in scs)}, one CUDA-graph replay per step",
                   "controllers": len(scs), "sample_steps_per_step": units_step,
                   "autotune_layouts_changed": chosen, "precision": args.precision,
                   "l2": f"flushed between timed steps ({L2_FLUSH_BYTES >> 20} MiB write)",
                   "fit_and_create_s": t_fit},
        "gpu_launches": 2 * args.steps,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "k_rollout_persistent",
                     "peak_note": note + "; whole batched step timed"},
        "cpu_baseline": None,
        "e2e": {"value": units_step * args.steps * ws / e2e_s, "unit": "sample-steps/s",
                "h2d_bytes_per_step": sum(4 * (5 + 2 * sc.params.T) for sc in scs),
                "d2h_bytes_per_step": sum(4 * 2 * sc.params.T for sc in scs)},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def main():
    if len(sys.argv) >= 2 and sys.argv[1] == "--cpu-child":
        _cpu_child(int(sys.argv[2]), int(sys.argv[3]), sys.argv[4] if len(sys.argv) > 4 else WORKLOAD)
        return
    if len(sys.argv) >= 2 and sys.argv[1] == "--grad-cpu-child":
        _grad_cpu_child(int(sys.argv[2]))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=400)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--ref-rows", type=int, default=128,
                    help="samples per reference (oracle) step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--workload", default=WORKLOAD, help="scenario name (cfg2 is the reported workload)")
    ap.add_argument("--precision", default="fp16split", choices=sorted(PRECISIONS))
    ap.add_argument("--batch", type=int, default=64, help="controllers in the cfg5 workload")
    ap.add_argument("--horizon", type=int, default=None,
                    help="override the workload's horizon T (short cases for profiler captures)")
    ap.add_argument("--samples", type=int, default=None,
                    help="override the workload's sample count K (small cases for profiler captures)")
    ap.add_argument("--no-alu-peaks", action="store_true", help="skip the FP32/SFU throughput probes")
    ap.add_argument("--no-legs", action="store_true", help="skip the secondary workload legs (cfg3, cfg5)")
    ap.add_argument("--no-fp32-path", action="store_true",
                    help="skip timing the plain FP32 CUDA-core path beside the headline path")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "cfg5":
        run_batched(args)
    elif args.workload == "cfg4":
        run_grad(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
