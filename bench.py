#!/usr/bin/env python3
"""Benchmark: domain-decomposed projective dynamics on the 390K-tet shell.

One step = one frame of the sweater-scale shell (325 x 100 x 2 hexes x 6 =
390,000 tets, 98,475 vertices, 200 domains), 20 PD iterations, dt = 1/150 s,
driven collar: inertia, then 20 x (fused local step and RHS assembly,
subspace solve), then the velocity update, all in libpdgb300's kernels.

Prints one JSON line.  `value` is PD iterations per second (whole job) of
the FP32 solve; `ms_per_step` is ms per frame.  The same line carries the
mixed-precision leg (BF16 matrices on the tensor cores in the correction
form), the frame-0 error of both against the FP64 oracle (computed on the
host cores meanwhile), the per-phase bytes and rates, the end-to-end rate
with host copies, the serving stream and the CPU baseline.  `--impl
reference` times the FP64 CPU oracle on the same workload instead (the
reference arm of this method).
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ms/frame and PD iters/s at 390K tets (FP32 vs mixed) at stated error; p99 frame latency; HBM GB/s"
UNIT = "PD iters/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--precision", choices=["fp32", "bf16", "tf32"], default="fp32")
    p.add_argument("--refine", type=int, default=0)
    p.add_argument("--correction", action="store_true",
                   help="solve each PD iteration for the correction b - K x (FP64 residual)")
    p.add_argument("--streaming", action="store_true",
                   help="the whole subspace solve as one cooperative streaming launch")
    p.add_argument("--modal", action="store_true",
                   help="the paper's own global step: normal modes per domain + Chebyshev-Jacobi sweeps")
    p.add_argument("--modes", type=int, default=20)
    p.add_argument("--sweeps", type=int, default=20)
    p.add_argument("--single-level", action="store_true",
                   help="one dense S^-1 for the interface instead of the two-level interface solve")
    p.add_argument("--iters", type=int, default=20, help="PD iterations per frame")
    p.add_argument("--small", action="store_true", help="small shell (profiling captures)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-serving", action="store_true",
                   help="skip the serving stream (64 Poisson requests, 5K-200K tets, 60 frames each)")
    p.add_argument("--serving-requests", type=int, default=64)
    p.add_argument("--serving-budget-gib", type=float, default=16.0)
    p.add_argument("--no-mixed", action="store_true",
                   help="skip the mixed-precision leg (BF16 matrices on the tensor cores, correction form)")
    p.add_argument("--no-oracle-check", action="store_true",
                   help="skip the frame-0 error of each precision against the FP64 oracle")
    return p.parse_args()


# traffic / algorithmic bytes of the kernel behind a phase, read from its ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum per launch), keyed by
# (phase, precision, interface solve); a kernel changed since its capture has no entry.
# ("dd_interior", fp32, two levels): the ncu capture of the interior k_axpy_tma launch on the
# 153,600-tet shell; the interior is one tile stream per domain, so the ratio carries over to the
# full-size launch.
# Thread instructions per tet and SIMT efficiency of the fused local step from its ncu capture
# (profiles/k_local_assemble_shell153k_fp32.md): its roofline is the issue rate, not HBM.
LOCAL_THREAD_INSTR_PER_TET, LOCAL_SIMT = 1052.0, 22.41
TRAFFIC_RATIO = {("dd_interior", "fp32", "two"): 0.9931, ("dd_interior", "bf16", "two"): 0.991}



def workload(small: bool):
    from workloads.meshes import sweater_shell
    if small:
        # 153,600 tets; interface ~6K vertices: S^-1 ~150 MB, still larger than L2
        return sweater_shell(n_theta=200, n_z=64, n_r=2, dom_theta=16, dom_z=5)
    return sweater_shell()


def dist_setup(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if _has_cuda() else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local


def _has_cuda():
    import torch
    return torch.cuda.is_available()


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def whole_job_rate(units_per_rank: int, local_ms: float, world: int) -> tuple:
    """(value, max_ms): units of all ranks / slowest rank's time (replicas: weak scaling)."""
    t = max_over_ranks(local_ms, world)
    return world * units_per_rank / (t / 1e3), t


def max_over_ranks(x: float, world: int) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if _has_cuda() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.dev = device_index
        # the clock samples are kept as evidence in $PD_RECORD_DIR (a temporary directory if unset)
        self.path = os.path.join(os.environ.get("PD_RECORD_DIR") or tempfile.gettempdir(),
                                 f"clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "20", "-i", str(self.dev)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self, begin: bool):
        """Host wall time of the timed region's start and end: samples outside it are not counted."""
        if begin:
            self.t0 = time.time()
        else:
            self.t1 = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        return self.summarize(self.path, getattr(self, "t0", None), getattr(self, "t1", None))

    @staticmethod
    def summarize(path, t0, t1):
        """Median SM clock, max clock and the throttle reasons seen in the samples of
        the timed window [t0, t1] (host wall time; all samples if none fall inside)."""
        import datetime
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except ValueError:
                continue
        inside = [r for r in rows if t0 is not None and t1 is not None and t0 - 0.05 <= r[0] <= t1 + 0.05]
        use = inside or rows
        sm = [r[1] for r in use]
        smax = [r[2] for r in use]
        reasons = set()
        for r in use:
            for n, v in zip(names, r[3]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "in_timed_window": bool(inside)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def host_info():
    """Host cores and CPU model (the CPU baseline's hardware)."""
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                low = line.lower()
                if low.startswith("model name") or low.startswith("cpu part") or low.startswith("hardware"):
                    model = line.split(":", 1)[1].strip()
                    if low.startswith("model name"):
                        break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu": model, "machine": platform.machine()}


_ORACLE_JOB = """
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
from bench import workload
from oracle.pd_oracle import PDOracle
w = workload({small!r})
o = PDOracle(w.rest, w.tets, w.pinned, w.gamma_s, w.gamma_v, w.density, w.dt)
x = w.rest.copy(); v = np.zeros_like(x)
y = o.inertial_target(x, v, w.gravity)
xp = w.pin_targets(0)
x = y.copy(); x[o.pin_ids] = xp
mode = {mode!r}
if mode == "frame":
    # frame 0 from rest with the benchmark's iterations: the FP64 reference of the accuracy check
    xo, _ = o.step(w.rest, np.zeros_like(w.rest), w.pin_targets(0), w.gravity, {iters})
    np.save({out!r}, xo)
    print(json.dumps({{"done": True}}))
else:
    t = time.perf_counter()
    for _ in range({n}):
        R, V = o.local(x)
        b = o.rhs(y, R, V)
        x[o.free] = o.global_solve(b, xp)
    dt = time.perf_counter() - t
    print(json.dumps({{"seconds": dt, "iters": {n}}}))
"""


class OracleJobs:
    """The FP64 oracle on the host cores, in child processes started before the
    first CUDA call and run one after the other in a background thread: the
    timed CPU baseline (3 PD iterations of frame 0, on one thread and on all
    cores) and the FP64 frame 0 that each precision's first frame is checked
    against."""

    def __init__(self, small: bool, iters: int, check: bool):
        import threading
        self.small, self.iters, self.check = small, iters, check
        self.results = {}
        self.out = os.path.join(tempfile.mkdtemp(prefix="pd_oracle_"), "frame0.npy")
        self.thread = threading.Thread(target=self._run, daemon=True)
        self.thread.start()

    def _one(self, mode, threads, n=3):
        code = _ORACLE_JOB.format(root=ROOT, small=self.small, mode=mode, iters=self.iters, out=self.out, n=n)
        env = dict(os.environ)
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
        env["CUDA_VISIBLE_DEVICES"] = ""
        try:
            r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=900)
        except subprocess.TimeoutExpired:
            return None, "timeout"
        if r.returncode != 0:
            return None, r.stderr[-400:]
        return json.loads(r.stdout.strip().splitlines()[-1]), None

    def _run(self):
        self.results["one_thread"] = self._one("sample", 1)
        self.results["all_cores"] = self._one("sample", os.cpu_count() or 1)
        if self.check:
            self.results["frame"] = self._one("frame", os.cpu_count() or 1)

    def join(self, timeout=600):
        self.thread.join(timeout)
        return self.results

    def frame0(self):
        import numpy as np
        d = self.results.get("frame", (None, "not run"))[0]
        return np.load(self.out) if d and os.path.exists(self.out) else None


def run_serving(args):
    """Serving stream: Poisson arrivals of garment requests of mixed sizes,
    continuous batching (admission in the background while resident requests
    advance).  Returns the per-request frame latency (wall time between a
    request's frames, every stall included) p50/p99, the GPU time of the
    batched frames, aggregate tets*iters/s over the wall time, and the same
    requests run one at a time on the single-mesh stepper (mesh set-up and
    prefactorisation included, as the server's wall time includes them)."""
    import numpy as np
    import torch

    from paper_2405_12484_gb300.sim import Mesh, Server
    from workloads.meshes import request_workload, serving_requests
    reqs = serving_requests(n_req=args.serving_requests)
    frames = 60
    works = []
    for arrival, gen, size, seed in reqs:
        w = request_workload(gen, size, seed, n_iter=20)
        drive = (0.2, 1.0, 0) if gen == "shell" else None
        works.append((arrival, w, drive))
    budget = int(args.serving_budget_gib * (1 << 30))
    S = Server(budget, max_slots=64, n_iter=20)
    t0 = time.perf_counter()
    subs, pending = [], list(works)        # subs: (request id, n_tets, arrival)
    gpu_ms, active_hist, tick_ms = [], [], []

    def unfinished():
        return any(S.poll(i)[0] in (0, 1) for i, _, _ in subs)

    while pending or unfinished():
        now = time.perf_counter() - t0
        while pending and pending[0][0] <= now:
            a, w, d = pending.pop(0)
            subs.append((S.submit(w, frames, d), w.n_t, a))
        t_tick = time.perf_counter()
        n, ms = S.tick()
        if n > 0:
            gpu_ms.append(ms)
            active_hist.append(n)
            tick_ms.append((time.perf_counter() - t_tick) * 1e3)
        elif pending and not subs:
            time.sleep(min(0.002, max(0.0, pending[0][0] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    lat, first = [], []
    failed = 0
    for i, _, _ in subs:
        if S.poll(i)[0] == 2:
            ms = S.fetch(i)[1].tolist()
            first.append(ms[0])
            lat.extend(ms[1:])
        else:
            failed += 1
    tet_iters = sum(nt for _, nt, _ in subs) * frames * 20
    stats = S.stats()
    S.close()
    # one at a time, plain single-mesh stepper (set-up and prefactorisation included)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    seq_gpu_ms = 0.0
    for _, w, d in works:
        m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density)
        m.set_materials(w.gamma_s, w.gamma_v)
        m.prefactor(w.dt)
        pins = [torch.as_tensor(w.pin_targets(n), dtype=torch.float32, device="cuda") for n in range(frames)] \
            if d is not None else [None] * frames
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for n in range(frames):
            m.step(pins[n], w.gravity, 20)
        e1.record()
        e1.synchronize()
        seq_gpu_ms += e0.elapsed_time(e1)
        m.close()
    wall_seq = time.perf_counter() - t1
    return {"requests": len(works), "failed": failed, "frames_per_request": frames, "pd_iters_per_frame": 20,
            "hbm_budget_gib": args.serving_budget_gib, "peak_budgeted_gib": stats["peak_bytes"] / (1 << 30),
            "frame_latency_ms": {"p50": pct(lat, 0.5), "p99": pct(lat, 0.99), "max": max(lat),
                                 "what": "per request, wall time between its consecutive frames (stalls included)"},
            "first_frame_latency_ms": {"p50": pct(first, 0.5), "p99": pct(first, 0.99), "max": max(first),
                                       "what": "per request, from the end of its admission to its first frame"},
            "batched_frame_gpu_ms": {"p50": pct(gpu_ms, 0.5), "p99": pct(gpu_ms, 0.99), "max": max(gpu_ms)},
            "tick_wall_ms": {"p50": pct(tick_ms, 0.5), "p99": pct(tick_ms, 0.99), "max": max(tick_ms),
                             "what": "host wall time of pd_server_tick calls that ran a frame"},
            "mean_resident": float(np.mean(active_hist)), "max_resident": int(max(active_hist)),
            "wall_s": wall, "tet_iters_per_s_wall": tet_iters / wall,
            "tet_iters_per_s_gpu": tet_iters / (sum(gpu_ms) / 1e3),
            "one_at_a_time": {"wall_s": wall_seq, "gpu_frame_s": seq_gpu_ms / 1e3,
                              "tet_iters_per_s_gpu": tet_iters / (seq_gpu_ms / 1e3),
                              "tet_iters_per_s_wall": tet_iters / wall_seq}}


def workload_config(w, args, world):
    """The `config` of both arms: the workload, not the implementation."""
    return {"workload": (f"{w.name}: 390,000-tet thick cylindrical shell, 98,475 vertices, 200 domains"
                         if not args.small else f"{w.name} (small profiling case)"),
            "pd_iters_per_frame": args.iters, "dt": w.dt,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "per-iteration working set > 129 MB L2 (the solve's matrices alone > 0.3 GB): no flush needed"}


def run_reference(args, rank, world):
    """Reference arm: the FP64 CPU oracle.  A frame of the workload (20 PD
    iterations, ~75 s on one host core) is too long for a timed step, so a
    step is one PD iteration of frame 0 (the bounded sample): value = PD
    iterations/s, ms_per_step = ms per such step."""
    if rank != 0:
        return
    import numpy as np

    from oracle.pd_oracle import PDOracle
    w = workload(args.small)
    o = PDOracle(w.rest, w.tets, w.pinned, w.gamma_s, w.gamma_v, w.density, w.dt)
    x = w.rest.copy()
    v = np.zeros_like(x)
    y = o.inertial_target(x, v, w.gravity)
    xp = w.pin_targets(0)
    x = y.copy()
    x[o.pin_ids] = xp

    def one():
        R, V = o.local(x)
        b = o.rhs(y, R, V)
        x[o.free] = o.global_solve(b, xp)

    for _ in range(args.warmup):
        one()
    t = time.perf_counter()
    for _ in range(args.steps):
        one()
    sec = time.perf_counter() - t
    value = args.steps / sec
    hi = host_info()
    sample = f"each step: 1 PD iteration of frame 0 of the same workload (FP64, 1 thread); {args.steps} steps"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(w, args, world),
        "step": "one PD iteration (a frame is pd_iters_per_frame of them)",
        "solver": "FP64 oracle: banded Cholesky of the full matrix",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                         "nproc": hi["nproc"], "cpu": hi["cpu"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "gpu_launches": 0,
    }
    print(json.dumps(line))


def dominant_phase(per_launch_ms: dict, phase_bytes: dict, phase_launches: dict) -> str:
    """The kernel class with the largest time per PD iteration (mean time per
    launch x launches per iteration); among near-ties (kernels that run side
    by side) the one streaming the most bytes per launch."""
    per_iter = {k: v * max(1, phase_launches.get(k, 1)) for k, v in per_launch_ms.items()
                if k not in ("inertia", "velocity") and v > 0}
    t_max = max(per_iter.values())
    return max((k for k, v in per_iter.items() if v >= 0.9 * t_max), key=lambda k: phase_bytes.get(k, 0))


def time_leg(m, w, info, pins, n_iter, K, W, stream, local, world, phase_report=True):
    """Warm-up with every phase timed (the phase with the largest time per
    frame is the dominant kernel), then K frames timed with CUDA events on the
    mesh's stream (only the dominant kernel carries events), clocks sampled
    meanwhile; then the per-phase report.  Returns a dict."""
    import torch
    from paper_2405_12484_gb300.sim import phase_bit
    m.enable_timing(-1)
    for n in range(W):
        m.step(pins[n], w.gravity, n_iter)
    m.sync()
    warm = m.phase_times()
    dominant = dominant_phase(warm, info["phase_bytes"], info.get("phase_launches", {}))
    # events around the dominant kernel in one PD iteration of every frame (an event pair
    # in every iteration would add its own cost to the frame time)
    sample_it = n_iter // 2
    m.enable_timing(phase_bit(dominant), iteration=sample_it)
    for n in range(2):
        m.step(pins[n], w.gravity, n_iter)
    m.sync()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    clocks = ClockSampler(local)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    clocks.mark(True)
    ev[0].record(stream)
    for k in range(K):
        m.step(pins[W + k], w.gravity, n_iter)
        ev[k + 1].record(stream)
    ev[K].synchronize()
    clocks.mark(False)
    torch.cuda.synchronize()
    clock_info = clocks.stop()
    barrier(world)
    m.sync()
    frame_ms = [ev[k].elapsed_time(ev[k + 1]) for k in range(K)]
    total_ms = ev[0].elapsed_time(ev[K])
    phase = m.phase_times()
    out = {"dominant": dominant, "dom_ms": phase.get(dominant, 0.0), "frame_ms": frame_ms, "total_ms": total_ms,
           "clocks": clock_info, "dom_sampled_iteration": sample_it}
    if phase_report:
        peak, _ = measured_peaks()
        m.enable_timing(-1)
        for n in range(3):
            m.step(pins[n], w.gravity, n_iter)
        pt = m.phase_times()
        out["phases"] = {}
        for k, ms in pt.items():
            if ms > 0:
                by = info["phase_bytes"].get(k, 0)
                out["phases"][k] = {"ms": ms, "bytes": by, "GB/s": by / (ms * 1e-3) / 1e9,
                                    "frac": by / (ms * 1e-3) / 1e9 / peak}
        m.enable_timing(phase_bit(dominant), iteration=sample_it)
    return out


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(q * len(xs)))]


def frame0_error(m, w, x0ref, n_iter):
    """Relative error (and displacement-relative error) of the first frame from rest against the FP64 oracle."""
    import numpy as np
    import torch
    m.set_state(torch.as_tensor(w.rest, dtype=torch.float32), torch.zeros((w.n_v, 3)))
    x = torch.empty((w.n_v, 3), device="cuda")
    m.step(torch.as_tensor(w.pin_targets(0), dtype=torch.float32), w.gravity, n_iter, x_out=x)
    m.sync()
    xg = x.cpu().numpy().astype(np.float64)
    return {"e_frame0": float(np.linalg.norm(xg - x0ref) / np.linalg.norm(x0ref)),
            "e_frame0_disp": float(np.linalg.norm(xg - x0ref) / np.linalg.norm(x0ref - w.rest))}


def main():
    args = parse()
    rank, world, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    # the oracle's host-side jobs start before the first CUDA call (child processes)
    jobs = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        jobs = OracleJobs(args.small, args.iters, check=not args.no_oracle_check)
    import numpy as np
    import torch

    import __graft_entry__
    from paper_2405_12484_gb300.sim import Mesh, phase_bit

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a GPU (the CUDA library has no CPU path)")
    torch.cuda.set_device(local)
    __graft_entry__.build()
    w = workload(args.small)
    n_iter = args.iters
    stream = torch.cuda.current_stream()
    m = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, stream=stream)
    m.set_materials(w.gamma_s, w.gamma_v)
    t0 = time.perf_counter()
    m.prefactor(w.dt, precision=args.precision, refine_steps=args.refine, use_graphs=True,
                correction=args.correction, single_level=args.single_level, streaming=args.streaming,
                modal=args.modal, modes=args.modes, jacobi_sweeps=args.sweeps if args.modal else 0)
    prefactor_s = time.perf_counter() - t0
    info = m.info()
    K, W = args.steps, max(3, args.warmup)
    # per-frame pin targets resident on the device before the timed region
    pins = torch.as_tensor(np.stack([w.pin_targets(n) for n in range(W + K)]), dtype=torch.float32,
                           device="cuda").contiguous()
    x_out = torch.empty((w.n_v, 3), device="cuda", dtype=torch.float32)

    # ---- timed region: K frames, inputs resident in HBM
    leg = time_leg(m, w, info, pins, n_iter, K, W, stream, local, world)
    value, total_ms = whole_job_rate(K * n_iter, leg["total_ms"], world)
    ms_frame = total_ms / K
    dominant = leg["dominant"]

    peak, peak_kind = measured_peaks()
    dom_ms = leg["dom_ms"]
    dom_bytes = info["phase_bytes"][dominant]
    achieved = dom_bytes / (dom_ms * 1e-3) / 1e9 if dom_ms > 0 else None
    # DRAM traffic per launch from an ncu capture of the same kernel (summarised under
    # profiles/), as the ratio traffic / algorithmic bytes scaled to this launch's bytes
    ratio = TRAFFIC_RATIO.get((dominant, args.precision, "single" if not info["two_level"] else "two"))
    traffic = ratio * dom_bytes if (ratio is not None and not args.small) else None
    roofline = {"bound": "hbm", "kernel": dominant, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None, "peak_kind": peak_kind,
                "traffic": traffic, "algorithmic_bytes": dom_bytes, "avg_launch_ms": dom_ms,
                "launches_timed": K * max(1, info["phase_launches"][dominant]),
                "timed": f"CUDA events on the mesh stream around each launch of the kernel in PD iteration "
                         f"{leg['dom_sampled_iteration']} of every timed frame ({info['phase_launches'][dominant]} "
                         f"per iteration; bytes and time per launch)"}
    if dominant in ("dd_interior", "dd_interior2"):
        roofline["note"] = ("runs on a low-priority side stream beside the interface chain (off the critical "
                            "path): its live duration includes the time it yields the GPU to that chain; a large "
                            "product goes out as two launches of half its tiles, each timed and counted alone")
    # the same figures for the kernel class that takes the most time on the critical path (the
    # side-stream products excluded), from the phase-report frames where every phase carries events
    critical = None
    ph = leg.get("phases", {})
    cands = {k: v["ms"] * max(1, info["phase_launches"].get(k, 1)) for k, v in ph.items()
             if k not in ("inertia", "velocity", "dd_interior", "dd_interior2") and v.get("bytes", 0) > 0}
    if cands:
        ck = max(cands, key=cands.get)
        critical = {"kernel": ck, "achieved": ph[ck]["GB/s"], "peak": peak, "unit": "GB/s", "frac": ph[ck]["frac"],
                    "algorithmic_bytes": ph[ck]["bytes"], "avg_launch_ms": ph[ck]["ms"],
                    "timed": "phase-report frames after the timed region, every kernel class between CUDA events"}
        if ck == "local" and not args.small:
            # issue-rate roofline: warp instructions of the launch against 4 per SM and cycle at the SM clock
            sm_hz = (leg["clocks"].get("sm_max_mhz") or 2070.0) * 1e6
            warp_instr = w.n_t * LOCAL_THREAD_INSTR_PER_TET / LOCAL_SIMT
            peak_issue = torch.cuda.get_device_properties(local).multi_processor_count * 4 * sm_hz
            achieved_issue = warp_instr / (ph[ck]["ms"] * 1e-3)
            critical["alu"] = {"bound": "alu", "warp_instructions": warp_instr, "achieved": achieved_issue,
                               "peak": peak_issue, "unit": "warp instructions/s", "frac": achieved_issue / peak_issue,
                               "source": "instructions per tet and SIMT efficiency of k_local_assemble from its ncu "
                                         "capture over the phase's time (which includes k_assemble_shared); "
                                         "peak = SMs x 4 schedulers x 1 instruction per cycle x SM clock"}

    # ---- end to end through the C ABI with host buffers (pinned), copies inside the timed region;
    # the same captured frame as the timed region (with the dominant kernel's events)
    pins_h = torch.as_tensor(np.stack([w.pin_targets(n) for n in range(K)]), dtype=torch.float32).pin_memory()
    out_h = torch.empty((4, w.n_v, 3), dtype=torch.float32).pin_memory()   # every frame read back, ring of 4
    pin_d = torch.empty((int(w.pinned.sum()), 3), device="cuda")
    for n in range(2):
        m.step(pins[n], w.gravity, n_iter, x_out=x_out)
    m.sync()
    barrier(world)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for k in range(K):
        pin_d.copy_(pins_h[k], non_blocking=True)
        m.step(pin_d, w.gravity, n_iter, x_out=x_out)
        out_h[k % 4].copy_(x_out, non_blocking=True)
    e1.record(stream)
    e1.synchronize()
    e2e_value, e2e_ms = whole_job_rate(K * n_iter, e0.elapsed_time(e1), world)
    m.sync()

    # ---- mixed precision: BF16 matrices on the tensor cores, the correction form (the residual
    # b - K x formed per tet inside the fused local step), same frames, same timing
    mixed, mixed_tf32 = None, None
    mm, mt = None, None
    plain = (args.precision == "fp32" and not args.correction and not args.modal and not args.streaming
             and not args.single_level and args.refine == 0)

    def mixed_leg(prec, kernels):
        mx = Mesh(w.rest, w.tets, w.pinned, w.tet_domain, w.n_domains, w.density, stream=stream)
        mx.set_materials(w.gamma_s, w.gamma_v)
        mx.prefactor(w.dt, precision=prec, correction=True, use_graphs=True)
        lm = time_leg(mx, w, mx.info(), pins, n_iter, K, W, stream, local, 1)
        return mx, {"precision": prec, "form": "correction (residual per PD iteration, FP32 vectors)",
                    "ms_per_frame": lm["total_ms"] / K, "pd_iters_per_s": K * n_iter / (lm["total_ms"] / 1e3),
                    "frame_ms": {"p50": pct(lm["frame_ms"], 0.5), "p99": pct(lm["frame_ms"], 0.99)},
                    "dominant": lm["dominant"], "phases": lm.get("phases", {}), "clocks": lm["clocks"],
                    "tensor_core_kernels": kernels}

    if rank == 0 and plain and not args.no_mixed:
        mm, mixed = mixed_leg("bf16", ["k_axpy_mma<false> (interior, boundary-mode and back-substitution products)",
                                       "k_rowdot_mma (second-level and coarse row-form products)"])
        mt, mixed_tf32 = mixed_leg("tf32", ["k_axpy_mma<true> (interior, boundary-mode and back-substitution "
                                            "products; the row-form products stay FP32-sized on the CUDA cores)"])

    # ---- accuracy of each precision's first frame against the FP64 oracle (host-side job)
    accuracy = None
    if jobs is not None and not args.no_oracle_check:
        jobs.join(timeout=900)
        ref = jobs.frame0()
        if ref is not None:
            accuracy = {"fp32" if args.precision == "fp32" else args.precision: frame0_error(m, w, ref, n_iter)}
            if mm is not None:
                accuracy["bf16_correction"] = frame0_error(mm, w, ref, n_iter)
            if mt is not None:
                accuracy["tf32_correction"] = frame0_error(mt, w, ref, n_iter)
        else:
            accuracy = {"error": str(jobs.results.get("frame", (None, "not run"))[1])}
    for mx in (mm, mt):
        if mx is not None:
            mx.close()

    cpu = None
    if jobs is not None:
        res = jobs.join(timeout=900)
        hi = host_info()
        one, err1 = res.get("one_thread", (None, "not run"))
        alln, errn = res.get("all_cores", (None, "not run"))
        if alln is not None:
            cpu = {"value": alln["iters"] / alln["seconds"], "unit": UNIT, "cores": hi["nproc"], "kind": "oracle",
                   "sample": f"{alln['iters']} PD iterations of frame 0 of the same workload, FP64, "
                             f"BLAS threads = {hi['nproc']}",
                   "one_thread": (one["iters"] / one["seconds"]) if one else None,
                   "nproc": hi["nproc"], "cpu": hi["cpu"]}
        else:
            cpu = {"value": None, "unit": UNIT, "cores": hi["nproc"], "kind": "oracle",
                   "sample": f"failed: {errn or err1}"}

    launches = K * (info["launches_per_frame"] + n_iter * info["launches_per_iter"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms_frame, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if args.precision == "fp32" else args.precision, "data": "synthetic",
            "config": workload_config(w, args, world),
            "solver": {"precision": args.precision, "refine_steps": args.refine, "correction_form": args.correction,
                       "method": ("modal, %d modes, %d Chebyshev-Jacobi sweeps" % (args.modes, args.sweeps)
                                  if args.modal else "exact subspace solve"),
                       "n_interface": info["n_interface"], "two_level": bool(info["two_level"]),
                       "n_groups": info["n_groups"], "n_top_interface": info["n_top_interface"],
                       "prefactor_s": prefactor_s},
            "frame_ms": {"p50": pct(leg["frame_ms"], 0.5), "p99": pct(leg["frame_ms"], 0.99),
                         "min": min(leg["frame_ms"]), "max": max(leg["frame_ms"])},
            "roofline": roofline,
            "roofline_critical_path": critical,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(pin_d.numel() * 4),
                    "d2h_bytes_per_step": int(w.n_v * 3 * 4), "ms_per_step": e2e_ms / K},
            "gpu_launches": launches,
            "clocks": leg["clocks"],
            "phases": leg.get("phases", {}),
        }
        if mixed is not None:
            line["mixed_precision"] = mixed
            line["mixed_precision_tf32"] = mixed_tf32
        if accuracy is not None:
            line["accuracy_vs_fp64"] = accuracy
        if not args.no_serving and world == 1:
            line["serving"] = run_serving(args)
        print(json.dumps(line))
    m.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    if "reference" in sys.argv:
        # the oracle's timed arm runs on one host thread; fix it before numpy loads
        for _k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ[_k] = "1"
    main()
