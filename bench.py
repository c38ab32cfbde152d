"""Throughput benchmark of the fused D2Q9 cavity step on GB300.

Workload (one GPU): the square lid-driven cavity of 2048 x 2048 nodes, Re = 8000, U = 0.05,
FP32 arithmetic on FP32 shifted-deviation storage (the precision-study / roofline configuration;
its 302 MB population working set exceeds the 129 MB L2, so no L2 flush is needed).

One benchmark step = one pass of the whole hot path over the cavity: 100 fused
stream-collide-wall time steps (Eq. 1-3, Sec. 2.2 ii) with the two observing points sampled every
2 steps (Sec. 3.3), the FP64 Eq. 6 residual and mass reduction on the 100th step, and the FP64
stream function with its primary-vortex minimum and centre (Tables 1-2 post-processing).
The metric is lattice updates per second (GLUPS = nx*ny*100 per step / time).

  value     device time (CUDA events on the library's stream) with the state resident in HBM
  e2e       the same metric through the C ABI with HOST buffers: every step uploads the initial
            macroscopic field (rho, u_x, u_y; FP64, pinned) with lbm_set_moments, advances 100
            steps, reads the residual and downloads rho, u_x, u_y with lbm_moments
  roofline  the step kernel: 18 populations x 4 bytes per node and launch / its average duration
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the same workload (first steps of
            the same 2048^2 cavity): its OpenMP build on every host core, and the plain build
            on one thread

--impl reference runs that oracle as the reference arm.  Under torchrun (N > 1) every rank runs
an independent replica (weak scaling; the path needs no exchange between cavities).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

NX = NY = 2048
RE, U = 8000.0, 0.05
STORAGE = "f32s"
CHUNK = 100
BYTES_PER_LU = 18 * 4  # 9 populations read + 9 written, 4 bytes each
METRIC = "D2Q9 GLUPS (fused step, lattice updates per second)"
WORKLOAD = "square lid-driven cavity 2048x2048, Re=8000, U=0.05, FP32 arithmetic, FP32 shifted-deviation storage"
PROFILE = os.path.join(ROOT, "profiles", "k_step_f32s_2048x2048.txt")


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ clocks during the timed region
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index, self.proc, self.lines = index, None, []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU oracle leg
def oracle_sample(steps: int, openmp: bool = False):
    """FP64 oracle on the first `steps` time steps of the benchmark cavity: the plain build on one
    thread, or (openmp) the same source built with OpenMP on every host core."""
    import oracle as O
    p = O.Params.from_re(NX, NY, RE, U)
    f = O.init(p)
    t0 = time.perf_counter()
    O.run(p, f, steps, openmp=openmp)
    dt = time.perf_counter() - t0
    return NX * NY * steps / dt / 1e9, dt


def reference_arm(args, rank):
    if rank != 0:
        return
    import oracle as O
    O.build(openmp=True)
    cores = O.threads(openmp=True)
    p = O.Params.from_re(NX, NY, RE, U)
    f = O.init(p)
    for _ in range(args.warmup):
        f = O.step(p, f, openmp=True)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f = O.step(p, f, openmp=True)
    dt = time.perf_counter() - t0
    v = NX * NY * args.steps / dt / 1e9
    sample = (f"{args.steps} time steps of the 2048x2048 cavity (one oracle step per benchmark step), "
              f"OpenMP build of the oracle on {cores} host threads")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "GLUPS", "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "Re": RE, "U": U,
                                        "oracle": f"FP64 CPU, AoS, {cores} threads"},
        "cpu_baseline": {"value": v, "unit": "GLUPS", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


# ------------------------------------------------------------------ our arm
def read_profile_traffic(shape: int):
    """Per-launch DRAM bytes of the step kernel's launch shape `shape` from the committed ncu
    summary, if it was taken on the current kernel source."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    vals = {}
    for ln in text.splitlines():
        if ":" in ln:
            k, v = ln.split(":", 1)
            vals[k.strip()] = v.strip()
    src = os.path.join(ROOT, "paper_2211_05009_gb300", "csrc", "lbm_step_kernel.cuh")
    digest = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if vals.get("kernel_source_sha256_16") != digest:
        return None
    try:
        return float(vals[f"dram_bytes_per_launch_shape_{shape}"])
    except (KeyError, ValueError):
        return None


def max_over_ranks(value: float, world: int) -> float:
    """Largest value over the ranks of the default process group (the slowest rank's time);
    works for NCCL (CUDA tensor) and gloo (CPU tensor) groups."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, seconds_max: float, world: int) -> float:
    """Aggregate rate of `world` replicas that each processed units_per_rank in at most seconds_max."""
    return world * units_per_rank / seconds_max


def measured_peak():
    try:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def our_arm(args, rank, world, local_rank):
    import torch
    from paper_2211_05009_gb300 import binding as B
    from paper_2211_05009_gb300.build import build

    torch.cuda.set_device(local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    build()
    stream = torch.cuda.current_stream()
    ctx = B.lbm_create(NX, NY, RE, U, STORAGE)
    B.lbm_set_stream(ctx, stream.cuda_stream)
    cap = 8192
    probes = [torch.zeros((cap, 2), dtype=torch.float64, device="cuda") for _ in range(2)]
    B.lbm_probe(ctx, 0.5, 0.5, 2, probes[0], cap)   # Sec. 3.3 observing point for Ar = 1
    B.lbm_probe(ctx, 0.5, 0.2, 2, probes[1], cap)

    cfg, tuned_glups = B.lbm_autotune(ctx, 40)  # pick the fastest launch shape of the step kernel

    def bench_step():
        B.lbm_step(ctx, CHUNK)
        return B.lbm_stream_function(ctx)  # synchronising: the vortex centre reaches the host

    for _ in range(args.warmup):
        bench_step()
    torch.cuda.synchronize()

    ev_chunk = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.4)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    for k in range(args.steps):
        ev_chunk[k][0].record(stream)
        B.lbm_step(ctx, CHUNK)
        ev_chunk[k][1].record(stream)
        psi_min, xc, yc = B.lbm_stream_function(ctx)
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    elapsed = start.elapsed_time(end) / 1e3
    step_kernel_s = sum(a.elapsed_time(b) for a, b in ev_chunk) / 1e3 / (CHUNK * args.steps)
    residual = B.lbm_residual(ctx)
    mass = B.lbm_mass(ctx)
    elapsed = max_over_ranks(elapsed, world)
    lu = NX * NY * CHUNK * args.steps
    value = whole_job_rate(lu, elapsed, world) / 1e9

    # end to end through the C ABI with pinned host buffers
    e2e = None
    if not args.no_e2e:
        n = NX * NY
        host_in = [torch.empty((NY, NX), dtype=torch.float64, pin_memory=True) for _ in range(3)]
        host_out = [torch.empty((NY, NX), dtype=torch.float64, pin_memory=True) for _ in range(3)]
        B.lbm_moments(ctx, *host_in)  # a developed field, as a warm start would supply
        e2e_steps = max(3, min(args.steps, 10))

        def e2e_step():
            B.lbm_set_moments(ctx, *host_in)
            B.lbm_step(ctx, CHUNK)
            r = B.lbm_residual(ctx)
            B.lbm_moments(ctx, *host_out)
            return r

        e2e_step()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            e2e_step()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        te = max_over_ranks(te, world)
        e2e = {"value": whole_job_rate(n * CHUNK * e2e_steps, te, world) / 1e9, "unit": "GLUPS",
               "h2d_bytes_per_step": 3 * 8 * n, "d2h_bytes_per_step": 3 * 8 * n + 8,
               "steps": e2e_steps, "host_buffers": "pinned"}

    B.lbm_destroy(ctx)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return

    peak, peak_kind = measured_peak()
    algo_bytes = BYTES_PER_LU * NX * NY
    achieved = algo_bytes / step_kernel_s / 1e9
    traffic = read_profile_traffic(cfg)
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle as O
        O.build()
        O.build(openmp=True)
        cores = O.threads(openmp=True)
        steps_1 = 64  # about 14 s of single-thread oracle work
        v1, dt1 = oracle_sample(steps_1)
        steps_n = 64 * max(1, min(16, cores // 2))  # about the same wall time on all cores
        vn, dtn = oracle_sample(steps_n, openmp=True)
        cpu = {"value": vn, "unit": "GLUPS", "cores": cores, "kind": "oracle",
               "sample": f"first {steps_n} time steps of the same 2048x2048 cavity ({dtn:.1f} s, FP64, "
                         f"OpenMP build on {cores} host threads)",
               "single_thread": {"value": v1, "unit": "GLUPS", "cores": 1,
                                 "sample": f"first {steps_1} time steps ({dt1:.1f} s, plain build, one thread)"}}
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed / args.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nx": NX, "ny": NY, "Re": RE, "U": U, "storage": STORAGE,
                   "lbm_steps_per_step": CHUNK, "parallelism": f"replicas{world}",
                   "l2": "population working set 302 MB > 129 MB L2; no flush"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "peak_kind": peak_kind, "kernel": f"k_step<float, shifted> launch shape {cfg}",
                     "algorithmic_bytes_per_launch": algo_bytes,
                     "avg_launch_us": step_kernel_s * 1e6},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": args.steps * (CHUNK + 1 + 2),
        "clocks": clk,
        "result": {"residual_eq6": residual, "mass": mass, "psi_min": psi_min, "xc": xc, "yc": yc,
                   "lbm_steps": (args.warmup + args.steps) * CHUNK},
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse_args()
    rank, world, local_rank = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    our_arm(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
