"""Command-line runner: one cavity, a fixed number of time steps, timing and observables.

  python -m paper_2211_05009_gb300.run --nx 2048 --ny 2048 --re 8000 --u 0.05 --dtype f32s --steps 1000

Prints one JSON line with the step rate (GLUPS from CUDA events on the library's stream), the
Eq. 6 residual, the mass and the primary-vortex minimum of Psi with its centre.  Also the command
the profiles under profiles/ were taken with.  --log PATH appends one JSON record per --log-every
steps (step, Eq. 6 residual, mass, elapsed seconds); the step rate then includes those reads.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from .build import build


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--re", type=float, default=8000.0)
    ap.add_argument("--u", type=float, default=0.05)
    ap.add_argument("--dtype", default="f32s", choices=sorted(B.DTYPES))
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=0)
    ap.add_argument("--config", type=int, default=None, help="launch shape of the step kernel")
    ap.add_argument("--autotune", action="store_true", help="pick the fastest launch shape first")
    ap.add_argument("--log", default=None, help="JSONL run log (one record per --log-every steps)")
    ap.add_argument("--log-every", type=int, default=1000)
    a = ap.parse_args(argv)
    build()
    stream = torch.cuda.current_stream()
    ctx = B.lbm_create(a.nx, a.ny, a.re, a.u, a.dtype)
    try:
        B.lbm_set_stream(ctx, stream.cuda_stream)
        if a.config is not None:
            B.lbm_set_launch_config(ctx, a.config)
        if a.autotune:
            B.lbm_autotune(ctx, 40)
        if a.warmup:
            B.lbm_step(ctx, a.warmup)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        if a.log:
            import time
            every = max(B.RESIDUAL_INTERVAL, a.log_every // B.RESIDUAL_INTERVAL * B.RESIDUAL_INTERVAL)
            w0 = time.perf_counter()
            with open(a.log, "a") as log:
                done = 0
                while done < a.steps:
                    n = min(every, a.steps - done)
                    B.lbm_step(ctx, n)
                    done += n
                    rec = {"step": B.lbm_get_info(ctx).step, "elapsed_s": time.perf_counter() - w0,
                           "mass": B.lbm_mass(ctx)}
                    if rec["step"] >= B.RESIDUAL_INTERVAL:
                        rec["residual"] = B.lbm_residual(ctx)
                    log.write(json.dumps(rec) + "\n")
                    log.flush()
        else:
            B.lbm_step(ctx, a.steps)
        t1.record(stream)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        out = {"nx": a.nx, "ny": a.ny, "Re": a.re, "U": a.u, "dtype": a.dtype, "steps": a.steps,
               "seconds": sec, "glups": a.nx * a.ny * a.steps / sec / 1e9 if sec > 0 else None,
               "mass": B.lbm_mass(ctx), "launch_config": B.lbm_get_info(ctx).launch_config}
        if a.warmup + a.steps >= B.RESIDUAL_INTERVAL:
            out["residual"] = B.lbm_residual(ctx)
        out["psi_min"], out["xc"], out["yc"] = B.lbm_stream_function(ctx)
        print(json.dumps(out), flush=True)
    finally:
        B.lbm_destroy(ctx)


if __name__ == "__main__":
    main()
