"""Precision study: one cavity stepped in every storage type against the FP64 run.

  python -m paper_2211_05009_gb300.precision --nx 2048 --ny 2048 --re 8000 --u 0.05 \
      --checkpoints 20000,50000,100000,200000

For each storage type (f64, f32, f32s, f16s, bf16s, q16s) the same cavity runs the same number of steps;
reported per type: step rate (GLUPS, device time), max and RMS |u - u_f64| / U, the error of the
primary-vortex minimum of Psi (relative) and of its centre (nodes), the Eq. 6 residual and mass.
The FP64 run is the reference (it matches the CPU oracle to 1e-12).  Prints one JSON document.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from .build import build

ORDER = ["f64", "f32", "f32s", "f16s", "bf16s", "q16s"]


def run_one(nx, ny, re, u, dtype, checkpoints, chunk=10_000):
    """Step one cavity to each checkpoint; returns (timing/observables at the last one, list of
    device (u_x, u_y) fields per checkpoint, list of (psi_min, xc, yc) per checkpoint)."""
    st = torch.cuda.current_stream()
    ctx = B.lbm_create(nx, ny, re, u, dtype)
    try:
        B.lbm_set_stream(ctx, st.cuda_stream)
        B.lbm_autotune(ctx, 20)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fields, psis, sec, done = [], [], 0.0, 0
        for ck in checkpoints:
            torch.cuda.synchronize()
            t0.record(st)
            while done < ck:
                n = min(chunk, ck - done)
                B.lbm_step(ctx, n)
                done += n
            t1.record(st)
            torch.cuda.synchronize()
            sec += t0.elapsed_time(t1) / 1e3
            ux = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
            uy = torch.empty_like(ux)
            B.lbm_moments(ctx, None, ux, uy)
            fields.append((ux, uy))
            psis.append(B.lbm_stream_function(ctx))
        steps = checkpoints[-1]
        psi_min, xc, yc = psis[-1]
        return {"dtype": dtype, "glups": nx * ny * steps / sec / 1e9, "seconds": sec,
                "launch_config": B.lbm_get_info(ctx).launch_config,
                "residual": B.lbm_residual(ctx) if steps >= 100 else None, "mass": B.lbm_mass(ctx),
                "psi_min": psi_min, "xc": xc, "yc": yc}, fields, psis
    finally:
        B.lbm_destroy(ctx)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--re", type=float, default=8000.0)
    ap.add_argument("--u", type=float, default=0.05)
    ap.add_argument("--steps", type=int, default=200_000)
    ap.add_argument("--checkpoints", default=None,
                    help="comma-separated step counts at which errors are reported (default: --steps)")
    ap.add_argument("--dtypes", default=",".join(ORDER))
    a = ap.parse_args(argv)
    build()
    cks = sorted(int(v) for v in a.checkpoints.split(",")) if a.checkpoints else [a.steps]
    rows, ref = [], None
    for dt in a.dtypes.split(","):
        row, fields, psis = run_one(a.nx, a.ny, a.re, a.u, dt, cks)
        if ref is None:
            ref = (fields, psis)
        row["errors"] = []
        for k, ck in enumerate(cks):
            ux, uy = fields[k]
            ux0, uy0 = ref[0][k]
            p, p0 = psis[k], ref[1][k]
            du = torch.maximum((ux - ux0).abs(), (uy - uy0).abs())
            row["errors"].append({
                "step": ck, "max_du_over_U": float(du.max()) / a.u,
                "rms_du_over_U": float(du.pow(2).mean().sqrt()) / a.u,
                "psi_min_rel_err": abs(p[0] - p0[0]) / abs(p0[0]),
                "psi_min_err_over_UL": abs(p[0] - p0[0]) / (a.u * a.nx),
                "centre_err_nodes": max(abs(p[1] - p0[1]), abs(p[2] - p0[2])) * a.nx})
        rows.append(row)
        if dt != ORDER[0]:
            del fields
    print(json.dumps({"nx": a.nx, "ny": a.ny, "Re": a.re, "U": a.u, "checkpoints": cks,
                      "reference": rows[0]["dtype"], "runs": rows}), flush=True)


if __name__ == "__main__":
    main()
