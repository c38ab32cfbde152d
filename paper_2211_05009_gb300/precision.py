"""Precision study: one cavity stepped in every storage type against the FP64 run.

  python -m paper_2211_05009_gb300.precision --nx 2048 --ny 2048 --re 8000 --u 0.05 --steps 200000

For each storage type (f64, f32, f32s, f16s, bf16s) the same cavity runs the same number of steps;
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

ORDER = ["f64", "f32", "f32s", "f16s", "bf16s"]


def run_one(nx, ny, re, u, dtype, steps, chunk=10_000):
    st = torch.cuda.current_stream()
    ctx = B.lbm_create(nx, ny, re, u, dtype)
    try:
        B.lbm_set_stream(ctx, st.cuda_stream)
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(st)
        left = steps
        while left > 0:
            n = min(chunk, left)
            B.lbm_step(ctx, n)
            left -= n
        t1.record(st)
        torch.cuda.synchronize()
        sec = t0.elapsed_time(t1) / 1e3
        ux = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
        uy = torch.empty_like(ux)
        B.lbm_moments(ctx, None, ux, uy)
        psi_min, xc, yc = B.lbm_stream_function(ctx)
        return {"dtype": dtype, "glups": nx * ny * steps / sec / 1e9, "seconds": sec,
                "residual": B.lbm_residual(ctx) if steps >= 100 else None, "mass": B.lbm_mass(ctx),
                "psi_min": psi_min, "xc": xc, "yc": yc}, ux, uy
    finally:
        B.lbm_destroy(ctx)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=2048)
    ap.add_argument("--ny", type=int, default=2048)
    ap.add_argument("--re", type=float, default=8000.0)
    ap.add_argument("--u", type=float, default=0.05)
    ap.add_argument("--steps", type=int, default=200_000)
    ap.add_argument("--dtypes", default=",".join(ORDER))
    a = ap.parse_args(argv)
    build()
    rows, ref = [], None
    for dt in a.dtypes.split(","):
        row, ux, uy = run_one(a.nx, a.ny, a.re, a.u, dt, a.steps)
        if ref is None:
            ref = (row, ux, uy)
        r0, ux0, uy0 = ref
        du = torch.maximum((ux - ux0).abs(), (uy - uy0).abs())
        row["max_du_over_U"] = float(du.max()) / a.u
        row["rms_du_over_U"] = float(du.pow(2).mean().sqrt()) / a.u
        row["psi_min_rel_err"] = abs(row["psi_min"] - r0["psi_min"]) / abs(r0["psi_min"])
        row["centre_err_nodes"] = max(abs(row["xc"] - r0["xc"]), abs(row["yc"] - r0["yc"])) * a.nx
        rows.append(row)
        del ux, uy
    print(json.dumps({"nx": a.nx, "ny": a.ny, "Re": a.re, "U": a.u, "steps": a.steps,
                      "reference": rows[0]["dtype"], "runs": rows}), flush=True)


if __name__ == "__main__":
    main()
