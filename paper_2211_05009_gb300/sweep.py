"""Re x Ar sweep of lid-driven rectangular cavities (Sec. 3.3, Fig. 17; Table 3 periods):
batched persistent run against one-cavity-at-a-time runs, time to steady state at equal residual.

  python -m paper_2211_05009_gb300.sweep --nx 500 --tol 1e-9 --max-steps 1000000 --sequential

Cavities: nx x round(nx Ar) nodes, U = 0.1 (lattice units), Re = U nx / nu.  Each runs until its
Eq. 6 residual is below tol or max-steps steps were taken.  The batched arm steps all cavities in
one persistent launch per 100 steps and retires converged ones; the sequential arm runs the same
cavities one after another through the single-cavity API (lbm_run_to_residual).  The batched
arm first lets lbm_batch_autotune pick its tile shape (inside its timed region).  Each cavity
records u_x, u_y at the Sec. 3.3 observing point every `probe-every` steps, and its flow state is
classified from that series (analysis.classify).  Prints one JSON document.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import binding as B
from .analysis import classify, observing_point
from .build import build

RE_DEFAULT = "4000,5000,6000,7000,8000"
AR_DEFAULT = "0.4,0.6,0.8,1.0,1.2,1.4,1.6,1.8,2.0"


# (Ar, Re) pairs at which Sec. 3.3 reports a flow state: the periodic entries of Table 3, and the
# cavities of Figs. 8-10 (Re 6000, 6500 and 8000 at Ar 0.5, 0.6, 0.8, 1.1, 1.2, 1.5, 1.6).
TABLE3_PAIRS = [(0.4, 8000)] + [(0.5, r) for r in (6500, 7000, 7500)] + \
    [(0.6, r) for r in (5500, 6000, 6500, 7000, 7500, 8000)] + \
    [(0.7, r) for r in (5000, 5500, 6000, 6500, 7000, 7500)] + [(0.8, 6000), (0.8, 6500)] + \
    [(1.2, r) for r in (4500, 5000, 5500, 6000)] + [(1.3, r) for r in (4500, 5000, 5500, 6000, 6500)] + \
    [(1.4, r) for r in (5000, 5500, 6000, 6500, 7000)] + [(1.7, 6500), (1.7, 7000)] + \
    [(1.8, 7000), (1.8, 7500), (1.9, 7000), (1.9, 7500)]
FIG8_10_PAIRS = [(ar, re) for re in (6000, 6500, 8000) for ar in (0.5, 0.6, 0.8, 1.1, 1.2, 1.5, 1.6)]


def cavity_list(nx, res, ars, U, extra_pairs=()):
    """The Re x Ar grid, then any (Ar, Re) pairs not on it, as cavities of nx x round(nx Ar)."""
    cases, seen = [], set()
    for ar, re in [(ar, re) for ar in ars for re in res] + list(extra_pairs):
        key = (round(float(ar), 6), round(float(re), 6))
        if key in seen:
            continue
        seen.add(key)
        cases.append({"Re": float(re), "Ar": float(ar), "nx": nx, "ny": int(round(nx * ar)), "U": U})
    return cases


def run_batched(cases, dtype, tol, max_steps, every, cap, tune_steps=50, save_series=None, shape=-1):
    st = torch.cuda.current_stream()
    b = B.lbm_batch_create([c["nx"] for c in cases], [c["ny"] for c in cases], [c["Re"] for c in cases],
                           [c["U"] for c in cases], dtype)
    try:
        B.lbm_batch_set_stream(b, st.cuda_stream)
        series = torch.zeros((len(cases), cap, 2), dtype=torch.float64, device="cuda")
        pts = [observing_point(c["Ar"]) for c in cases]
        B.lbm_batch_probe(b, [p[0] for p in pts], [p[1] for p in pts], every, series, cap)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        tune = None
        if shape >= 0:
            B.lbm_batch_set_shape(b, shape)
        elif tune_steps > 0:
            chosen, ms = B.lbm_batch_autotune(b, tune_steps)
            tune = {"chosen": chosen, "trial_ms": ms.tolist(), "steps": tune_steps}
        rc, done = B.lbm_batch_run_to_residual(b, len(cases), tol, max_steps)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        r, status = B.lbm_batch_residual(b, len(cases))
        shape, rows, blocks, graphs = B.lbm_batch_launch_info(b)
        out = []
        ser = series.cpu().numpy()
        if save_series:  # raw probe ring buffers [cavity][sample mod cap][u_x, u_y] and steps taken
            np.savez_compressed(save_series, series=ser.astype(np.float32), steps=np.asarray(done), every=every,
                                re=np.array([c["Re"] for c in cases]), ar=np.array([c["Ar"] for c in cases]))
        for i, c in enumerate(cases):
            n = int(done[i]) // every
            k = min(n, cap)
            ux = np.roll(ser[i, :, 0], -(n % cap))[-k:] if n > cap else ser[i, :k, 0]
            # steady per the paper's own Eq. 6 tolerance (1e-6), whatever the run tolerance
            steady = bool(status[i] == 1) or float(r[i]) < 1e-6
            fs = classify(ux, every, c["U"], c["nx"], converged=steady) if k >= 8 else None
            psi_min, xc, yc = B.lbm_batch_stream_function(b, i)
            out.append({**c, "steps": int(done[i]), "residual": float(r[i]), "status": int(status[i]),
                        "state": fs.state if fs else None,
                        "period_steps": fs.period_steps if fs else None,
                        "period_convective": fs.period_convective if fs else None,
                        "period_time_dx": fs.period_steps / c["nx"] if fs and fs.period_steps else None,
                        "psi_min": psi_min, "xc": xc, "yc": yc})
        lu = sum(c["nx"] * c["ny"] * o["steps"] for c, o in zip(cases, out))
        return {"wall_s": wall, "lattice_updates": lu, "glups": lu / wall / 1e9,
                "all_converged": rc == B.LBM_OK, "autotune": tune,
                "launch": {"shape": shape, "rows_per_item": rows, "blocks": blocks, "graph_replays": graphs},
                "cavities": out}
    finally:
        B.lbm_batch_destroy(b)


def run_sequential(cases, dtype, tol, max_steps, first_crossing=True):
    """One cavity at a time through the single-cavity API.  first_crossing: stop at the first
    100-step checkpoint whose Eq. 6 residual is below tol -- the batched arm's retirement rule --
    reading every checkpoint as it completes (lbm_step(100) + lbm_residual); otherwise
    lbm_run_to_residual, which reads one chunk behind and stops at two consecutive checkpoints
    below tol."""
    st = torch.cuda.current_stream()
    out, total, lu = [], 0.0, 0
    for c in cases:
        ctx = B.lbm_create(c["nx"], c["ny"], c["Re"], c["U"], dtype)
        try:
            B.lbm_set_stream(ctx, st.cuda_stream)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if first_crossing:
                done, ok = 0, False
                while done < max_steps and not ok:
                    B.lbm_step(ctx, B.RESIDUAL_INTERVAL)
                    done += B.RESIDUAL_INTERVAL
                    ok = B.lbm_residual(ctx) < tol
            else:
                rc, done = B.lbm_run_to_residual(ctx, tol, max_steps)
                ok = rc == B.LBM_OK
            torch.cuda.synchronize()
            wall = time.perf_counter() - t0
            total += wall
            lu += c["nx"] * c["ny"] * done
            out.append({"Re": c["Re"], "Ar": c["Ar"], "steps": done, "wall_s": wall,
                        "residual": B.lbm_residual(ctx) if done >= 100 else None,
                        "converged": ok})
        finally:
            B.lbm_destroy(ctx)
    return {"wall_s": total, "lattice_updates": lu, "glups": lu / total / 1e9,
            "rule": "first checkpoint below tol" if first_crossing else "lbm_run_to_residual",
            "cavities": out}


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--nx", type=int, default=500)
    ap.add_argument("--re", default=RE_DEFAULT)
    ap.add_argument("--ar", default=AR_DEFAULT)
    ap.add_argument("--u", type=float, default=0.1)
    ap.add_argument("--dtype", default="f32s")
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--max-steps", type=int, default=1_000_000)
    ap.add_argument("--probe-every", type=int, default=100)
    ap.add_argument("--sequential", action="store_true", help="also run the one-at-a-time arm")
    ap.add_argument("--also-run-to-residual", action="store_true",
                    help="time the one-at-a-time arm a second time through lbm_run_to_residual")
    ap.add_argument("--autotune-steps", type=int, default=50, help="steps per tile-shape trial (0: keep the default shape)")
    ap.add_argument("--shape", type=int, default=-1, help="use this tile shape (0..LBM_BATCH_SHAPES-1) instead of autotuning")
    ap.add_argument("--save-series", default=None, help="write the probe series of the batched arm (.npz)")
    ap.add_argument("--paper-pairs", action="store_true",
                    help="add every (Ar, Re) at which Sec. 3.3 reports a state (Table 3, Figs. 8-10)")
    a = ap.parse_args(argv)
    build()
    res = [float(v) for v in a.re.split(",")]
    ars = [float(v) for v in a.ar.split(",")]
    cases = cavity_list(a.nx, res, ars, a.u, TABLE3_PAIRS + FIG8_10_PAIRS if a.paper_pairs else ())
    cap = max(8, a.max_steps // a.probe_every)
    doc = {"nx": a.nx, "U": a.u, "dtype": a.dtype, "tol": a.tol, "max_steps": a.max_steps,
           "n_cavities": len(cases), "nodes": sum(c["nx"] * c["ny"] for c in cases)}
    doc["batched"] = run_batched(cases, a.dtype, a.tol, a.max_steps, a.probe_every, cap, a.autotune_steps,
                                 a.save_series, a.shape)
    if a.sequential:
        doc["sequential"] = run_sequential(cases, a.dtype, a.tol, a.max_steps)
        doc["speedup_time_to_steady"] = doc["sequential"]["wall_s"] / doc["batched"]["wall_s"]
        if a.also_run_to_residual:
            doc["sequential_run_to_residual"] = run_sequential(cases, a.dtype, a.tol, a.max_steps, False)
    print(json.dumps(doc), flush=True)


if __name__ == "__main__":
    main()
