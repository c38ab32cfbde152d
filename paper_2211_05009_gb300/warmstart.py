"""Learned warm start for the cavity solver: data, training and evaluation.

  python -m paper_2211_05009_gb300.warmstart --train 256 --test 64 --epochs 30 --out net.bin

1. Draws (Re, Ar) with Re ~ U[--re-min, --re-max], Ar ~ U[0.4, 2.0] (training seed 0, test seed 1,
   validation seed 2).
2. Coarse solutions: every draw on nxc x round(nxc Ar) nodes (nxc = nx / --coarse-ratio), run in
   one batch to its Eq. 6 tolerance or a step cap, at Re_c = min(Re, --coarse-re-max) (a coarse
   grid cannot go to tau -> 1/2); the network sees the true Re.
3. Training targets: the steady nx x round(nx Ar) fields of the training draws, from one batched
   run to --target-tol; draws that do not converge within the cap are excluded (and counted).
4. Training: the network (lbm_net, BF16 tensor-core kernels) maps [coarse field on the fine grid,
   Re, Ar, masks] to a correction of the fine field; Adam, mini-batches by gradient accumulation.
   At inference the correction is smoothed (--smooth box-filter passes, lbm_warm_smooth).
5. Fallback gate: on the validation draws, runs from rest and from the network's field pick the
   Reynolds number below which the warm start pays (least total steps); above it the solver
   starts from rest.
6. Evaluation on the test draws, batched runs to --tol at equal residual: from rest (Sec. 2.2 i,
   the fallback and the reference), from the interpolated coarse field and from the network's
   field, each set either at equilibrium or with the first-order Chapman-Enskog stress of its
   velocity field (LBM_INIT_NEQ), and the gated policy.  Reported: steps to the tolerance per
   draw, their totals and ratios (overall and by Re band), and wall times.
Prints one JSON document.
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np
import torch

from . import binding as B
from .build import build

U_LID = 0.1


def draws(n, seed, re_min, re_max):
    rng = np.random.default_rng(seed)
    return [(float(rng.uniform(re_min, re_max)), float(rng.uniform(0.4, 2.0))) for _ in range(n)]


def choose_gate(re, steps_rest, steps_warm, re_cap):
    """Fallback gate: the Reynolds number g minimising the total steps of the policy 'warm start
    if Re < g, else start from rest' on the given draws (candidates: every draw's Re and re_cap,
    which means warm everywhere).  Ties go to the smallest g (the most draws start from rest).
    Returns (g, total steps at g)."""
    re = np.asarray(re, dtype=float)
    rest = np.asarray(steps_rest, dtype=float)
    warm = np.asarray(steps_warm, dtype=float)
    cands = sorted(set(re.tolist())) + [float(re_cap)]
    totals = [float(np.where(re < g, warm, rest).sum()) for g in cands]
    k = int(np.argmin(totals))
    return cands[k], totals[k]


def pad16(n):
    return (n + 15) // 16 * 16


def batch_run(cases, dtype, tol, max_steps, init=None, flags=0):
    """cases: list of (nx, ny, Re).  init(i) -> (rho, ux, uy) device tensors or None; flags for
    lbm_batch_set_moments_ex.
    Returns (batch handle, steps per cavity, status, wall seconds)."""
    st = torch.cuda.current_stream()
    b = B.lbm_batch_create([c[0] for c in cases], [c[1] for c in cases], [c[2] for c in cases],
                           [U_LID] * len(cases), dtype)
    B.lbm_batch_set_stream(b, st.cuda_stream)
    if init is not None:
        for i in range(len(cases)):
            f = init(i)
            if f is not None:
                B.lbm_batch_set_moments(b, i, *f, flags=flags)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    B.lbm_batch_autotune(b, 20)
    rc, done = B.lbm_batch_run_to_residual(b, len(cases), tol, max_steps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    _, status = B.lbm_batch_residual(b, len(cases))
    return b, done, status, wall


def moments(b, i, nx, ny):
    out = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
    B.lbm_batch_moments(b, i, *out)
    return out


def make_input(coarse, re, ar, nx, ny):
    H = pad16(ny)
    inp = torch.empty((7, H, nx), dtype=torch.float32, device="cuda")
    rc, ux, uy = coarse
    B.lbm_warm_input(rc, ux, uy, rc.shape[1], rc.shape[0], re, ar, U_LID, nx, ny, H, inp,
                     torch.cuda.current_stream().cuda_stream)
    return inp, H


def target_tensor(fields, nx, ny, H):
    t = torch.empty((3, H, nx), dtype=torch.float32, device="cuda")
    B.lbm_warm_target(*fields, nx, ny, H, U_LID, t, torch.cuda.current_stream().cuda_stream)
    return t


def parser():
    ap = argparse.ArgumentParser()
    ap.add_argument("--train", type=int, default=256)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--val", type=int, default=48, help="validation draws that choose the fallback gate")
    ap.add_argument("--nx", type=int, default=128, help="fine grid width")
    ap.add_argument("--re-min", type=float, default=100.0)
    ap.add_argument("--re-max", type=float, default=1000.0)
    ap.add_argument("--width", type=int, default=20)
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--batch", type=int, default=8)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--dtype", default="f64", help="f64: FP32 storage stalls near 1e-6 (Eq. 6), above the tolerance")
    ap.add_argument("--tol", type=float, default=1e-9)
    ap.add_argument("--target-tol", type=float, default=1e-9)
    ap.add_argument("--max-steps", type=int, default=400_000)
    ap.add_argument("--coarse-tol", type=float, default=1e-7)
    ap.add_argument("--coarse-steps", type=int, default=150_000)
    ap.add_argument("--coarse-ratio", type=int, default=2, help="fine width / coarse width")
    ap.add_argument("--coarse-re-max", type=float, default=1e9)
    ap.add_argument("--smooth", type=int, default=4, help="box-filter passes over the network's correction")
    ap.add_argument("--out", default=None)
    return ap


def run(a) -> dict:
    """The whole pipeline (coarse runs, targets, training, gate, evaluation) for parsed arguments
    `a`; returns the report."""
    build()
    torch.manual_seed(0)
    st = torch.cuda.current_stream()
    report = {"args": vars(a)}
    NX, NXC = a.nx, a.nx // a.coarse_ratio
    train, test = draws(a.train, 0, a.re_min, a.re_max), draws(a.test, 1, a.re_min, a.re_max)
    val = draws(a.val, 2, a.re_min, a.re_max)
    allp = train + test + val

    # 2. coarse solutions of every draw
    cc = [(NXC, max(3, round(NXC * ar)), min(re, a.coarse_re_max)) for re, ar in allp]
    coarse, done_c, stat_c, wall_c = [], [], [], 0.0
    for k0 in range(0, len(cc), B.LBM_BATCH_MAX):  # one batch holds at most LBM_BATCH_MAX cavities
        part = cc[k0:k0 + B.LBM_BATCH_MAX]
        bc, d, st_, w = batch_run(part, a.dtype, a.coarse_tol, a.coarse_steps)
        coarse += [moments(bc, i, c[0], c[1]) for i, c in enumerate(part)]
        B.lbm_batch_destroy(bc)
        done_c += list(d)
        stat_c += list(st_)
        wall_c += w
    done_c, stat_c = np.array(done_c), np.array(stat_c)
    report["coarse"] = {"wall_s": wall_c, "converged": int((stat_c == 1).sum()), "n": len(cc),
                        "lattice_updates": int(sum(c[0] * c[1] * d for c, d in zip(cc, done_c)))}

    # 3. training targets
    if len(train) > B.LBM_BATCH_MAX:
        raise SystemExit(f"--train {len(train)}: at most {B.LBM_BATCH_MAX} (one batch of targets)")
    tc = [(NX, round(NX * ar), re) for re, ar in train]
    bt, done_t, stat_t, wall_t = batch_run(tc, a.dtype, a.target_tol, a.max_steps)
    r_t, _ = B.lbm_batch_residual(bt, len(tc))
    samples = []
    for i, (re, ar) in enumerate(train):
        if stat_t[i] != 1 or stat_c[i] != 1:  # no steady target, or a coarse run that did not settle
            continue
        ny = tc[i][1]
        inp, H = make_input(coarse[i], re, ar, NX, ny)
        tgt = target_tensor(moments(bt, i, NX, ny), NX, ny, H)
        # base = input channels 0..2, mask = the valid-row channel 6 (views, no copies)
        samples.append((inp, inp[:3], tgt, inp[6], H))
    B.lbm_batch_destroy(bt)
    report["targets"] = {"wall_s": wall_t, "converged": len(samples), "excluded": a.train - len(samples),
                         "residual_quantiles": np.quantile(r_t, [0, 0.5, 1]).tolist(),
                         "lattice_updates": int(sum(c[0] * c[1] * d for c, d in zip(tc, done_t)))}

    # 4. training
    net = B.lbm_net_create(a.width, 0)
    B.lbm_net_set_stream(net, st.cuda_stream)
    rng = np.random.default_rng(2)
    t0 = time.perf_counter()
    history = []
    for ep in range(a.epochs):
        order = rng.permutation(len(samples))
        tot = 0.0
        lr = a.lr * 0.5 * (1 + math.cos(math.pi * ep / a.epochs))
        for k in range(0, len(order), a.batch):
            idx = order[k:k + a.batch]
            B.lbm_net_zero_grads(net)
            for j in idx:
                inp, base, tgt, mask, H = samples[j]
                tot += B.lbm_net_backward(net, inp, base, tgt, mask, H, NX)
            B.lbm_net_adam_step(net, lr, grad_scale=1.0 / len(idx))
        history.append(tot / max(1, len(samples)))
    torch.cuda.synchronize()
    report["training"] = {"wall_s": time.perf_counter() - t0, "params": B.lbm_net_param_count(net),
                          "loss_first_epoch": history[0] if history else None,
                          "loss_last_epoch": history[-1] if history else None, "history": history}
    if a.out:
        B.lbm_net_save(net, a.out)

    def evaluator(dset, off):
        """Cases, network inputs and warm-field builder of a draw set whose coarse runs start at off."""
        cases = [(NX, round(NX * ar), re) for re, ar in dset]
        inps = [make_input(coarse[off + i], re, ar, NX, cases[i][1]) for i, (re, ar) in enumerate(dset)]

        def field(i, use_net):
            """(rho, ux, uy) of a warm start; None (start from rest) if the coarse run went non-finite."""
            nx, ny = NX, cases[i][1]
            if stat_c[off + i] == 3:
                return None
            inp, H = inps[i]
            out = torch.zeros((3, H, NX), dtype=torch.float32, device="cuda")
            if use_net:
                B.lbm_net_forward(net, inp, H, NX, out)
                if a.smooth > 0:
                    B.lbm_warm_smooth(out, ny, H, NX, a.smooth, torch.empty_like(out), st.cuda_stream)
            f = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
            B.lbm_warm_output(inp, out, nx, ny, H, U_LID, *f, st.cuda_stream)
            return f
        return cases, field

    # 5. fallback gate from the validation draws
    gate = None
    if val:
        vc, vfield = evaluator(val, len(train) + len(test))
        bv, v_rest, _, _ = batch_run(vc, a.dtype, a.tol, a.max_steps)
        B.lbm_batch_destroy(bv)
        bv, v_net, _, _ = batch_run(vc, a.dtype, a.tol, a.max_steps, lambda i: vfield(i, True), B.LBM_INIT_NEQ)
        B.lbm_batch_destroy(bv)
        gate, total = choose_gate([re for re, _ in val], v_rest, v_net, a.re_max + 1.0)
        report["gate"] = {"re_gate": gate, "val_total_rest": int(v_rest.sum()), "val_total_network": int(v_net.sum()),
                          "val_total_gated": int(total), "n_val": len(val)}

    # 6. evaluation: rest vs interpolated coarse vs network, all to the same tolerance
    ec, field_from = evaluator(test, len(train))
    res_t = np.array([re for re, _ in test])
    arm_list = [("rest", None, 0),
                ("coarse", lambda i: field_from(i, False), 0),
                ("coarse_neq", lambda i: field_from(i, False), B.LBM_INIT_NEQ),
                ("network", lambda i: field_from(i, True), 0),
                ("network_neq", lambda i: field_from(i, True), B.LBM_INIT_NEQ)]
    if gate is not None:
        arm_list.append(("network_gated", lambda i: field_from(i, True) if res_t[i] < gate else None, B.LBM_INIT_NEQ))
    arms = {}
    for name, init, flags in arm_list:
        b, done, status, wall = batch_run(ec, a.dtype, a.tol, a.max_steps, init, flags)
        r_end, _ = B.lbm_batch_residual(b, len(ec))
        if name == "rest":  # the converged fields measure the warm fields' velocity error
            steady = [[t.cpu().numpy() for t in moments(b, i, NX, c[1])] for i, c in enumerate(ec)]
        B.lbm_batch_destroy(b)
        arms[name] = {"steps": done.tolist(), "status": status.tolist(), "wall_s": wall,
                      "total_steps": int(done.sum()), "converged": int((status == 1).sum()),
                      "final_residual": r_end.tolist()}
    # relative L2 velocity error of the two warm fields against the converged run from rest
    verr = {"coarse": [], "network": []}
    for i in range(len(test)):
        _, sx, sy = steady[i]
        norm = np.sqrt((sx * sx + sy * sy).sum())
        for k, use_net in (("coarse", False), ("network", True)):
            f = field_from(i, use_net)
            if f is None:
                continue
            wx, wy = f[1].cpu().numpy(), f[2].cpu().numpy()
            verr[k].append(float(np.sqrt(((wx - sx) ** 2 + (wy - sy) ** 2).sum()) / norm))
    report["velocity_error"] = {k: {"median": float(np.median(v)), "max": float(np.max(v))} for k, v in verr.items() if v}
    # steps ratio of each warm arm over rest; a draw whose warm run hit the cap counts at the cap
    rest = np.array(arms["rest"]["steps"], dtype=float)
    ev = {"n": len(test), "rest_converged": arms["rest"]["converged"],
          "total_steps": {k: v["total_steps"] for k, v in arms.items()},
          "wall_s": {k: v["wall_s"] for k, v in arms.items()},
          "converged": {k: v["converged"] for k, v in arms.items()}, "ratio_over_rest": {}}
    ok = np.array(arms["rest"]["status"]) == 1
    for k in [n for n in arms if n != "rest"]:
        r = np.array(arms[k]["steps"], dtype=float)[ok] / rest[ok]
        band = {}
        for lo, hi in ((0, 400), (400, 700), (700, 1e9)):
            sel = (res_t[ok] >= lo) & (res_t[ok] < hi)
            if sel.any():
                band[f"Re_{lo}_{hi if hi < 1e9 else 'up'}"] = {"n": int(sel.sum()), "median": float(np.median(r[sel]))}
        ev["ratio_over_rest"][k] = {"median": float(np.median(r)), "mean": float(np.mean(r)),
                                    "fraction_faster": float(np.mean(r < 1)),
                                    "total_steps_ratio": float(np.array(arms[k]["steps"], dtype=float)[ok].sum()
                                                               / rest[ok].sum()),
                                    "by_re": band}
    report["evaluation"] = ev
    report["arms"] = arms
    report["draws_test"] = test
    B.lbm_net_destroy(net)
    return report


def main(argv=None):
    print(json.dumps(run(parser().parse_args(argv))), flush=True)


if __name__ == "__main__":
    main()
