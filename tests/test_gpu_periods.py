"""A periodic state of the Ar = 0.6 cavity against the paper's period (Table 3), GPU path.

500 x 300 nodes, Re = 6000, U = 0.1, FP32 shifted storage; u_x at the Sec. 3.3 observing point
(x, y) = (0.5, 0.3) every 100 steps for 1e6 steps; the last quarter of the series is classified
(paper_2211_05009_gb300.analysis) and its period, in steps times dt = dx = 1/500 (reading of the
unstated time unit: cavity width 1, dx = dt), is compared with Table 3's 21.08 within 3 %.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300.analysis import classify  # noqa: E402
from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table3_periods.txt")


def table3():
    out = {}
    for ln in open(GOLDEN):
        if ln.strip() and not ln.startswith("#"):
            ar, re, t = ln.split()
            out[(float(ar), float(re))] = float(t)
    return out


def test_ar06_re6000_period_matches_table3():
    nx, ar, re, every, steps = 500, 0.6, 6000.0, 100, 1_000_000
    want = table3()[(ar, re)]
    with Cavity(nx, round(nx * ar), Re=re, U=0.1, dtype="f32s") as cav:
        q, series = cav.probe(0.5, 0.3, every=every, cap=steps // every)
        cav.step(steps)
        ux = series.cpu().numpy()[:, 0]
    fs = classify(ux, every, 0.1, nx)
    assert fs.state == "periodic"
    period_time = fs.period_steps / nx  # steps x dt, dt = 1/500
    print(f"period {fs.period_steps:.0f} steps = {period_time:.3f} (Table 3: {want})")
    assert abs(period_time - want) < 0.03 * want


def test_eleven_table3_periods_in_one_batch():
    """Eleven Table 3 cavities (Ar 0.5 / 0.6 / 0.7, Re 5500-7500) stepped together in the batched
    persistent kernel for 1.2e6 steps, u_x at the Sec. 3.3 observing point every 100 steps: each
    is periodic by the classification rule and its period (steps x dt, dt = 1/500) is within 3 %
    of Table 3.  (Measured: 1.3-1.6 % below the paper's values for all eleven.)"""
    from paper_2211_05009_gb300 import binding as B
    from paper_2211_05009_gb300.analysis import observing_point
    want = table3()
    pairs = [(0.5, 6500.0), (0.5, 7000.0), (0.5, 7500.0), (0.6, 6000.0), (0.6, 6500.0), (0.6, 7000.0),
             (0.6, 7500.0), (0.7, 5500.0), (0.7, 6000.0), (0.7, 6500.0), (0.7, 7000.0)]
    nx, every, steps = 500, 100, 1_200_000
    cap = steps // every
    b = B.lbm_batch_create([nx] * len(pairs), [round(nx * a) for a, _ in pairs], [r for _, r in pairs],
                           [0.1] * len(pairs), "f32s")
    try:
        B.lbm_batch_set_stream(b, torch.cuda.current_stream().cuda_stream)
        series = torch.zeros((len(pairs), cap, 2), dtype=torch.float64, device="cuda")
        pts = [observing_point(a) for a, _ in pairs]
        B.lbm_batch_probe(b, [p[0] for p in pts], [p[1] for p in pts], every, series, cap)
        B.lbm_batch_step(b, steps)
        ser = series.cpu().numpy()
    finally:
        B.lbm_batch_destroy(b)
    for i, (ar, re) in enumerate(pairs):
        fs = classify(ser[i, :, 0], every, 0.1, nx)
        assert fs.state == "periodic", (ar, re, fs)
        t = fs.period_steps / nx
        print(f"Ar {ar} Re {re:.0f}: period {t:.3f} (Table 3: {want[(ar, re)]})")
        assert abs(t - want[(ar, re)]) < 0.03 * want[(ar, re)]
