"""The flow-state rule of paper_2211_05009_gb300.analysis on signals whose state is known."""
import numpy as np

from paper_2211_05009_gb300.analysis import classify, observing_point


def test_constant_signal_is_steady():
    s = classify(np.full(400, 0.0123), every=100, U=0.1, nx=500)
    assert s.state == "steady" and s.period_steps is None


def test_converged_run_is_steady():
    s = classify(np.sin(np.arange(400)), every=100, U=0.1, nx=500, converged=True)
    assert s.state == "steady"


def test_sinusoid_is_periodic_with_its_period():
    every, period = 100, 3137.0  # steps
    t = np.arange(4000) * every
    ux = 0.01 + 1e-3 * np.sin(2 * np.pi * t / period) + 3e-4 * np.sin(4 * np.pi * t / period + 1.0)
    s = classify(ux, every=every, U=0.1, nx=500)
    assert s.state == "periodic"
    assert abs(s.period_steps - period) < 0.02 * period
    assert abs(s.period_convective - period * 0.1 / 500) < 0.02 * period * 0.1 / 500


def test_drifting_periodic_signal_is_periodic():
    """A cycle on a slow linear drift (the wall mass leak of long runs) is still periodic."""
    every, period = 100, 5011.0
    t = np.arange(6000) * every
    ux = 0.02 + 2e-3 * np.sin(2 * np.pi * t / period) + 4e-8 * t
    s = classify(ux, every=every, U=0.1, nx=500)
    assert s.state == "periodic" and abs(s.period_steps - period) < 0.02 * period


def test_oscillation_below_plot_resolution_is_steady():
    """Peak-to-peak 4e-5 U: below the 1e-3 U an oscillation needs to show in a U_x plot."""
    t = np.arange(4000) * 100
    ux = 0.03 + 2e-6 * np.sin(2 * np.pi * t / 7000.0)
    s = classify(ux, every=100, U=0.1, nx=500)
    assert s.state == "steady" and s.amplitude < 1e-3 * 0.1


def test_modulated_cycle_is_aperiodic_with_its_dominant_period():
    """Amplitude modulation by an incommensurate slow cycle: not periodic, but the carrier period
    is reported as the dominant one."""
    every, period = 100, 3000.0
    t = np.arange(8000) * every
    ux = 0.02 + 2e-3 * np.sin(2 * np.pi * t / period) * (1 + 0.3 * np.sin(2 * np.pi * t / (period * 7.31)))
    s = classify(ux, every=every, U=0.1, nx=500)
    assert s.state == "aperiodic"
    assert s.dominant_period_steps is not None and abs(s.dominant_period_steps - period) < 0.03 * period


def test_incommensurate_and_noisy_signal_is_aperiodic():
    rng = np.random.default_rng(0)
    t = np.arange(4000, dtype=float)
    ux = np.sin(t / 7.3) + np.sin(t / (7.3 * np.sqrt(2))) + 0.5 * rng.normal(size=t.size)
    assert classify(ux, every=100, U=0.1, nx=500).state == "aperiodic"


def test_logistic_map_chaos_is_aperiodic():
    x = np.empty(4000)
    x[0] = 0.3
    for i in range(1, len(x)):
        x[i] = 3.9 * x[i - 1] * (1 - x[i - 1])
    assert classify(1e-3 * x, every=100, U=0.1, nx=500).state == "aperiodic"


def test_observing_points_of_sec_3_3():
    assert observing_point(0.4) == (0.5, 0.2)
    assert observing_point(0.5) == observing_point(0.6) == (0.5, 0.3)
    assert observing_point(1.2) == (0.5, 0.5)


def test_sweep_pairs_cover_every_state_the_paper_reports():
    """The sweep's paper pairs are exactly the periodic entries of Table 3 plus the Fig. 8-10
    cavities (golden files, transcribed from the paper), and its case list has no duplicates."""
    import os
    from paper_2211_05009_gb300 import sweep as S
    gold = os.path.join(os.path.dirname(__file__), "golden")
    t3 = {(float(a), float(r)) for a, r, _ in
          (ln.split() for ln in open(os.path.join(gold, "table3_periods.txt")) if ln[0].isdigit())}
    assert t3 == {(float(a), float(r)) for a, r in S.TABLE3_PAIRS} and len(t3) == 38
    st = {(float(a), float(r)) for r, a, *_ in
          (ln.split() for ln in open(os.path.join(gold, "states_sec33.txt")) if ln[0].isdigit())}
    assert st == {(float(a), float(r)) for a, r in S.FIG8_10_PAIRS} and len(st) == 21
    cases = S.cavity_list(500, [4000.0, 8000.0], [0.6, 1.2], 0.1, S.TABLE3_PAIRS + S.FIG8_10_PAIRS)
    keys = [(c["Ar"], c["Re"]) for c in cases]
    assert len(keys) == len(set(keys)) and all(c["ny"] == round(500 * c["Ar"]) for c in cases)
