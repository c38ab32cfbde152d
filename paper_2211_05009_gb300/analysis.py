"""Post-processing of observing-point time series (Sec. 3.3): flow-state classification and the
period of periodic states (Fig. 8-17, Table 3).

The paper judges the state by eye from U_x(t) and the U_x-U_y phase plot; this module states the
rule this library uses instead (host-side, on the probe series the GPU wrote):

  * the last `tail` fraction of the samples is analysed (transients excluded);
  * steady     -- the run met the Eq. 6 tolerance, or the peak-to-peak range of u_x over the tail
                  is below `steady_tol` * U;
  * periodic   -- the normalised autocorrelation of u_x - mean has, after its first zero crossing,
                  a maximum >= `acf_min` (0.95) and the successive maxima of u_x over the tail
                  differ by less than `amp_tol` (1 %) of the peak-to-peak range; the period is the
                  lag of that autocorrelation maximum (parabolic refinement), in steps;
  * aperiodic  -- otherwise.
Periods are also given in convective units T U / L (L = nx), since the paper's time unit in
Table 3 ("step*dt") is not stated.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class FlowState:
    state: str               # "steady", "periodic" or "aperiodic"
    period_steps: float | None
    period_convective: float | None
    amplitude: float         # peak-to-peak of u_x over the analysed tail
    acf_peak: float | None


def _autocorr(x: np.ndarray) -> np.ndarray:
    x = x - x.mean()
    n = len(x)
    f = np.fft.rfft(x, 2 * n)
    ac = np.fft.irfft(f * np.conj(f))[:n]
    return ac / ac[0] if ac[0] > 0 else ac


def classify(ux: np.ndarray, every: int, U: float, nx: int, converged: bool = False,
             tail: float = 0.25, steady_tol: float = 1e-6, acf_min: float = 0.95,
             amp_tol: float = 0.01) -> FlowState:
    """Classify a probe series u_x(t) sampled every `every` steps."""
    ux = np.asarray(ux, dtype=np.float64)
    seg = ux[int(len(ux) * (1.0 - tail)):]
    if len(seg) < 4:
        raise ValueError("series too short to classify")
    amp = float(seg.max() - seg.min())
    if converged or amp < steady_tol * abs(U):
        return FlowState("steady", None, None, amp, None)
    ac = _autocorr(seg)
    neg = np.nonzero(ac < 0)[0]
    if len(neg) == 0:
        return FlowState("aperiodic", None, None, amp, None)
    start = neg[0]
    lag = start + int(np.argmax(ac[start:len(ac) // 2])) if start < len(ac) // 2 else None
    if lag is None or lag <= 0 or lag + 1 >= len(ac):
        return FlowState("aperiodic", None, None, amp, None)
    peak = float(ac[lag])
    # parabolic refinement of the lag
    y0, y1, y2 = ac[lag - 1], ac[lag], ac[lag + 1]
    den = y0 - 2 * y1 + y2
    frac = 0.5 * (y0 - y2) / den if den != 0 else 0.0
    period = (lag + frac) * every
    # successive maxima of u_x: one per period window
    w = max(1, lag)
    maxima = [seg[i:i + w].max() for i in range(0, len(seg) - w + 1, w)]
    spread = (max(maxima) - min(maxima)) if maxima else np.inf
    if peak >= acf_min and spread < amp_tol * amp:
        return FlowState("periodic", period, period * U / nx, amp, peak)
    return FlowState("aperiodic", None, None, amp, peak)


def observing_point(ar: float) -> tuple[float, float]:
    """The observing point of Sec. 3.3 in width units: (0.5, 0.2) for Ar = 0.4, (0.5, 0.3) for
    Ar = 0.5 and 0.6, (0.5, 0.5) otherwise."""
    if abs(ar - 0.4) < 1e-9:
        return 0.5, 0.2
    if abs(ar - 0.5) < 1e-9 or abs(ar - 0.6) < 1e-9:
        return 0.5, 0.3
    return 0.5, 0.5
