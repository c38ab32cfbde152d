"""Post-processing of observing-point time series (Sec. 3.3): flow-state classification and the
period of periodic states (Fig. 8-17, Table 3).

The paper judges the state by eye from U_x(t) and the U_x-U_y phase plot; this module states the
rule this library uses instead (host-side, on the probe series the GPU wrote):

  * the last `tail` fraction of the samples is analysed (transients excluded), after removing its
    least-squares linear trend (the non-equilibrium-extrapolation walls leak mass at a steady
    rate, so long runs drift slowly under the oscillation);
  * steady     -- the run met the Eq. 6 tolerance, or the peak-to-peak range of the detrended
                  u_x is below `steady_tol` * U (1e-3: an oscillation that small does not show
                  in the paper's U_x plots);
  * periodic   -- the normalised autocorrelation of the detrended u_x has, after its first zero
                  crossing, a maximum >= `acf_min` (0.95), and the maxima of successive period
                  windows differ by less than `amp_tol` (2 %) of the range; the period is the
                  lag of that autocorrelation maximum (parabolic refinement), in steps;
  * aperiodic  -- otherwise; the lag of the autocorrelation maximum is still reported as the
                  dominant period when that maximum is >= 0.8 (modulated or drifting
                  oscillations whose main cycle can be read off).
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
    amplitude: float         # peak-to-peak of the detrended u_x over the analysed tail
    acf_peak: float | None
    dominant_period_steps: float | None = None  # autocorrelation lag when its peak >= 0.8


def _autocorr(x: np.ndarray) -> np.ndarray:
    x = x - x.mean()
    n = len(x)
    f = np.fft.rfft(x, 2 * n)
    ac = np.fft.irfft(f * np.conj(f))[:n]
    return ac / ac[0] if ac[0] > 0 else ac


def _detrend(x: np.ndarray, window: int = 1) -> np.ndarray:
    """x minus the least-squares line through the means of consecutive `window`-sample blocks
    (block means of a cycle of about `window` samples do not tilt with its phase, as a fit to the
    raw samples would: the regression slope of N whole sine cycles is ~1/N of the amplitude)."""
    nb = len(x) // window
    if nb < 2:
        window, nb = 1, len(x)
    m = x[:nb * window].reshape(nb, window).mean(axis=1)
    c = (np.arange(nb) + 0.5) * window - 0.5
    A = np.vstack([c, np.ones_like(c)]).T
    coef, *_ = np.linalg.lstsq(A, m, rcond=None)
    return x - (coef[0] * np.arange(len(x)) + coef[1])


def _acf_peak(ac: np.ndarray):
    """(lag, refined lag) of the autocorrelation maximum after its first zero crossing, or None."""
    neg = np.nonzero(ac < 0)[0]
    if len(neg) == 0 or neg[0] >= len(ac) // 2:
        return None
    lag = int(neg[0] + np.argmax(ac[neg[0]:len(ac) // 2]))
    if lag <= 0 or lag + 1 >= len(ac):
        return None
    y0, y1, y2 = ac[lag - 1], ac[lag], ac[lag + 1]
    den = y0 - 2 * y1 + y2
    return lag, lag + (0.5 * (y0 - y2) / den if den != 0 else 0.0)


def classify(ux: np.ndarray, every: int, U: float, nx: int, converged: bool = False,
             tail: float = 0.25, steady_tol: float = 1e-3, acf_min: float = 0.95,
             amp_tol: float = 0.02) -> FlowState:
    """Classify a probe series u_x(t) sampled every `every` steps."""
    ux = np.asarray(ux, dtype=np.float64)
    seg = ux[int(len(ux) * (1.0 - tail)):]
    if len(seg) < 4:
        raise ValueError("series too short to classify")
    if converged:
        return FlowState("steady", None, None, float(seg.max() - seg.min()), None)
    # the trend is fitted to per-cycle means (if there is a cycle), so that the oscillation
    # itself does not tilt it
    first = _acf_peak(_autocorr(seg))
    d = _detrend(seg, first[0] if first is not None else 1)
    amp = float(d.max() - d.min())
    if amp < steady_tol * abs(U):
        return FlowState("steady", None, None, amp, None)
    ac = _autocorr(d)
    pk = _acf_peak(ac)
    if pk is None:
        return FlowState("aperiodic", None, None, amp, None)
    lag, refined = pk
    peak = float(ac[lag])
    period = refined * every
    dominant = period if peak >= 0.8 else None
    # maxima of successive period windows
    maxima = [d[i:i + lag].max() for i in range(0, len(d) - lag + 1, lag)]
    spread = (max(maxima) - min(maxima)) if maxima else np.inf
    if peak >= acf_min and spread < amp_tol * amp:
        return FlowState("periodic", period, period * U / nx, amp, peak, period)
    return FlowState("aperiodic", None, None, amp, peak, dominant)


def observing_point(ar: float) -> tuple[float, float]:
    """The observing point of Sec. 3.3 in width units: (0.5, 0.2) for Ar = 0.4, (0.5, 0.3) for
    Ar = 0.5 and 0.6, (0.5, 0.5) otherwise."""
    if abs(ar - 0.4) < 1e-9:
        return 0.5, 0.2
    if abs(ar - 0.5) < 1e-9 or abs(ar - 0.6) < 1e-9:
        return 0.5, 0.3
    return 0.5, 0.5
