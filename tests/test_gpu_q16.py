"""LBM_Q16S storage (the 16-bit code of tests/q16_ref.py) on the GPU, through the C ABI.

  * the code: populations written with lbm_set_populations and read back with
    lbm_get_populations are exactly the reference's encode/decode (bit-exact);
  * the cavity of the precision study (2048^2, Re 8000, U 0.05) after 2e4 steps: velocity within
    1e-3 U of the FP64 GPU run (itself pinned to the oracle), the primary-vortex minimum of Psi
    within 1e-3 in the paper's normalisation Psi / (U L), its centre within 2 nodes (1e-3 of the
    width); binary16 and bfloat16 storage miss the velocity bound and are expected failures;
  * out-of-range values make the next checkpoint report divergence; save/load round trip.
"""
import os
import tempfile

import numpy as np
import pytest

from tests import q16_ref as Q
from tests.inputs import uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import binding as B  # noqa: E402
from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def test_codes_match_the_reference_bit_for_bit():
    nx, ny, U = 70, 37, 0.07
    S = np.array([Q.scale(j, U) for j in range(9)])
    r = uniform(11, (9, ny, nx))
    # deviations over the whole range, including saturation, exact zeros and grid midpoints; on a
    # 2^-25 S lattice, so that h 2^-124 / S, an FP32 subnormal below S/4, is exact and the code is
    # the one rounding of h (off that lattice the library rounds twice there, rarely differently)
    h = S[:, None, None] * np.round(2.3 * r * 2.0 ** 25) * 2.0 ** -25
    h[:, 0, :5] = 0.0
    h[1, 1, :4] = (Q.values()[[100, 101, 5000, 20001]] + Q.values()[[101, 102, 5001, 20002]]) / 2 * S[1]
    f_in = W[:, None, None] + h
    with Cavity(nx, ny, Re=100.0, U=U, dtype="q16s") as cav:
        cav.set_populations(f_in)
        got = cav.populations(host=True)
    for j in range(9):
        h32 = (f_in[j] - W[j]).astype(np.float32).astype(np.float64)  # what the library encodes
        want = Q.decode(Q.encode(h32, S[j]), S[j]) + W[j]
        assert np.array_equal(got[j], want), j


@pytest.fixture(scope="module")
def f64_run_2048():
    nx = ny = 2048
    with Cavity(nx, ny, Re=8000.0, U=0.05, dtype="f64") as cav:
        cav.step(20_000)
        _, ux, uy = cav.moments()
        psi = cav.stream_function()
    return ux, uy, psi


@pytest.mark.parametrize("dtype", [
    "q16s",
    pytest.param("f16s", marks=pytest.mark.xfail(
        strict=True, reason="binary16 storage misses 1e-3 U in this cavity (about 5e-3 U after 2e4 "
                            "steps, 1.5e-2 U after 2e5)")),
    pytest.param("bf16s", marks=pytest.mark.xfail(
        strict=True, reason="bfloat16 storage misses 1e-3 U in this cavity (about 8e-2 U after 2e4 "
                            "steps, 2.7e-1 U after 2e5)"))])
def test_precision_study_cavity_2048_re8000(f64_run_2048, dtype):
    ux0, uy0, (pmin0, xc0, yc0) = f64_run_2048
    nx, U = 2048, 0.05
    with Cavity(nx, nx, Re=8000.0, U=U, dtype=dtype) as cav:
        cav.step(20_000)
        _, ux, uy = cav.moments()
        pmin, xc, yc = cav.stream_function()
    du = float(torch.maximum((ux - ux0).abs(), (uy - uy0).abs()).max())
    dpsi = abs(pmin - pmin0) / (U * nx)
    dc = max(abs(xc - xc0), abs(yc - yc0)) * nx
    print(f"{dtype}: max|du| = {du / U:.3e} U, Psi_min {pmin:.6f} vs {pmin0:.6f} "
          f"({dpsi:.2e} of U L), centre {dc:.0f} nodes")
    assert du <= 1e-3 * U
    assert dpsi <= 1e-3
    assert dc <= 2


def test_out_of_range_reports_divergence():
    nx, ny, U = 24, 20, 0.1
    # density 1.5 at rest: w_j / 2 is far beyond every direction's largest code until the reference
    # density has followed the mass (first checkpoint), so the checkpoint step saturates
    f0 = np.broadcast_to(1.5 * W[:, None, None], (9, ny, nx)).copy()
    with Cavity(nx, ny, Re=100.0, U=U, dtype="q16s") as cav:
        cav.set_populations(f0)
        cav.step(100)
        with pytest.raises(B.LBMError) as e:
            cav.residual()
        assert e.value.code == B.LBM_EDIVERGED


def test_save_load_round_trip_and_reference_density():
    """A continued run is bitwise the uninterrupted one; the reference density follows the mass."""
    nx, ny = 61, 45
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "q.bin")
        with Cavity(nx, ny, Re=300.0, U=0.1, dtype="q16s") as a:
            a.step(2000)
            fa = a.populations(host=True)
            ma = a.mass()
        with Cavity(nx, ny, Re=300.0, U=0.1, dtype="q16s") as b:
            b.step(1000)
            b.save(path)
        with Cavity(nx, ny, Re=300.0, U=0.1, dtype="q16s") as c:
            c.load(path)
            c.step(1000)
            assert np.array_equal(c.populations(host=True), fa)
    # mass from the stored codes follows the FP64 run (the walls leak some 20 mass units here)
    with Cavity(nx, ny, Re=300.0, U=0.1, dtype="f64") as r:
        r.step(2000)
        assert abs(ma - r.mass()) < 1e-5 * nx * ny


def test_batch_rejects_q16():
    with pytest.raises(B.LBMError) as e:
        B.lbm_batch_create([16], [16], [100.0], [0.1], "q16s")
    assert e.value.code == B.LBM_EINVAL
