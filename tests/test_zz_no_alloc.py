"""The allocation-free stream function (lbm_stream_function_static) against the context-based
one (lbm_stream_function), through the C ABI.

lbm_stream_function_static exists for callers that cannot call cudaMalloc (an application that
reserves all device memory at start-up, for instance); it keeps its scratch in a fixed device
array.  This file is collected last so that a run stopping at the first failure has run every
other test first; it must also pass on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import binding as B  # noqa: E402
from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402


def reference(cav):
    """psi field and (psi_min, xc, yc) from the context-based entry point, plus the device u_x."""
    psi_min, xc, yc, psi = cav.stream_function(psi=True)
    _, ux, _ = cav.moments()
    return ux, psi, (psi_min, xc, yc)


def static_call(ux, ny, nx):
    psi = torch.full((ny, nx), float("nan"), dtype=torch.float64, device="cuda")
    res = torch.full((3,), float("nan"), dtype=torch.float64, device="cuda")
    rc = B.lbm_stream_function_static(ux, nx, ny, psi, res, torch.cuda.current_stream().cuda_stream)
    assert rc == B.LBM_OK
    torch.cuda.synchronize()
    return psi, res.cpu().numpy()


def test_static_matches_context_entry_point_twice():
    """Two calls in a row (on two different fields and grid shapes): each must reproduce the
    context-based result -- Psi to 1e-12 and the same minimum node -- and the CPU oracle's
    stream function of the same u_x field (trapezoid rule from Psi = 0 on the bottom wall)."""
    for (nx, ny, steps) in [(200, 160, 700), (97, 133, 400)]:
        with Cavity(nx, ny, Re=400.0, U=0.1, dtype="f64") as cav:
            cav.step(steps)
            ux, psi_ref, (vmin, xc, yc) = reference(cav)
        psi, res = static_call(ux, ny, nx)
        assert torch.abs(psi - psi_ref).max().item() < 1e-12
        assert abs(res[0] - vmin) < 1e-12
        assert res[1] == xc and res[2] == yc
        ux_h = ux.cpu().numpy()
        psi_o, (omin, oi, oj), _ = O.stream_function(O.Params(nx, ny, 0.8, 0.1), ux_h)
        assert np.abs(psi.cpu().numpy() - psi_o).max() < 1e-12
        assert abs(res[0] - omin) < 1e-12
        assert res[1] == oi / nx and res[2] == oj / nx


def test_static_repeated_same_input_is_identical():
    with Cavity(64, 64, Re=100.0, U=0.1, dtype="f64") as cav:
        cav.step(300)
        ux, psi_ref, ref = reference(cav)
    a_psi, a = static_call(ux, 64, 64)
    b_psi, b = static_call(ux, 64, 64)
    assert np.array_equal(a, b) and torch.equal(a_psi, b_psi)
    assert abs(a[0] - ref[0]) < 1e-12


def test_static_rejects_grids_beyond_its_scratch():
    nx, ny = 8192, 4096  # needs more than LBM_STATIC_SCRATCH_DOUBLES
    assert nx * ((ny + 31) // 32) > B.LBM_STATIC_SCRATCH_DOUBLES
    ux = torch.zeros(16, dtype=torch.float64, device="cuda")  # never read: rejected up front
    res = torch.zeros(3, dtype=torch.float64, device="cuda")
    assert B.lbm_stream_function_static(ux, nx, ny, None, res) == B.LBM_ETOOBIG
    # fits the scratch, but one launch row per 32-row segment exceeds the grid's y limit
    nx, ny = 1, 3_000_000
    assert nx * ((ny + 31) // 32) + 2 * ((ny + 31) // 32) <= B.LBM_STATIC_SCRATCH_DOUBLES
    assert B.lbm_stream_function_static(ux, nx, ny, None, res) == B.LBM_ETOOBIG
    assert B.lbm_stream_function_static(None, 16, 16, None, res) == B.LBM_EINVAL
