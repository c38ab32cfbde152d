"""The GPU path run to the Eq. 6 steady state reproduces the paper's own square-cavity numbers
(Table 1, row c: 256 x 256 nodes, U = 0.1).  Values are read from tests/golden/.

The paper prints -Psi (its primary vortex is a maximum) normalised by U L, and centres as
node / 256.  The paper does not state its wall placement, corner treatment or output instant
beyond "steady" (Eq. 6 < 1e-6), so the check is loose: primary vortex strength within 3 % and
its centre within one node; secondary (corner) vortex strengths within 20 % -- the spread between
the paper's own row c and the literature rows a/b of the same table reaches 20 % there (Re = 1000,
lower-left vortex: 1.84e-4 against 2.31e-4) -- and their centres within two nodes.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_square_cavity_256.txt")


def table1():
    rows = {}
    for ln in open(GOLDEN):
        if ln.startswith("#") or not ln.strip():
            continue
        v = [float(t) for t in ln.split()]
        rows[int(v[0])] = v[1:]
    return rows


@pytest.mark.parametrize("Re", [400, 1000])
def test_table1_row_c(Re):
    want = table1()[Re]
    nx = ny = 256
    U = 0.1
    with Cavity(nx, ny, Re=float(Re), U=U, dtype="f64") as cav:
        ok, steps = cav.run_to_residual(1e-6, 2_000_000)
        assert ok, "no steady state"
        psi_min, xc, yc = cav.stream_function()
        (_, _, _), (ll, lli, llj) = cav.stream_function_window(0, nx // 2, 0, ny // 3)
        (_, _, _), (lr, lri, lrj) = cav.stream_function_window(nx // 2, nx, 0, ny // 3)
    scale = U * nx
    got = [-psi_min / scale, xc, yc, -ll / scale, lli / nx, llj / nx, -lr / scale, lri / nx, lrj / nx]
    print(f"Re={Re} steps={steps}")
    print("  paper:", want)
    print("  ours :", [round(v, 6) for v in got])
    # centres: the paper prints node/256 rounded to 4 digits
    node = lambda v: round(v * nx)  # noqa: E731
    assert abs(got[0] - want[0]) < 0.03 * want[0]
    assert abs(node(got[1]) - node(want[1])) <= 1 and abs(node(got[2]) - node(want[2])) <= 1
    for k in (3, 6):
        assert abs(got[k] - want[k]) < 0.20 * abs(want[k])
        assert abs(node(got[k + 1]) - node(want[k + 1])) <= 2 and abs(node(got[k + 2]) - node(want[k + 2])) <= 2
