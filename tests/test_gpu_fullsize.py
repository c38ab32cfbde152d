"""Full-size checks in the launch configuration the benchmark times (2048 x 2048, FP32 shifted
storage, Re = 8000, U = 0.05): one step of the GPU is compared with the oracle at sampled nodes
(all corners and their neighbours, ring nodes, rows under the lid, random interior nodes),
starting from the GPU's own stored state; the 500 x (500 Ar) cavities are checked the same way."""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402


def sample_nodes(nx, ny, n_random, seed):
    rng = np.random.default_rng(seed)
    pts = set()
    for x in (0, 1, 2, nx - 3, nx - 2, nx - 1):
        for y in (0, 1, 2, ny - 3, ny - 2, ny - 1):
            pts.add((x, y))
    for x in rng.integers(0, nx, 64):
        pts.update({(int(x), 0), (int(x), 1), (int(x), ny - 2), (int(x), ny - 1)})
    for y in rng.integers(0, ny, 64):
        pts.update({(0, int(y)), (1, int(y)), (nx - 2, int(y)), (nx - 1, int(y))})
    for x, y in zip(rng.integers(0, nx, n_random), rng.integers(0, ny, n_random)):
        pts.add((int(x), int(y)))
    return sorted(pts)


@pytest.mark.parametrize("nx,ny,Re,U,warm", [
    (2048, 2048, 8000.0, 0.05, 300),
    (500, 500, 6000.0, 0.1, 200),
    (500, 1000, 8000.0, 0.1, 200),
    (500, 200, 4000.0, 0.1, 200),
])
def test_fullsize_step_sampled(nx, ny, Re, U, warm):
    p = O.Params.from_re(nx, ny, Re, U)
    with Cavity(nx, ny, Re=Re, U=U, dtype="f32s") as cav:
        cav.step(warm)
        fin = cav.populations(host=True)
        cav.step(1)
        fout = cav.populations(host=True)
        assert np.isfinite(cav.mass())
    fin_aos = O.from_soa(fin)
    del fin
    worst = 0.0
    for (x, y) in sample_nodes(nx, ny, 3000, seed=0):
        ref = O.step_node(p, fin_aos, x, y)
        got = fout[:, y, x]
        worst = max(worst, float(np.max(np.abs(got - ref) / np.abs(ref))))
    print(f"{nx}x{ny}: one-step sampled max rel err {worst:.3e}")
    assert worst < 2e-6


def test_fullsize_long_run_properties():
    """1000 steps at 2048^2: the Eq. 6 residual and the mass are finite, the flow has started
    under the lid, the lid row carries u = U, and the primary vortex sits under the lid."""
    nx = ny = 2048
    with Cavity(nx, ny, Re=8000.0, U=0.05, dtype="f32s") as cav:
        m0 = cav.mass()
        cav.step(1000)
        r = cav.residual()
        m1 = cav.mass()
        rho, ux, uy = (t.cpu().numpy() for t in cav.moments())
        psi_min, xc, yc = cav.stream_function()
    assert np.isfinite(r) and 0 < r < 1
    assert abs(m1 - m0) / m0 < 1e-3
    assert np.abs(ux[-1, 1:-1] - 0.05).max() < 1e-6
    assert np.abs(uy[-1]).max() < 1e-6 and np.abs(ux[0]).max() < 1e-6
    assert psi_min < 0 and yc > 0.9
