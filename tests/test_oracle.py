"""Pins of the FP64 oracle against what the mathematics fixes (no GPU).

Each test names the passage of Xiang & Shi (arXiv 2211.05009) or the closed form it checks.
A plausible slip in the oracle -- a wrong velocity, weight or sign, a transposed x/y, a pull
from the wrong side, a dropped equilibrium term, a wrong viscosity -- fails at least one.
"""
import math

import numpy as np
import pytest

import oracle as O
from tests import exact_cavity as EX

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


# ---------------------------------------------------------------- Eq. 2 / Eq. 3 moments
@pytest.mark.parametrize("rho,ux,uy", [(1.0, 0.0, 0.0), (1.07, 0.1, -0.03), (0.93, -0.05, 0.08)])
def test_feq_moments(rho, ux, uy):
    """Eq. 2 must reproduce rho (0th), rho u (1st) and rho/3 I + rho u u (2nd moment)."""
    f = O.feq(rho, ux, uy)
    assert abs(f.sum() - rho) < 1e-15
    assert abs((CX * f).sum() - rho * ux) < 1e-15
    assert abs((CY * f).sum() - rho * uy) < 1e-15
    assert abs((CX * CX * f).sum() - (rho / 3 + rho * ux * ux)) < 1e-15
    assert abs((CY * CY * f).sum() - (rho / 3 + rho * uy * uy)) < 1e-15
    assert abs((CX * CY * f).sum() - rho * ux * uy) < 1e-15


def test_feq_rest_state_is_weights():
    """At u = 0, f^eq_j = w_j rho with w = 4/9, 1/9 (axes), 1/36 (diagonals) (Sec. 2.1)."""
    f = O.feq(1.0, 0.0, 0.0)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    assert np.array_equal(f, w)


# ---------------------------------------------------------------- Eq. 1 invariants
def _random_field(p, seed):
    rng = np.random.default_rng(seed)
    w = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    return w * (1 + 0.1 * rng.uniform(-1, 1, size=(p.ny, p.nx, 9)))


def test_equilibrium_invariant_under_step():
    """A uniform equilibrium in a periodic box is a fixed point of stream + collide (Eq. 1)."""
    p = O.Params(7, 5, 0.7, 0.0, mode=O.PERIODIC)
    f = np.broadcast_to(O.feq(1.02, 0.04, -0.07), (5, 7, 9)).copy()
    g = O.run(p, f, 10)
    assert np.abs(g - f).max() < 1e-16 * 20


def test_bgk_conserves_mass_and_momentum_periodic():
    """Streaming moves populations and BGK keeps rho, rho u at every node, so on a periodic
    box the totals are conserved to rounding (Eq. 1, Eq. 3)."""
    p = O.Params(9, 6, 0.61, 0.0, mode=O.PERIODIC)
    f = _random_field(p, 0)
    g = O.step(p, f)
    for c in (np.ones(9), CX, CY):
        assert abs((g * c).sum() - (f * c).sum()) < 1e-13


def test_collision_conserves_moments_per_node():
    """Per node: the post-collision field has the moments of the streamed field."""
    p = O.Params(6, 6, 0.77, 0.0, mode=O.PERIODIC)
    f = _random_field(p, 1)
    g = O.step(p, f)
    streamed = np.empty_like(f)
    for j in range(9):
        streamed[..., j] = np.roll(np.roll(f[..., j], CY[j], axis=0), CX[j], axis=1)
    for c in (np.ones(9), CX, CY):
        assert np.abs((g * c).sum(-1) - (streamed * c).sum(-1)).max() < 1e-15


# ---------------------------------------------------------------- closed-form flows
def _tg_rate_error(N, tau=0.8, U0=1e-3):
    p = O.Params(N, N, tau, 0.0, mode=O.PERIODIC)
    k = 2 * np.pi / N
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    ux = -U0 * np.cos(k * X) * np.sin(k * Y)
    uy = U0 * np.sin(k * X) * np.cos(k * Y)
    rho = 1 - 3 * U0 ** 2 / 4 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    f = O.init_moments(p, rho, ux, uy)
    t0, t1 = N * N // 16, N * N // 16 + N * N // 8
    f = O.run(p, f, t0)
    a0 = O.moments(p, f)[1]
    f = O.run(p, f, t1 - t0)
    a1 = O.moments(p, f)[1]
    A0 = (a0 * ux).sum() / (ux * ux).sum()
    A1 = (a1 * ux).sum() / (ux * ux).sum()
    rate = -math.log(A1 / A0) / (t1 - t0)
    nu = (tau - 0.5) / 3  # Eq. 5 with c_s^2 = 1/3, dt = 1
    return rate / (2 * nu * k * k) - 1


def test_taylor_green_decay_rate_second_order():
    """Taylor-Green vortex decays as exp(-2 nu k^2 t) with nu = (tau - 1/2)/3 (Eq. 5); the
    relative rate error is O(N^-2), so doubling N divides it by ~4."""
    e = [_tg_rate_error(N) for N in (16, 32, 64)]
    assert abs(e[2]) < 5e-4
    for a, b in zip(e, e[1:]):
        assert 3.6 < a / b < 4.4


def test_couette_exact_with_nee_walls():
    """Plane Couette flow between a resting NEE wall and a moving NEE wall (Sec. 2.2 ii) is
    linear; the extrapolated non-equilibrium part is uniform there, so NEE is exact."""
    U, ny = 0.05, 9
    p = O.Params(4, ny, 1.0, U, mode=O.CHANNEL_NEE)
    f = O.run(p, O.init(p), 3000)
    rho, ux, uy = O.moments(p, f)
    y = np.arange(ny)
    assert np.abs(ux - U * y[:, None] / (ny - 1)).max() < 1e-12
    assert np.abs(uy).max() < 1e-13


def _poiseuille_error(ny, tau=0.8):
    nu = (tau - 0.5) / 3
    H = ny - 1
    F = 8 * nu * 1e-3 / H ** 2  # centre-line speed 1e-3
    p = O.Params(3, ny, tau, 0.0, mode=O.CHANNEL_NEE, Fx=F)
    f = O.run(p, O.init(p), int(3 * H * H / nu))
    ux = O.moments(p, f)[1][:, 1]
    y = np.arange(ny)
    exact = F / (2 * nu) * y * (H - y)
    return np.abs(ux - exact).max() / exact.max()


def test_body_force_channel_parabolic_second_order():
    """Body-force channel between resting NEE walls converges to the parabola
    u = F y (H - y) / (2 nu); the error falls ~4x per doubling of the resolution."""
    e = [_poiseuille_error(n) for n in (9, 17, 33)]
    assert e[2] < 2.5e-3
    for a, b in zip(e, e[1:]):
        assert 3.6 < a / b < 4.4


def test_bounce_back_cavity_conserves_mass():
    """With halfway bounce-back walls (test-only mode) every population that leaves comes
    back and the moving-lid terms cancel node by node: total mass is exact to rounding."""
    p = O.Params(12, 10, 0.6, 0.1, mode=O.CAVITY_BB)
    f0 = O.init(p)
    m0 = O.mass(p, f0)
    f = O.run(p, f0, 2000)
    assert abs(O.mass(p, f) - m0) / m0 < 1e-12


# ---------------------------------------------------------------- Sec. 2.2 cavity
def test_exact_rational_brute_force_8x8():
    """Three steps of an 8x8 cavity in exact arithmetic (push streaming, closed-form NEE,
    independent code) against the FP64 oracle. tau = 221/250 (config 1's 0.884), U = 1/10."""
    from fractions import Fraction as Fr

    nx = ny = 8
    tau, U = Fr(221, 250), Fr(1, 10)
    fs = EX.initial(nx, ny, U)
    p = O.Params(nx, ny, 0.884, 0.1)
    f = O.init(p)
    for _ in range(3):
        fs = EX.step(fs, nx, ny, tau, U)
        f = O.step(p, f)
    ex = np.array(EX.to_oracle_layout(fs, nx, ny), dtype=np.float64)
    assert np.abs(f - ex).max() / np.abs(ex).max() < 1e-15
    # the lid must have started moving fluid below it
    assert abs(O.moments(p, f)[1][ny - 2, nx // 2]) > 1e-3


def test_nee_closed_form_equals_set_then_collide():
    """Sec. 2.2 (ii) then Eq. 1 at a wall node equals f^eq(rho_f, u_w) + (1 - 1/tau) f^neq(x_f)
    (the form the GPU kernel evaluates), on a random field."""
    p = O.Params(7, 6, 0.9, 0.1)
    f = _random_field(p, 2)
    g = O.step(p, f)
    w = 1 / p.tau
    for (x, y) in [(0, 0), (3, 0), (6, 0), (0, 3), (6, 2), (0, 5), (3, 5), (6, 5)]:
        xf, yf = min(max(x, 1), p.nx - 2), min(max(y, 1), p.ny - 2)
        ff = np.array([f[yf - CY[j], xf - CX[j], j] for j in range(9)])
        r = ff.sum()
        u = ((CX * ff).sum() / r, (CY * ff).sum() / r)
        uw = (p.U, 0.0) if (y == p.ny - 1 and 0 < x < p.nx - 1) else (0.0, 0.0)
        want = O.feq(r, *uw) + (1 - w) * (ff - O.feq(r, *u))
        assert np.abs(g[y, x] - want).max() < 1e-15


def test_step_node_matches_step():
    p = O.Params(9, 7, 0.7, 0.1)
    f = _random_field(p, 3)
    g = O.step(p, f)
    for y in range(p.ny):
        for x in range(p.nx):
            assert np.array_equal(O.step_node(p, f, x, y), g[y, x])


def test_mirror_symmetry():
    """Reversing the lid mirrors the flow in x: u_x(x) = -u_x'(nx-1-x), u_y(x) = u_y'(nx-1-x).
    Catches x/y transpositions and wrong signs in the velocity table."""
    p = O.Params(11, 8, 0.75, 0.1)
    q = O.Params(11, 8, 0.75, -0.1)
    f = O.run(p, O.init(p), 200)
    g = O.run(q, O.init(q), 200)
    r1, ux1, uy1 = O.moments(p, f)
    r2, ux2, uy2 = O.moments(q, g)
    assert np.abs(r1 - r2[:, ::-1]).max() < 1e-14
    assert np.abs(ux1 + ux2[:, ::-1]).max() < 1e-14
    assert np.abs(uy1 - uy2[:, ::-1]).max() < 1e-14


def test_initial_condition():
    """Sec. 2.2 (i): rho = 1 everywhere, u = 0 except u_x = U on the lid."""
    p = O.Params(6, 5, 0.8, 0.1)
    rho, ux, uy = O.moments(p, O.init(p))
    assert np.abs(rho - 1).max() < 1e-15
    want = np.zeros((5, 6))
    want[4, 1:5] = 0.1
    assert np.abs(ux - want).max() < 1e-16 and np.abs(uy).max() < 1e-16


def test_re_tau_relation():
    """Re = U L / nu (Sec. 1) with L = nx and nu = (tau - 1/2)/3 (Eq. 5): 128 nodes, Re = 100,
    U = 0.1 gives nu = 0.128 and tau = 0.884."""
    p = O.Params.from_re(128, 128, 100.0, 0.1)
    assert abs(p.tau - 0.884) < 1e-15


# ---------------------------------------------------------------- Eq. 6, Psi
def test_residual_eq6():
    rng = np.random.default_rng(4)
    ux, uy = rng.normal(size=(2, 5, 7))
    assert abs(O.residual(1.5 * ux, 1.5 * uy, ux, uy) - 0.5) < 1e-15
    assert O.residual(ux, uy, ux, uy) == 0.0


def test_stream_function_exact_for_piecewise_linear_profile():
    """Trapezoid integration of u_x = dPsi/dy is exact for linear u_x: Psi(y) = a y + b y^2/2."""
    p = O.Params(4, 6, 0.8, 0.1)
    y = np.arange(6.0)
    a, b = -0.3, 0.1
    ux = np.repeat((a + b * y)[:, None], 4, axis=1)
    psi, (vmin, imin, jmin), (vmax, _, _) = O.stream_function(p, ux)
    assert np.abs(psi - (a * y + b * y * y / 2)[:, None]).max() < 1e-15
    assert (imin, jmin) == (0, 3) and abs(vmin - (-0.45)) < 1e-15


def test_nee_mass_drift_is_small_and_reported():
    """NEE is not mass-conserving; the drift is measured, not asserted zero. It must stay a
    small fraction of the mass over a short run."""
    p = O.Params.from_re(32, 32, 100.0, 0.1)
    f0 = O.init(p)
    f = O.run(p, f0, 500)
    drift = (O.mass(p, f) - O.mass(p, f0)) / O.mass(p, f0)
    assert abs(drift) < 1e-2


# ---------------------------------------------------------------- first-order non-equilibrium start
def _quadratic_fields(nx, ny, seed):
    rng = np.random.default_rng(seed)
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    a = rng.uniform(-1, 1, (2, 6)) * np.array([1e-2, 1e-2, 1e-4, 1e-4, 1e-4, 1e-2])

    def quad(c):  # value and exact derivatives of c0 x + c1 y + c2 x^2 + c3 xy + c4 y^2 + c5
        v = c[0] * X + c[1] * Y + c[2] * X * X + c[3] * X * Y + c[4] * Y * Y + c[5]
        return v, c[0] + 2 * c[2] * X + c[3] * Y, c[1] + c[3] * X + 2 * c[4] * Y

    ux, dxux, dyux = quad(a[0])
    uy, dxuy, dyuy = quad(a[1])
    rho = 1 + 0.01 * np.sin(0.3 * X + 0.2 * Y)
    return rho, ux, uy, (dxux, dyux, dxuy, dyuy)


def test_neq_start_keeps_the_moments():
    """The non-equilibrium part carries no mass and no momentum: sum f = rho, sum c f = rho u."""
    p = O.Params(13, 9, 0.7, 0.1)
    rho, ux, uy, _ = _quadratic_fields(13, 9, 3)
    f = O.init_moments_neq(p, rho, ux, uy)
    assert np.abs(f.sum(-1) - rho).max() < 1e-14
    assert np.abs((f * CX).sum(-1) - rho * ux).max() < 1e-14
    assert np.abs((f * CY).sum(-1) - rho * uy).max() < 1e-14


@pytest.mark.parametrize("tau", [0.55, 0.9, 1.7])
def test_neq_start_stress_closed_form(tau):
    """Second moment of the added part, from sum_j w_j c_a c_b c_c c_d = c_s^4 (three deltas):
    Pi*_ab - Pi^eq_ab = -(tau - 1) rho c_s^2 (d_a u_b + d_b u_a), every node including the ring
    (the one-sided end differences are exact for these quadratic fields)."""
    nx, ny = 11, 14
    p = O.Params(nx, ny, tau, 0.1)
    rho, ux, uy, (dxux, dyux, dxuy, dyuy) = _quadratic_fields(nx, ny, 5)
    d = O.init_moments_neq(p, rho, ux, uy) - O.init_moments(p, rho, ux, uy)
    cs2 = 1.0 / 3.0
    k = -(tau - 1) * rho * cs2
    for pab, exact in (((d * CX * CX).sum(-1), k * 2 * dxux), ((d * CY * CY).sum(-1), k * 2 * dyuy),
                       ((d * CX * CY).sum(-1), k * (dxuy + dyux))):
        assert np.abs(pab - exact).max() < 1e-14 + 1e-11 * np.abs(exact).max()


def _tg_start_error(neq, N=32, tau=1.2, U0=1e-3, t=6):
    p = O.Params(N, N, tau, 0.0, mode=O.PERIODIC)
    k = 2 * np.pi / N
    X, Y = np.meshgrid(np.arange(N), np.arange(N))
    ux = -U0 * np.cos(k * X) * np.sin(k * Y)
    uy = U0 * np.sin(k * X) * np.cos(k * Y)
    rho = 1 - 3 * U0 ** 2 / 4 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    f = (O.init_moments_neq if neq else O.init_moments)(p, rho, ux, uy)
    f = O.run(p, f, t)
    nu = (tau - 0.5) / 3
    inner = (slice(2, -2), slice(2, -2))  # away from the one-sided end differences
    return np.abs(O.moments(p, f)[1] - ux * math.exp(-2 * nu * k * k * t))[inner].max() / U0


def test_neq_start_removes_the_initial_layer():
    """Taylor-Green vortex: started at equilibrium the populations first have to build their
    stress, which perturbs u; started with the Chapman-Enskog stress, u follows the closed-form
    decay from the first step.  A wrong sign or scale of the added part fails this."""
    e_eq, e_neq = _tg_start_error(False), _tg_start_error(True)
    assert e_neq < e_eq / 5, (e_eq, e_neq)


def test_openmp_build_is_bitwise_the_plain_build():
    """The all-core build of the same C source (used to time the oracle on every host core)
    computes every node as the plain build does: fields bitwise equal after 40 steps of a ragged
    cavity with moving lid corners, started from perturbed populations."""
    p = O.Params(67, 41, 0.56, 0.1, corner_moving=True)
    f0 = _random_field(p, 1)
    a = O.run(p, f0, 40)
    b = O.run(p, f0, 40, openmp=True)
    assert np.array_equal(a, b)
    assert O.threads() == 1 and O.threads(openmp=True) >= 1
