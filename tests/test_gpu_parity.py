"""GPU (sm_103a) path against the FP64 oracle, element by element, through the C ABI.

Tolerances (from the accuracy targets of the method's GPU path):
  FP64 storage          max |f_gpu - f_ref| / |f_ref| <= 1e-12 (f >= w_min rho > 0)
  FP32, FP32 shifted    max |u_gpu - u_ref| <= 1e-5 U
  16-bit storage        max |u_gpu - u_ref| <= 1e-3 U over a short run (LBM_Q16S, binary16; bfloat16
                        misses it and is marked as an expected failure with its measured error)
"""
import os
import tempfile

import numpy as np
import pytest

import oracle as O
from tests.inputs import uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import binding as B  # noqa: E402
from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def gpu_state(cav: Cavity):
    f = cav.populations(host=True)
    rho, ux, uy = cav.moments(host=True)
    return f, rho, ux, uy


def oracle_state(p: O.Params, steps: int, f0=None):
    f = O.run(p, O.init(p) if f0 is None else f0, steps)
    rho, ux, uy = O.moments(p, f)
    return O.to_soa(f), rho, ux, uy


def make(nx, ny, tau, U, dtype, corners=False):
    return Cavity(nx, ny, tau=tau, U=U, dtype=dtype, corners_moving=corners)


def test_create_flags_takes_re_in_the_library():
    """lbm_create_flags(Re, LBM_FLAG_LID_CORNERS_MOVING): tau from Re in the library (Eq. 5,
    L = nx), populations equal the oracle's run of the same Re with moving lid corners."""
    nx, ny, Re, U, steps = 129, 40, 80.0, 0.1, 300
    p = O.Params.from_re(nx, ny, Re, U, corner_moving=True)
    with Cavity(nx, ny, Re=Re, U=U, dtype="f64", corners_moving=True) as cav:
        assert cav.info.flags == B.LBM_FLAG_LID_CORNERS_MOVING
        assert abs(cav.tau - p.tau) < 1e-15
        cav.step(steps)
        f, _, _, _ = gpu_state(cav)
    fr, _, _, _ = oracle_state(p, steps)
    assert (np.abs(f - fr) / np.abs(fr)).max() < 1e-12


# ---------------------------------------------------------------- FP64 parity
@pytest.mark.parametrize("nx,ny,steps,corners", [
    (128, 128, 1000, False),   # square cavity, Re = 100 (tau = 0.884)
    (133, 77, 600, False),     # ragged: several warps per row, odd sizes
    (129, 40, 300, True),      # right wall lands on a warp boundary; moving lid corners
    (3, 3, 50, False),         # smallest cavity
    (5, 4, 80, False),
    (66, 9, 200, False),       # right wall in the last slot of a lane (FP64: 2 nodes per lane)
])
def test_f64_populations_match_oracle(nx, ny, steps, corners):
    tau = 3 * 0.1 * nx / 100 + 0.5 if nx >= 100 else 0.8
    p = O.Params(nx, ny, tau, 0.1, corner_moving=corners)
    with make(nx, ny, tau, 0.1, "f64", corners) as cav:
        cav.step(steps)
        f, rho, ux, uy = gpu_state(cav)
    fr, rr, uxr, uyr = oracle_state(p, steps)
    assert (np.abs(f - fr) / np.abs(fr)).max() < 1e-12
    assert np.abs(ux - uxr).max() < 1e-13 and np.abs(uy - uyr).max() < 1e-13
    assert np.abs(rho - rr).max() < 1e-13


def test_config1_full_run_f64():
    """128 x 128, Re = 100, U = 0.1, FP64, 10,000 steps: fields and the stream-function minimum."""
    nx = ny = 128
    p = O.Params.from_re(nx, ny, 100.0, 0.1)
    with Cavity(nx, ny, Re=100.0, U=0.1, dtype="f64") as cav:
        cav.step(10_000)
        f, rho, ux, uy = gpu_state(cav)
        psi_min, xc, yc, psi = cav.stream_function(psi=True, host=True)
        r = cav.residual()
    fr, rr, uxr, uyr = oracle_state(p, 10_000)
    assert (np.abs(f - fr) / np.abs(fr)).max() < 1e-12
    assert np.abs(ux - uxr).max() < 1e-12 * 0.1
    psir, (vmin, i, j), _ = O.stream_function(p, uxr)
    assert np.abs(psi - psir).max() < 1e-12
    assert abs(psi_min - vmin) < 1e-12 and (xc, yc) == (i / nx, j / nx)
    assert 0 < r < 1e-2


# ---------------------------------------------------------------- reduced precision
@pytest.mark.parametrize("dtype", ["f32", "f32s"])
@pytest.mark.parametrize("nx,ny,Re,steps", [(133, 77, 400.0, 1000), (500, 500, 4000.0, 1000)])
def test_fp32_velocity_matches_oracle(dtype, nx, ny, Re, steps):
    p = O.Params.from_re(nx, ny, Re, 0.1)
    with Cavity(nx, ny, Re=Re, U=0.1, dtype=dtype) as cav:
        cav.step(steps)
        _, rho, ux, uy = gpu_state(cav)
    _, rr, uxr, uyr = oracle_state(p, steps)
    err = max(np.abs(ux - uxr).max(), np.abs(uy - uyr).max())
    print(f"{dtype} {nx}x{ny} Re={Re}: max|du| = {err:.3e} = {err / 0.1:.3e} U")
    assert err <= 1e-5 * 0.1


def test_fp32s_rectangular_ar2_re8000():
    """500 x 1000 (Ar = 2), Re = 8000, FP32 shifted storage, first 1000 steps vs the oracle."""
    nx, ny, Re = 500, 1000, 8000.0
    p = O.Params.from_re(nx, ny, Re, 0.1)
    with Cavity(nx, ny, Re=Re, U=0.1, dtype="f32s") as cav:
        cav.step(1000)
        _, rho, ux, uy = gpu_state(cav)
    _, rr, uxr, uyr = oracle_state(p, 1000)
    err = max(np.abs(ux - uxr).max(), np.abs(uy - uyr).max())
    print(f"f32s 500x1000 Re=8000: max|du| = {err / 0.1:.3e} U")
    assert err <= 1e-5 * 0.1


@pytest.mark.parametrize("dtype", [
    "q16s", "f16s",
    pytest.param("bf16s", marks=pytest.mark.xfail(
        strict=True, reason="bfloat16 storage misses the 1e-3 U bound: 4.7e-3 U here (and 2.7e-1 U "
                            "after 2e5 steps of the 2048^2 Re 8000 cavity)"))])
def test_16bit_storage_velocity_error(dtype):
    """Reduced-precision storage within 1e-3 U of the FP64 oracle over a short run."""
    nx, ny, Re, steps = 133, 77, 400.0, 300
    p = O.Params.from_re(nx, ny, Re, 0.1)
    with Cavity(nx, ny, Re=Re, U=0.1, dtype=dtype) as cav:
        cav.step(steps)
        _, rho, ux, uy = gpu_state(cav)
    _, rr, uxr, uyr = oracle_state(p, steps)
    err = max(np.abs(ux - uxr).max(), np.abs(uy - uyr).max())
    print(f"{dtype} {nx}x{ny} Re={Re} {steps} steps: max|du| = {err / 0.1:.3e} U")
    assert err <= 1e-3 * 0.1


# ---------------------------------------------------------------- arbitrary input fields
@pytest.mark.parametrize("dtype,tol", [("f64", 1e-12), ("f32", 2e-6), ("f32s", 2e-6)])
def test_random_populations_one_step(dtype, tol):
    """Random populations w (1 + 0.1 r) in, one step, every node out (seed 0)."""
    nx, ny = 70, 37
    f0 = W[:, None, None] * (1 + 0.1 * uniform(0, (9, ny, nx)))
    p = O.Params(nx, ny, 0.7, 0.1)
    with make(nx, ny, 0.7, 0.1, dtype) as cav:
        cav.set_populations(f0)
        if dtype == "f64":
            fin = f0
        else:  # the oracle starts from what the GPU stored
            fin = cav.populations(host=True)
        cav.step(1)
        f1 = cav.populations(host=True)
    ref = O.to_soa(O.step(p, O.from_soa(fin)))
    err = (np.abs(f1 - ref) / np.abs(ref)).max()
    print(f"{dtype}: one-step max rel err {err:.3e}")
    assert err < tol


def test_set_moments_gives_equilibrium():
    nx, ny = 40, 30
    r = uniform(1, (3, ny, nx))
    rho, ux, uy = 1 + 0.01 * r[0], 0.05 * r[1], 0.05 * r[2]
    p = O.Params(nx, ny, 0.8, 0.1)
    with make(nx, ny, 0.8, 0.1, "f64") as cav:
        cav.set_moments(rho, ux, uy)
        f = cav.populations(host=True)
        assert cav.step_count == 0
    ref = O.to_soa(O.init_moments(p, rho, ux, uy))
    assert np.abs(f - ref).max() < 1e-16 * 8


def test_set_moments_keeps_graphs_and_matches_a_fresh_context():
    """Re-seeding a running context (whose 100-step graphs exist) with lbm_set_moments gives, over
    the next 200 steps, bitwise the populations, Eq. 6 residual and probe series of a fresh context
    seeded the same way: the graphs it keeps (no probe moved) are the ones a fresh context builds."""
    nx, ny, Re, U = 96, 70, 400.0, 0.1
    st = torch.cuda.current_stream().cuda_stream
    cap, every = 200, 2
    out = []
    for fresh in (False, True):
        ctx = B.lbm_create(nx, ny, Re, U, "f32s")
        try:
            B.lbm_set_stream(ctx, st)
            series = torch.full((cap, 2), float("nan"), dtype=torch.float64, device="cuda")
            B.lbm_probe(ctx, 0.5, 0.4, every, series, cap)
            seed = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
            if fresh:
                seed_ctx = B.lbm_create(nx, ny, Re, U, "f32s")
                B.lbm_set_stream(seed_ctx, st)
                B.lbm_step(seed_ctx, 300)
                B.lbm_moments(seed_ctx, *seed)
                B.lbm_destroy(seed_ctx)
            else:
                B.lbm_step(ctx, 300)  # builds and replays the graphs
                B.lbm_moments(ctx, *seed)
            B.lbm_set_moments(ctx, *seed)
            B.lbm_step(ctx, 200)
            r = B.lbm_residual(ctx)
            f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
            B.lbm_get_populations(ctx, f)
            torch.cuda.synchronize()
            out.append((f.cpu(), r, series[:200 // every].cpu()))
        finally:
            B.lbm_destroy(ctx)
    (f0, r0, s0), (f1, r1, s1) = out
    assert torch.equal(f0, f1) and r0 == r1 and torch.equal(s0, s1)
    assert torch.isfinite(s0).all()


@pytest.mark.parametrize("dtype", ["f64", "f32s", "q16s"])
def test_moments_through_pinned_host_buffers_equal_the_device_path(dtype):
    """lbm_set_moments from, and lbm_moments into, page-locked host buffers (read and written by the
    kernels over the host link) give bitwise what device buffers give."""
    nx, ny = 200, 130
    st = torch.cuda.current_stream().cuda_stream
    r = uniform(5, (3, ny, nx))
    seed = [1 + 0.01 * r[0], 0.05 * r[1], 0.05 * r[2]]
    out = []
    for pinned in (False, True):
        ctx = B.lbm_create(nx, ny, 300.0, 0.1, dtype)
        try:
            B.lbm_set_stream(ctx, st)
            if pinned:
                src = [torch.tensor(a).pin_memory() for a in seed]
                dst = [torch.full((ny, nx), float("nan"), dtype=torch.float64).pin_memory() for _ in range(3)]
            else:
                src = [torch.tensor(a, device="cuda") for a in seed]
                dst = [torch.full((ny, nx), float("nan"), dtype=torch.float64, device="cuda") for _ in range(3)]
            B.lbm_set_moments(ctx, *src)
            B.lbm_step(ctx, 150)
            B.lbm_moments(ctx, *dst)
            torch.cuda.synchronize()
            out.append([d.cpu() for d in dst])
        finally:
            B.lbm_destroy(ctx)
    for a, b in zip(*out):
        assert torch.isfinite(a).all() and torch.equal(a, b)


@pytest.mark.parametrize("dtype,tol", [("f64", 1e-13), ("f32s", 3e-7), ("f32", 3e-7), ("f16s", 2e-3)])
def test_set_moments_neq_matches_oracle(dtype, tol):
    """LBM_INIT_NEQ: f^eq plus (1 - 1/tau) times the first-order Chapman-Enskog part, on
    random fields (gradients at every node including the ring), then 60 steps (f64)."""
    nx, ny, tau = 37, 29, 0.9
    r = uniform(2, (3, ny, nx))
    rho, ux, uy = 1 + 0.01 * r[0], 0.05 * r[1], 0.05 * r[2]
    p = O.Params(nx, ny, tau, 0.1)
    ref0 = O.init_moments_neq(p, rho, ux, uy)
    with make(nx, ny, tau, 0.1, dtype) as cav:
        cav.set_moments(rho, ux, uy, neq=True)
        f = cav.populations(host=True)
        assert np.abs(f - O.to_soa(ref0)).max() < tol * 1.0
        if dtype == "f64":
            cav.step(60)
            ref = O.to_soa(O.run(p, ref0, 60))
            assert (np.abs(cav.populations(host=True) - ref) / ref).max() < 1e-12


# ---------------------------------------------------------------- reductions and post-processing
def test_residual_and_mass_match_oracle():
    nx, ny = 96, 64
    p = O.Params.from_re(nx, ny, 200.0, 0.1)
    f0 = O.init(p)
    f1 = O.run(p, f0, 100)
    f2 = O.run(p, f1, 100)
    u = [O.moments(p, f)[1:] for f in (f0, f1, f2)]
    with Cavity(nx, ny, Re=200.0, U=0.1, dtype="f64") as cav:
        with pytest.raises(B.LBMError) as e:
            cav.residual()
        assert e.value.code == B.LBM_ENOTREADY
        assert abs(cav.mass() - O.mass(p, f0)) < 1e-10
        cav.step(100)
        r1 = cav.residual()
        cav.step(100)
        r2 = cav.residual()
        m2 = cav.mass()
    assert abs(r1 - O.residual(*u[1], *u[0])) < 1e-10 * r1
    assert abs(r2 - O.residual(*u[2], *u[1])) < 1e-10 * r2
    assert abs(m2 - O.mass(p, f2)) < 1e-10


def test_residual_with_unaligned_calls():
    """Chunks of 37, 63, 100 and 1 steps give the same checkpoints as one call of 200."""
    nx, ny = 50, 40
    with Cavity(nx, ny, Re=100.0, U=0.1, dtype="f64") as a, Cavity(nx, ny, Re=100.0, U=0.1, dtype="f64") as b:
        a.step(200)
        for n in (37, 63, 99, 1):
            b.step(n)
        assert a.residual() == b.residual()
        assert np.array_equal(a.populations(host=True), b.populations(host=True))


def test_stream_function_window_extrema():
    nx, ny = 80, 80
    p = O.Params.from_re(nx, ny, 400.0, 0.1)
    with Cavity(nx, ny, Re=400.0, U=0.1, dtype="f64") as cav:
        cav.step(3000)
        (vmin, imin, jmin), (vmax, imax, jmax) = cav.stream_function_window(nx // 2, nx, 0, ny // 3)
        _, ux, _ = cav.moments(host=True)
    psi, _, _ = O.stream_function(p, ux)
    win = psi[0:ny // 3, nx // 2:nx]
    jm, im = np.unravel_index(np.argmax(win), win.shape)
    assert (imax, jmax) == (nx // 2 + im, jm) and abs(vmax - win.max()) < 1e-13
    jm, im = np.unravel_index(np.argmin(win), win.shape)
    assert (imin, jmin) == (nx // 2 + im, jm) and abs(vmin - win.min()) < 1e-13


def test_probe_series_matches_oracle():
    nx, ny, every, steps = 40, 48, 2, 60
    p = O.Params.from_re(nx, ny, 100.0, 0.1)
    px, py = 20, 24  # x = 0.5, y = 0.6 in width units
    with Cavity(nx, ny, Re=100.0, U=0.1, dtype="f64") as cav:
        cav.step(3)
        q, series = cav.probe(0.5, 0.6, every=every, cap=64)
        cav.step(steps)
        n = cav.probe_count(q)
        s = series.cpu().numpy()
    f = O.run(p, O.init(p), 3)
    want = []
    for t in range(4, 3 + steps + 1):
        f = O.step(p, f)
        if t % every == 0:
            _, ux, uy = O.moments(p, f)
            want.append((ux[py, px], uy[py, px]))
    assert n == len(want)
    assert np.abs(s[:n] - np.array(want)).max() < 1e-14


# ---------------------------------------------------------------- run control, checkpoints, errors
def test_run_to_residual_converges():
    with Cavity(48, 48, Re=100.0, U=0.1, dtype="f64") as cav:
        ok, done = cav.run_to_residual(1e-6, 200_000)
        assert ok and done % 100 == 0 and cav.residual() < 1e-6
        assert cav.step_count == done


def test_save_load_bitwise_continuation():
    nx, ny = 61, 45
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        with Cavity(nx, ny, Re=300.0, U=0.1, dtype="f32s") as a:
            a.step(2000)
            fa = a.populations(host=True)
            ra = a.residual()
        with Cavity(nx, ny, Re=300.0, U=0.1, dtype="f32s") as b:
            b.step(1000)
            b.save(path)
        with Cavity(nx, ny, Re=300.0, U=0.1, dtype="f32s") as c:
            c.load(path)
            assert c.step_count == 1000
            c.step(1000)
            assert np.array_equal(c.populations(host=True), fa)
            assert c.residual() == ra
        with Cavity(nx + 1, ny, Re=300.0, U=0.1, dtype="f32s") as d2:
            with pytest.raises(B.LBMError) as e:
                d2.load(path)
            assert e.value.code == B.LBM_EIO


def test_nan_input_reports_divergence():
    nx, ny = 20, 20
    f0 = np.broadcast_to(W[:, None, None], (9, ny, nx)).copy()
    f0[3, 10, 10] = np.nan
    with make(nx, ny, 0.8, 0.1, "f32s") as cav:
        cav.set_populations(f0)
        cav.step(100)
        with pytest.raises(B.LBMError) as e:
            cav.residual()
        assert e.value.code == B.LBM_EDIVERGED
        with pytest.raises(B.LBMError) as e:
            cav.mass()
        assert e.value.code == B.LBM_EDIVERGED


def test_allocator_hook_failure_reports_enomem():
    import ctypes
    calls = []

    def alloc(nbytes, user):
        calls.append(nbytes)
        return None

    def release(ptr, user):
        pass

    a, r = B.ALLOC_FN(alloc), B.RELEASE_FN(release)
    B.lbm_set_allocator(a, r)
    try:
        with pytest.raises(B.LBMError) as e:
            B.lbm_create(32, 32, 100.0, 0.1, "f32s")
        assert e.value.code == B.LBM_ENOMEM and calls
    finally:
        B.lbm_set_allocator(None, None)
    del ctypes


def test_torch_caching_allocator_hook():
    """Device memory from PyTorch's caching allocator through the allocator hook."""
    live = {}

    def alloc(nbytes, user):
        p = torch.cuda.caching_allocator_alloc(nbytes)
        live[p] = nbytes
        return p

    def release(ptr, user):
        torch.cuda.caching_allocator_delete(ptr)
        live.pop(ptr, None)

    a, r = B.ALLOC_FN(alloc), B.RELEASE_FN(release)
    B.lbm_set_allocator(a, r)
    try:
        with Cavity(64, 64, Re=100.0, U=0.1, dtype="f64") as cav:
            assert live
            cav.step(100)
            f = cav.populations(host=True)
    finally:
        B.lbm_set_allocator(None, None)
    assert not live
    p = O.Params.from_re(64, 64, 100.0, 0.1)
    ref = O.to_soa(O.run(p, O.init(p), 100))
    assert (np.abs(f - ref) / ref).max() < 1e-12


def test_device_and_host_buffers_agree():
    with Cavity(33, 21, Re=100.0, U=0.1, dtype="f32s") as cav:
        cav.step(50)
        d = [t.cpu().numpy() for t in cav.moments()]
        h = cav.moments(host=True)
        for a, b in zip(d, h):
            assert np.array_equal(a, b)
