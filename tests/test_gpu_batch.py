"""The batched persistent sweep (lbm_batch_*) against the single-cavity path and the oracle.

A batch steps cavities of uneven sizes in one cooperative launch per checkpoint interval; the
per-node arithmetic is the single-cavity kernel's, so populations must agree bitwise, and
per-cavity Eq. 6 residuals must agree to rounding (their partial sums are grouped differently).
"""
import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import binding as B  # noqa: E402
from paper_2211_05009_gb300.cavity import Cavity  # noqa: E402

CASES = [(64, 48, 100.0, 0.1), (97, 130, 400.0, 0.1), (50, 20, 300.0, 0.05), (130, 65, 1000.0, 0.1), (3, 5, 10.0, 0.1)]


def make_batch(cases, dtype):
    nx, ny, re, u = zip(*cases)
    b = B.lbm_batch_create(nx, ny, re, u, dtype)
    B.lbm_batch_set_stream(b, torch.cuda.current_stream().cuda_stream)
    return b


def batch_pop(b, i, nx, ny):
    f = torch.empty((9, ny, nx), dtype=torch.float64, device="cuda")
    B.lbm_batch_get_populations(b, i, f)
    return f.cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32s", "f16s", "f64"])
def test_batch_matches_single_cavity_bitwise(dtype):
    steps = 250
    b = make_batch(CASES, dtype)
    try:
        B.lbm_batch_step(b, steps)
        r_b, st = B.lbm_batch_residual(b, len(CASES))
        for i, (nx, ny, re, u) in enumerate(CASES):
            with Cavity(nx, ny, Re=re, U=u, dtype=dtype) as cav:
                cav.step(steps)
                ref = cav.populations(host=True)
                r_s = cav.residual()
            got = batch_pop(b, i, nx, ny)
            if dtype == "f64":  # FP64: equal to rounding (the compiler may contract differently)
                assert (np.abs(got - ref) / ref).max() < 1e-13, f"cavity {i}"
            else:
                assert np.array_equal(got, ref), f"cavity {i}"
            # Eq. 6 partial sums are grouped per thread in the arithmetic type, differently here
            assert abs(r_b[i] - r_s) <= (1e-12 if dtype == "f64" else 1e-6) * r_s + 1e-300
            assert st[i] == 0
    finally:
        B.lbm_batch_destroy(b)


def test_batch_f64_matches_oracle():
    steps = 200
    b = make_batch(CASES[:3], "f64")
    try:
        B.lbm_batch_step(b, steps)
        for i, (nx, ny, re, u) in enumerate(CASES[:3]):
            p = O.Params.from_re(nx, ny, re, u)
            ref = O.to_soa(O.run(p, O.init(p), steps))
            assert (np.abs(batch_pop(b, i, nx, ny) - ref) / ref).max() < 1e-12
    finally:
        B.lbm_batch_destroy(b)


def test_batch_run_to_residual_retires_each_cavity():
    cases = [(48, 48, 50.0, 0.1), (40, 60, 100.0, 0.1), (64, 32, 200.0, 0.1)]
    tol = 1e-6
    b = make_batch(cases, "f32s")
    try:
        rc, done = B.lbm_batch_run_to_residual(b, len(cases), tol, 200_000)
        assert rc == B.LBM_OK
        r, st = B.lbm_batch_residual(b, len(cases))
        assert (st == 1).all() and (r < tol).all()
        assert len(set(done.tolist())) > 1  # they retire at different steps
        steps = B.lbm_batch_cavity_steps(b, len(cases))
        assert (steps == done).all() and (done % 100 == 0).all()
        for i, (nx, ny, re, u) in enumerate(cases):
            with Cavity(nx, ny, Re=re, U=u, dtype="f32s") as cav:
                cav.step(int(done[i]))
                assert np.array_equal(batch_pop(b, i, nx, ny), cav.populations(host=True))
                assert cav.residual() < tol
                # the checkpoint before retirement was still above tol
            with Cavity(nx, ny, Re=re, U=u, dtype="f32s") as cav:
                cav.step(int(done[i]) - 100)
                assert cav.residual() >= tol
    finally:
        B.lbm_batch_destroy(b)


def test_batch_probe_and_stream_function_match_single():
    cases = CASES[:4]
    cap, every, steps = 64, 2, 120
    b = make_batch(cases, "f32s")
    series = torch.zeros((len(cases), cap, 2), dtype=torch.float64, device="cuda")
    try:
        B.lbm_batch_step(b, 7)
        B.lbm_batch_probe(b, [0.5] * 4, [0.3] * 4, every, series, cap)
        B.lbm_batch_step(b, steps)
        s_b = series.cpu().numpy()
        for i, (nx, ny, re, u) in enumerate(cases):
            with Cavity(nx, ny, Re=re, U=u, dtype="f32s") as cav:
                cav.step(7)
                q, ser = cav.probe(0.5, 0.3, every=every, cap=cap)
                cav.step(steps)
                n = cav.probe_count(q)
                assert np.array_equal(s_b[i, :n], ser.cpu().numpy()[:n])
                assert B.lbm_batch_stream_function(b, i) == cav.stream_function()
    finally:
        B.lbm_batch_destroy(b)


def test_batch_barrier_timeout_reports_etimeout():
    """A block that never reaches the grid barrier (a launch parameter makes block 0 leave before
    its first barrier) makes every other block's bounded wait run out: the call returns
    LBM_ETIMEOUT, no hang, and the GPU stays usable."""
    b = make_batch(CASES[:2], "f32s")
    try:
        B.lbm_batch_set_barrier_limit(b, 0.05, absent_block=0)
        with pytest.raises(B.LBMError) as e:
            B.lbm_batch_step(b, 10)
        assert e.value.code == B.LBM_ETIMEOUT
    finally:
        B.lbm_batch_destroy(b)
    b = make_batch(CASES[:2], "f32s")
    try:
        B.lbm_batch_step(b, 10)
    finally:
        B.lbm_batch_destroy(b)


def test_batch_rejects_bad_arguments():
    with pytest.raises(B.LBMError) as e:
        B.lbm_batch_create([10, 2], [10, 10], [100.0, 100.0], [0.1, 0.1], "f32s")
    assert e.value.code == B.LBM_EINVAL and "cavity 1" in str(e.value)


def single_reference(cases, dtype, steps, probe=None):
    """Populations, residual and (optionally) probe series of each case run alone."""
    out = []
    for nx, ny, re, u in cases:
        with Cavity(nx, ny, Re=re, U=u, dtype=dtype) as cav:
            ser = None
            if probe:
                q, ser = cav.probe(probe[0], probe[1], every=probe[2], cap=probe[3])
            cav.step(steps)
            out.append((cav.populations(host=True), cav.residual(), None if ser is None else ser.cpu().numpy()))
    return out


@pytest.mark.parametrize("dtype", ["f32s", "bf16s", "f64"])
def test_every_tile_shape_matches_single_cavity(dtype):
    """Each tile shape (rows per item, load path, blocks per SM) produces the single-cavity
    populations and probe samples; whole checkpoint intervals run as graph replays."""
    steps, cap, every = 250, 200, 2
    ref = single_reference(CASES, dtype, steps, probe=(0.5, 0.3, every, cap))
    for shape in range(B.LBM_BATCH_SHAPES):
        b = make_batch(CASES, dtype)
        series = torch.zeros((len(CASES), cap, 2), dtype=torch.float64, device="cuda")
        try:
            B.lbm_batch_set_shape(b, shape)
            B.lbm_batch_probe(b, [0.5] * len(CASES), [0.3] * len(CASES), every, series, cap)
            B.lbm_batch_step(b, steps)
            sh, rows, blocks, graphs = B.lbm_batch_launch_info(b)
            assert sh == shape and rows in (1, 2, 4) and blocks >= 152
            assert graphs == 2, "steps 0..200 should run as two captured intervals"
            r_b, st = B.lbm_batch_residual(b, len(CASES))
            s_b = series.cpu().numpy()
            for i, (nx, ny, re, u) in enumerate(CASES):
                got = batch_pop(b, i, nx, ny)
                pop, r_s, ser = ref[i]
                if dtype == "f64":
                    assert (np.abs(got - pop) / pop).max() < 1e-13, f"shape {shape} cavity {i}"
                    assert np.allclose(s_b[i, :steps // every], ser[:steps // every], rtol=1e-12, atol=1e-16)
                else:
                    assert np.array_equal(got, pop), f"shape {shape} cavity {i}"
                    assert np.array_equal(s_b[i, :steps // every], ser[:steps // every]), f"shape {shape} cavity {i}"
                assert abs(r_b[i] - r_s) <= (1e-12 if dtype == "f64" else 1e-6) * r_s + 1e-300
        finally:
            B.lbm_batch_destroy(b)


def test_autotune_leaves_the_state_unchanged():
    """lbm_batch_autotune in the middle of an interval: the batch continues exactly as one that
    was never tuned (populations and probe series bitwise; residual to rounding)."""
    cases = CASES[:4]
    cap, every = 300, 3
    rows = []  # rows per work item of each tile shape
    b = make_batch(cases, "f32s")
    try:
        for s in range(B.LBM_BATCH_SHAPES):
            B.lbm_batch_set_shape(b, s)
            rows.append(B.lbm_batch_launch_info(b)[1])
    finally:
        B.lbm_batch_destroy(b)
    runs = []
    for tune in (False, True):
        b = make_batch(cases, "f32s")
        series = torch.zeros((len(cases), cap, 2), dtype=torch.float64, device="cuda")
        try:
            B.lbm_batch_probe(b, [0.5] * 4, [0.4] * 4, every, series, cap)
            B.lbm_batch_step(b, 150)
            chosen = None
            if tune:
                chosen, ms = B.lbm_batch_autotune(b, 20)
                assert 0 <= chosen < B.LBM_BATCH_SHAPES and (ms > 0).all()
                # the fewest rows per item among the shapes within 2 % of the fastest trial
                near = [s for s in range(B.LBM_BATCH_SHAPES) if ms[s] <= np.float32(1.02) * ms.min()]
                assert chosen in near and rows[chosen] == min(rows[s] for s in near)
                assert B.lbm_batch_launch_info(b)[0] == chosen
            B.lbm_batch_step(b, 250)
            r, _ = B.lbm_batch_residual(b, len(cases))
            pops = [batch_pop(b, i, c[0], c[1]) for i, c in enumerate(cases)]
            steps = B.lbm_batch_cavity_steps(b, len(cases))
            runs.append((pops, series.cpu().numpy(), r, steps))
        finally:
            B.lbm_batch_destroy(b)
    (p0, s0, r0, t0), (p1, s1, r1, t1) = runs
    assert (t0 == 400).all() and (t1 == 400).all()
    for a, c in zip(p0, p1):
        assert np.array_equal(a, c)
    assert np.array_equal(s0, s1)
    assert np.allclose(r0, r1, rtol=1e-6, atol=0)


def test_batch_set_moments_neq_matches_single_cavity():
    """lbm_batch_set_moments_ex(LBM_INIT_NEQ) gives cavity i the single-cavity warm start, and
    both continue identically."""
    from tests.inputs import uniform
    cases = CASES[:3]
    b = make_batch(cases, "f32s")
    fields = []
    try:
        for i, (nx, ny, re, u) in enumerate(cases):
            r = uniform(10 + i, (3, ny, nx))
            fl = [torch.from_numpy(a).cuda() for a in (1 + 0.01 * r[0], 0.03 * r[1], 0.03 * r[2])]
            fields.append(fl)
            B.lbm_batch_set_moments(b, i, *fl, flags=B.LBM_INIT_NEQ)
        B.lbm_batch_step(b, 130)
        for i, (nx, ny, re, u) in enumerate(cases):
            with Cavity(nx, ny, Re=re, U=u, dtype="f32s") as cav:
                cav.set_moments(*fields[i], neq=True)
                cav.step(130)
                assert np.array_equal(batch_pop(b, i, nx, ny), cav.populations(host=True)), f"cavity {i}"
    finally:
        B.lbm_batch_destroy(b)
