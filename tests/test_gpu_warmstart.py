"""The warm-start network's GPU kernels against the FP64 network oracle (oracle/unet.py).

The oracle rounds to bfloat16 exactly the operands the GPU feeds to its tensor cores, so what
remains is FP32 accumulation order and occasional bfloat16 rounding-boundary flips of
intermediate activations; tolerances are stated per check.
"""
import numpy as np
import pytest

from oracle import unet as U
from tests.inputs import uniform

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2211_05009_gb300 import binding as B  # noqa: E402


@pytest.mark.parametrize("M,N,K,split", [(100, 77, 72, 1), (64, 64, 32, 1), (130, 300, 1000, 1),
                                         (48, 200, 4096, 8), (7, 9, 8, 1)])
def test_gemm_bf16_matches_fp64_of_bf16_inputs(M, N, K, split):
    g = torch.Generator(device="cpu").manual_seed(M * 1000 + N)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bm = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    op = 2 if split > 1 else 0
    assert B.lbm_nn_gemm_bf16(M, N, K, A, K, Bm, K, C, N, op, split) == B.LBM_OK
    ref = A.double().cpu().numpy() @ Bm.double().cpu().numpy().T
    err = np.abs(C.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-5, err
    # accumulate adds onto C
    assert B.lbm_nn_gemm_bf16(M, N, K, A, K, Bm, K, C, N, 1, 1) == B.LBM_OK
    err2 = np.abs(C.cpu().numpy() - 2 * ref).max() / np.abs(ref).max()
    assert err2 < 2e-5


@pytest.mark.parametrize("M,N,K,trans,split", [(128, 128, 64, 0, 1), (200, 300, 1000, 0, 1), (7, 9, 8, 0, 1),
                                               (256, 96, 200, 0, 1), (130, 129, 72, 0, 1), (4096, 20, 184, 1, 1),
                                               (1000, 40, 360, 1, 1), (180, 20, 8192, 1, 8), (333, 3, 16, 1, 1)])
def test_gemm_tcgen05_matches_fp64_and_mma_sync(M, N, K, trans, split):
    g = torch.Generator(device="cpu").manual_seed(M * 7 + N * 3 + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    Bm = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    shape = (N, M) if trans else (M, N)
    C = torch.full(shape, float("nan"), dtype=torch.float32, device="cuda") if split == 1 else \
        torch.zeros(shape, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    ldc = M if trans else N
    op = 2 if split > 1 else 0
    assert B.lbm_nn_gemm_bf16_tc05(M, N, K, A, K, Bm, K, C, ldc, op, err, trans, split) == B.LBM_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A.double().cpu().numpy() @ Bm.double().cpu().numpy().T
    got = C.cpu().numpy().T if trans else C.cpu().numpy()
    e = np.abs(got - ref).max() / np.abs(ref).max()
    assert e < 1e-5, e
    C2 = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    assert B.lbm_nn_gemm_bf16(M, N, K, A, K, Bm, K, C2, N, 0, 1) == B.LBM_OK
    assert np.allclose(got, C2.cpu().numpy(), rtol=1e-5, atol=1e-5 * float(np.abs(ref).max()))


def test_gemm_rejects_unaligned_k():
    A = torch.zeros(8, 12, dtype=torch.bfloat16, device="cuda")
    C = torch.zeros(8, 8, dtype=torch.float32, device="cuda")
    assert B.lbm_nn_gemm_bf16(8, 8, 12, A, 12, A, 12, C, 8, 0, 1) == B.LBM_EINVAL


def _setup(width=4, H=64, W=64, seed=7, backend=1):
    n = B.lbm_net_create(width, 0)
    B.lbm_net_set_backend(n, backend)
    B.lbm_net_set_stream(n, torch.cuda.current_stream().cuda_stream)
    params = U.init_params(width, seed=seed)
    assert B.lbm_net_param_count(n) == params.size
    B.lbm_net_set_params(n, torch.tensor(params, dtype=torch.float32, device="cuda"))
    x = uniform(seed, (7, H, W))
    base = 0.3 * uniform(seed + 1, (3, H, W))
    tgt = 0.3 * uniform(seed + 2, (3, H, W))
    mask = (uniform(seed + 3, (H, W)) > -0.6).astype(np.float64)
    # the oracle sees exactly the FP32 values the GPU holds
    params32 = params.astype(np.float32).astype(np.float64)
    arrs = [a.astype(np.float32).astype(np.float64) for a in (x, base, tgt, mask)]
    dev = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in arrs]
    return n, params32, arrs, dev


@pytest.mark.parametrize("backend", [1, 0, 3])
def test_network_forward_matches_oracle(backend):
    H = W = 64
    n, p, (x, base, tgt, mask), (dx, dbase, dtgt, dmask) = _setup(H=H, W=W, backend=backend)
    try:
        out = torch.empty(3, H, W, dtype=torch.float32, device="cuda")
        B.lbm_net_forward(n, dx, H, W, out)
        torch.cuda.synchronize()
        ref, _ = U.forward(p, 4, x, rnd=True)
        got = out.double().cpu().numpy()
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        print(f"backend {backend}: forward rel err {err:.2e}")
        assert err < 5e-3
    finally:
        B.lbm_net_destroy(n)


@pytest.mark.parametrize("backend", [1, 0, 3])
def test_network_loss_and_gradients_match_oracle(backend):
    H = W = 64
    n, p, (x, base, tgt, mask), (dx, dbase, dtgt, dmask) = _setup(H=H, W=W, backend=backend)
    try:
        B.lbm_net_zero_grads(n)
        loss = B.lbm_net_backward(n, dx, dbase, dtgt, dmask, H, W)
        g = torch.empty(B.lbm_net_param_count(n), dtype=torch.float32, device="cuda")
        B.lbm_net_get_grads(n, g)
        g = g.double().cpu().numpy()
        out, cache = U.forward(p, 4, x, rnd=True)
        ref_loss, gout = U.loss_and_grad(out, base, tgt, mask)
        ref = U.backward(p, 4, cache, gout, rnd=True)
        assert abs(loss - ref_loss) < 1e-3 * ref_loss
        # BF16 rounding of slightly different activations flips different operands on the two
        # sides, and the flips compound with depth: the scale of that effect is the difference
        # between the oracle with and without BF16 rounding.  Per tensor, the GPU must agree with
        # the rounded oracle to within twice that scale (or 1 % of the tensor's norm); overall to 1 %.
        out_x, cache_x = U.forward(p, 4, x, rnd=False)
        exact = U.backward(p, 4, cache_x, U.loss_and_grad(out_x, base, tgt, mask)[1], rnd=False)
        off, worst = 0, 0.0
        for ci, co in U.conv_list(4):
            for sz in (co * ci * 9, co):
                a, b, e = g[off:off + sz], ref[off:off + sz], exact[off:off + sz]
                scale = max(np.linalg.norm(b - e), 1e-2 * np.linalg.norm(b))
                worst = max(worst, np.linalg.norm(a - b) / scale)
                off += sz
        total = np.linalg.norm(g - ref) / np.linalg.norm(ref)
        print(f"loss {loss:.6e} vs {ref_loss:.6e}; worst per-tensor error / rounding scale {worst:.2f}; "
              f"overall rel err {total:.2e}")
        assert worst < 2.0
        assert total < 1e-2
    finally:
        B.lbm_net_destroy(n)


def test_adam_training_overfits_one_sample():
    """A smooth correction field is learnable: Adam on one sample cuts the loss at least 4x."""
    H, W = 64, 128
    n, p, arrs, (dx, dbase, dtgt, dmask) = _setup(H=H, W=W)
    try:
        yy, xx = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        smooth = 0.2 * np.sin(2 * np.pi * yy / H) * np.cos(2 * np.pi * xx / W)
        tgt = dbase + torch.tensor(np.stack([smooth, -smooth, 0.5 * smooth]), dtype=torch.float32, device="cuda")
        losses = []
        for it in range(100):
            B.lbm_net_zero_grads(n)
            losses.append(B.lbm_net_backward(n, dx, dbase, tgt.contiguous(), dmask, H, W))
            B.lbm_net_adam_step(n, 2e-3)
        print(f"loss {losses[0]:.4e} -> {losses[-1]:.4e}")
        assert losses[-1] < 0.25 * losses[0]
    finally:
        B.lbm_net_destroy(n)


def test_network_rejects_bad_shapes():
    n = B.lbm_net_create(4, 0)
    try:
        t = torch.zeros(7 * 40 * 64, dtype=torch.float32, device="cuda")
        with pytest.raises(B.LBMError) as e:
            B.lbm_net_forward(n, t, 40, 64, t)
        assert e.value.code == B.LBM_EINVAL
    finally:
        B.lbm_net_destroy(n)


def test_warm_target_and_output_roundtrip():
    """lbm_warm_target scales a fine field (zero padding rows); lbm_warm_output with a zero
    correction turns the same scaled channels back into the field."""
    nx, ny, H, U0 = 48, 37, 48, 0.1
    r = uniform(21, (3, ny, nx))
    rho, ux, uy = 1 + 0.01 * r[0], 0.05 * r[1], 0.05 * r[2]
    d = [torch.tensor(a, device="cuda") for a in (rho, ux, uy)]
    t = torch.full((3, H, nx), 7.0, dtype=torch.float32, device="cuda")
    B.lbm_warm_target(*d, nx, ny, H, U0, t)
    torch.cuda.synchronize()
    t_h = t.cpu().numpy()
    exp = np.stack([(rho - 1) * B.LBM_WARM_RHO_SCALE, ux / U0, uy / U0]).astype(np.float32)
    assert np.array_equal(t_h[:, :ny], exp) and not t_h[:, ny:].any()
    inp = torch.zeros((7, H, nx), dtype=torch.float32, device="cuda")
    inp[:3] = t
    out = torch.zeros((3, H, nx), dtype=torch.float32, device="cuda")
    f = [torch.empty((ny, nx), dtype=torch.float64, device="cuda") for _ in range(3)]
    B.lbm_warm_output(inp, out, nx, ny, H, U0, *f)
    torch.cuda.synchronize()
    for got, ref in zip(f, (rho, ux, uy)):
        assert np.abs(got.cpu().numpy() - ref).max() < 1e-8


def test_warm_smooth_matches_box_filter():
    """lbm_warm_smooth: `passes` 3x3 means over rows [0, ny), indices clamped to those rows and the
    columns; the padding rows are left as they were."""
    H, W, ny, passes = 32, 40, 27, 3
    a = uniform(31, (3, H, W)).astype(np.float32)
    ref = a.astype(np.float64).copy()
    for _ in range(passes):
        v = ref[:, :ny]
        yi = np.clip(np.arange(ny)[:, None] + np.array([-1, 0, 1])[None], 0, ny - 1)
        xi = np.clip(np.arange(W)[:, None] + np.array([-1, 0, 1])[None], 0, W - 1)
        acc = np.zeros_like(v)
        for dy in range(3):
            for dx in range(3):
                acc += v[:, yi[:, dy]][:, :, xi[:, dx]]
        ref[:, :ny] = acc / 9
    t = torch.tensor(a, device="cuda")
    scratch = torch.empty_like(t)
    B.lbm_warm_smooth(t, ny, H, W, passes, scratch)
    torch.cuda.synchronize()
    got = t.cpu().numpy()
    assert np.abs(got - ref).max() < 1e-6
    assert np.array_equal(got[:, ny:], a[:, ny:])


def test_gemm_tcgen05_strided_operands_ignore_the_padding():
    """Row strides larger than K (lda = K + 24, ldb = K + 8): the columns past K hold NaN and must
    never be read (the tensor maps end at K and fill zeros)."""
    M, N, K = 300, 72, 200
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.full((M, K + 24), float("nan")).to(torch.bfloat16)
    Bm = torch.full((N, K + 8), float("nan")).to(torch.bfloat16)
    A[:, :K] = torch.randn(M, K, generator=g).to(torch.bfloat16)
    Bm[:, :K] = torch.randn(N, K, generator=g).to(torch.bfloat16)
    A, Bm = A.cuda(), Bm.cuda()
    C = torch.zeros(M, N, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert B.lbm_nn_gemm_bf16_tc05(M, N, K, A, K + 24, Bm, K + 8, C, N, 0, err, 0, 1) == B.LBM_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    ref = A[:, :K].double().cpu().numpy() @ Bm[:, :K].double().cpu().numpy().T
    got = C.cpu().numpy()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() / np.abs(ref).max() < 1e-5


def _im2col_pk(x, H, W, K):
    """Pixel-major im2col from its definition: row p = y*W + x, column k = ci*9 + ky*3 + kx,
    padding 1, zeros past C*9 (numpy, float64)."""
    C = x.shape[0]
    xp = np.zeros((C, H + 2, W + 2))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((H * W, K))
    for ci in range(C):
        for ky in range(3):
            for kx in range(3):
                out[:, ci * 9 + ky * 3 + kx] = xp[ci, ky:ky + H, kx:kx + W].reshape(-1)
    return out


@pytest.mark.parametrize("c1,c2,H,W,N", [(3, 0, 16, 40, 20), (7, 5, 33, 9, 40), (20, 20, 64, 64, 160),
                                         (1, 0, 5, 3, 16), (40, 0, 24, 24, 72)])
def test_implicit_conv_equals_explicit_im2col_gemm(c1, c2, H, W, N):
    """lbm_nn_conv3x3_bf16_tc05 (im2col rows gathered inside the kernel) is bitwise the tcgen05
    GEMM on the explicit im2col of the same inputs, and within 1e-5 of the FP64 convolution of the
    BF16-rounded operands."""
    g = torch.Generator(device="cpu").manual_seed(c1 * 100 + H)
    C = c1 + c2
    K = (C * 9 + 7) // 8 * 8
    x = torch.randn(C, H, W, generator=g)
    Wt = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Wt[:, C * 9:] = 0
    x1 = x[:c1].contiguous().cuda()
    x2 = x[c1:].contiguous().cuda() if c2 else None
    Wd = Wt.cuda()
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = H * W
    out = torch.full((N, P), float("nan"), dtype=torch.float32, device="cuda")
    assert B.lbm_nn_conv3x3_bf16_tc05(x1, c1, x2, c2, H, W, K, Wd, N, out, P, 0, err, trans_c=1) == B.LBM_OK
    A = torch.tensor(_im2col_pk(x.double().numpy(), H, W, K)).to(torch.bfloat16)
    ref_c = torch.full((N, P), float("nan"), dtype=torch.float32, device="cuda")
    assert B.lbm_nn_gemm_bf16_tc05(P, N, K, A.cuda().contiguous(), K, Wd, K, ref_c, P, 0, err, 1, 1) == B.LBM_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    assert torch.equal(out, ref_c)
    ref = (A.double().numpy() @ Wt.double().numpy().T).T
    assert np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-5


@pytest.mark.parametrize("c1,c2,H,W,N,op,trans", [(3, 0, 2, 256, 20, 0, 1), (7, 5, 16, 128, 40, 0, 1),
                                                  (40, 20, 8, 64, 160, 0, 1), (70, 0, 32, 16, 72, 0, 1),
                                                  (100, 60, 64, 8, 256, 0, 1), (5, 0, 16, 32, 24, 1, 0)])
def test_tma_conv_matches_fp64_of_bf16_inputs(c1, c2, H, W, N, op, trans):
    """lbm_nn_conv3x3_bf16_tma: the tap-major weights are the permutation of their definition, and
    the convolution equals the FP64 product of the BF16-rounded explicit im2col and weights to FP32
    summation rounding (1e-5 of the sum of absolute products).  Covers one-row boxes (W >= 128),
    several-row boxes (W < 128), channel padding to 64, two 64-channel blocks per tap, N = 256, and
    the accumulate / row-major epilogue."""
    g = torch.Generator(device="cpu").manual_seed(c1 * 1000 + W)
    C, P = c1 + c2, H * W
    K = (C * 9 + 7) // 8 * 8
    Cp = (C + 63) // 64 * 64
    x = torch.randn(C, H, W, generator=g)
    Wt = torch.randn(N, K, generator=g).to(torch.bfloat16)
    Wt[:, C * 9:] = 0
    x1 = x[:c1].contiguous().cuda()
    x2 = x[c1:].contiguous().cuda() if c2 else None
    Wtap = torch.full((N, 9 * Cp), float("nan"), dtype=torch.bfloat16, device="cuda")
    assert B.lbm_nn_weights_tap_major(Wt.cuda(), K, C, N, Wtap) == B.LBM_OK
    want = torch.zeros(N, 9, Cp, dtype=torch.bfloat16)
    want[:, :, :C] = Wt[:, :C * 9].reshape(N, C, 9).transpose(1, 2)
    torch.cuda.synchronize()
    assert torch.equal(Wtap.cpu(), want.reshape(N, 9 * Cp))
    xs = torch.empty(P * Cp, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    init = torch.randn((N, P) if trans else (P, N), generator=g)
    out = init.clone().cuda()
    ldc = P if trans else N
    assert B.lbm_nn_conv3x3_bf16_tma(x1, c1, x2, c2, H, W, Wtap, N, out, ldc, op, xs, err, trans_c=trans) == B.LBM_OK
    torch.cuda.synchronize()
    assert int(err.item()) == 0
    A = torch.tensor(_im2col_pk(x.double().numpy(), H, W, K)).to(torch.bfloat16).double().numpy()[:, :C * 9]
    Wd = Wt[:, :C * 9].double().numpy()
    ref, scale = A @ Wd.T, np.abs(A) @ np.abs(Wd).T  # [P][N]
    if op == 1:
        ref = ref + (init.double().numpy().T if trans else init.double().numpy())
    got = out.double().cpu().numpy()
    got = got.T if trans else got
    assert np.all(np.isfinite(got))
    assert (np.abs(got - ref) / np.maximum(scale, 1e-30)).max() < 1e-5


def test_tma_conv_refuses_shapes_it_does_not_take():
    """W neither a multiple nor a divisor of 128, or H*W not a multiple of 128: LBM_EINVAL and
    nothing written."""
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    for H, W in ((16, 40), (3, 64), (1, 96)):
        x = torch.randn(4, H, W, device="cuda")
        Wtap = torch.zeros(16, 9 * 64, dtype=torch.bfloat16, device="cuda")
        xs = torch.full((H * W * 64,), 7.0, dtype=torch.bfloat16, device="cuda")
        out = torch.full((16, H * W), float("nan"), device="cuda")
        assert B.lbm_nn_conv3x3_bf16_tma(x, 4, None, 0, H, W, Wtap, 16, out, H * W, 0, xs, err, trans_c=1) == B.LBM_EINVAL
        torch.cuda.synchronize()
        assert torch.isnan(out).all() and (xs == 7.0).all()


def test_network_implicit_and_explicit_backends_agree():
    """The network's forward output and gradients with the implicit convolutions (backend 2) are
    bitwise those with explicit im2col (backend 1)."""
    H, W = 64, 128
    res = []
    for backend in (1, 2):
        n, p, arrs, (dx, dbase, dtgt, dmask) = _setup(H=H, W=W, backend=backend)
        try:
            out = torch.empty((3, H, W), dtype=torch.float32, device="cuda")
            B.lbm_net_forward(n, dx, H, W, out)
            B.lbm_net_zero_grads(n)
            loss = B.lbm_net_backward(n, dx, dbase, dtgt, dmask, H, W)
            g = torch.empty(B.lbm_net_param_count(n), dtype=torch.float32, device="cuda")
            B.lbm_net_get_grads(n, g)
            res.append((out.cpu(), loss, g.cpu()))
        finally:
            B.lbm_net_destroy(n)
    assert torch.equal(res[0][0], res[1][0]) and res[0][1] == res[1][1] and torch.equal(res[0][2], res[1][2])
