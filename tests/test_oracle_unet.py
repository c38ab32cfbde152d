"""Pins of the network oracle (oracle/unet.py) against central finite differences and closed forms.

The oracle's backward pass is what the GPU gradients are checked against, so its formulas are
pinned here by differentiating its own forward pass numerically (FP64, no BF16 rounding).
"""
import numpy as np

from oracle import unet as U


def test_bf16_rounding_is_nearest_even():
    # bfloat16 keeps 8 significant bits: the spacing at 1 is 2^-7
    x = np.array([1.0, 1.0 + 2 ** -7, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 3 * 2 ** -9, -2.5, 3.140625])
    # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: to even (1); 1 + 3*2^-8 ties to 1 + 2^-6 (even);
    # 1 + 3*2^-9 is past the midpoint and rounds up to 1 + 2^-7
    assert list(U.bf16(x)) == [1.0, 1.0 + 2 ** -7, 1.0, 1.0 + 2 ** -6, 1.0 + 2 ** -7, -2.5, 3.140625]


def test_conv_matches_direct_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 5, 6))
    w = rng.normal(size=(2, 3, 3, 3))
    b = rng.normal(size=2)
    y = U.conv_fwd(x, w, b, False, False)
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1)))
    for o in range(2):
        for i in range(5):
            for j in range(6):
                want = b[o] + sum(w[o, c, ky, kx] * xp[c, i + ky, j + kx]
                                  for c in range(3) for ky in range(3) for kx in range(3))
                assert abs(y[o, i, j] - want) < 1e-12


def test_conv_backward_by_finite_differences():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 6, 5))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    gy = rng.normal(size=(4, 6, 5))

    def L(x_, w_, b_):
        return float((U.conv_fwd(x_, w_, b_, True, False) * gy).sum())

    y = U.conv_fwd(x, w, b, True, False)
    dx, dw, db = U.conv_bwd(x, w, y, gy, True, False)
    eps = 1e-6
    for arr, grad in ((x, dx), (w, dw), (b, db)):
        for idx in [tuple(rng.integers(0, s) for s in arr.shape) for _ in range(12)]:
            a0 = arr[idx]
            arr[idx] = a0 + eps
            lp = L(x, w, b)
            arr[idx] = a0 - eps
            lm = L(x, w, b)
            arr[idx] = a0
            assert abs((lp - lm) / (2 * eps) - grad[idx]) < 1e-6 * (1 + abs(grad[idx]))


def test_pool_and_up_are_adjoint():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(2, 8, 6))
    g = rng.normal(size=(2, 4, 3))
    assert abs((U.pool(a) * g).sum() - (a * U.pool_back(g)).sum()) < 1e-12
    b = rng.normal(size=(2, 4, 3))
    h = rng.normal(size=(2, 8, 6))
    assert abs((U.up(b) * h).sum() - (b * U.up_back(h)).sum()) < 1e-12


def test_network_gradient_by_finite_differences():
    w, H, W = 1, 32, 32
    rng = np.random.default_rng(3)
    params = U.init_params(w, seed=4)
    x = rng.normal(size=(7, H, W))
    base = rng.normal(size=(3, H, W))
    tgt = rng.normal(size=(3, H, W))
    mask = (rng.uniform(size=(H, W)) > 0.2).astype(float)

    def L(p):
        out, _ = U.forward(p, w, x)
        return U.loss_and_grad(out, base, tgt, mask)[0]

    out, cache = U.forward(params, w, x)
    loss, gout = U.loss_and_grad(out, base, tgt, mask)
    g = U.backward(params, w, cache, gout)
    assert g.shape == params.shape
    eps = 1e-6
    idxs = rng.choice(params.size, size=40, replace=False)
    scale = np.abs(g).max()
    for i in idxs:
        p = params.copy()
        p[i] += eps
        lp = L(p)
        p[i] -= 2 * eps
        lm = L(p)
        assert abs((lp - lm) / (2 * eps) - g[i]) < 1e-5 * scale


def test_param_count_of_the_configured_width():
    """Width 20 gives the ~2M-parameter network (widths 20, 40, 80, 160, 160)."""
    n = sum(co * ci * 9 + co for ci, co in U.conv_list(20))
    assert 1.8e6 < n < 2.2e6


def test_loss_ignores_the_density_level_only():
    """The density channel is compared up to a constant, the velocity channels are not; the
    returned dloss/dout matches central differences of the loss, element by element."""
    rng = np.random.default_rng(8)
    H, W = 6, 5
    out, base, tgt = (rng.normal(size=(3, H, W)) for _ in range(3))
    mask = (rng.uniform(size=(H, W)) > 0.3).astype(float)
    loss, g = U.loss_and_grad(out, base, tgt, mask)
    shifted = tgt.copy()
    shifted[0] += 0.7
    assert abs(U.loss_and_grad(out, base, shifted, mask)[0] - loss) < 1e-12
    shifted = tgt.copy()
    shifted[1] += 0.7
    mean1 = (mask * (base[1] + out[1] - tgt[1])).sum() / mask.sum()
    expect = (0.49 - 1.4 * mean1) / 3  # e_1 shifts by -0.7 over the masked pixels
    assert abs(U.loss_and_grad(out, base, shifted, mask)[0] - loss - expect) < 1e-12
    eps = 1e-6
    for idx in [(0, 1, 1), (0, 4, 3), (1, 2, 0), (2, 5, 4), (0, 0, 0)]:
        o = out.copy()
        o[idx] += eps
        lp = U.loss_and_grad(o, base, tgt, mask)[0]
        o[idx] -= 2 * eps
        lm = U.loss_and_grad(o, base, tgt, mask)[0]
        assert abs((lp - lm) / (2 * eps) - g[idx]) < 1e-8
