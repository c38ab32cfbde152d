"""FP64 CPU oracle of the warm-start encoder-decoder (not in the paper).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, written from the definitions:
  conv3x3   y[co,i,j] = b[co] + sum_{ci,ky,kx} w[co,ci,ky,kx] xpad[ci,i+ky,j+kx]   (zero padding 1)
  its data gradient dx[ci,i,j] = sum_{co,ky,kx} w[co,ci,ky,kx] dz[co,i+1-ky,j+1-kx]
  its weight gradient dw[co,ci,ky,kx] = sum_{i,j} dz[co,i,j] xpad[ci,i+ky,j+kx], db[co] = sum dz
  leaky ReLU 0.1, 2x2 average pool, nearest x2 upsampling, channel concatenation,
  loss = mean over masked pixels and 3 channels of (base + out - target)^2.
Architecture: widths (w, 2w, 4w, 8w, 8w); encoder levels of two convs, pooling between them;
decoder levels (3..0) upsample, concatenate the encoder output of that level, two convs; a 3x3
head without activation.  The flat parameter vector lists, per conv in that order, w[co][ci][3][3]
then b[co].

`bf16=True` rounds to bfloat16 (round to nearest even, via float32) exactly the operands the GPU
path feeds to its tensor cores: weights and conv inputs in the forward product, weights and dZ in
the data gradient, dZ and conv inputs in the weight gradient.  Everything else is FP64.
"""
from __future__ import annotations

import numpy as np

LEAK = 0.1


def bf16(x: np.ndarray) -> np.ndarray:
    """Round to bfloat16 (nearest even) through float32; returns float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def widths(w: int):
    return [w, 2 * w, 4 * w, 8 * w, 8 * w]


def conv_list(w: int):
    ch = widths(w)
    io, prev = [], 7
    for l in range(5):
        io += [(prev, ch[l]), (ch[l], ch[l])]
        prev = ch[l]
    for l in range(3, -1, -1):
        io += [(ch[l + 1] + ch[l], ch[l]), (ch[l], ch[l])]
    io.append((ch[0], 3))
    return io


def unpack(params: np.ndarray, w: int):
    out, off = [], 0
    for ci, co in conv_list(w):
        n = co * ci * 9
        out.append((params[off:off + n].reshape(co, ci, 3, 3), params[off + n:off + n + co]))
        off += n + co
    assert off == params.size
    return out


def pack(grads) -> np.ndarray:
    return np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])


def conv_fwd(x, w, b, act, rnd):
    q = bf16 if rnd else (lambda a: a)
    xp = np.pad(q(x), ((0, 0), (1, 1), (1, 1)))
    H, W = x.shape[1:]
    wq = q(w)
    y = np.zeros((w.shape[0], H, W)) + b[:, None, None]
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("oc,chw->ohw", wq[:, :, ky, kx], xp[:, ky:ky + H, kx:kx + W])
    if act:
        y = np.where(y > 0, y, LEAK * y)
    return y


def conv_bwd(x, w, y, gy, act, rnd):
    """(dx, dw, db) of y = act(conv(x, w) + b) given dL/dy."""
    q = bf16 if rnd else (lambda a: a)
    dz = gy * np.where(y > 0, 1.0, LEAK) if act else gy
    H, W = x.shape[1:]
    db = dz.sum(axis=(1, 2))
    dzq = q(dz)
    xp = np.pad(q(x), ((0, 0), (1, 1), (1, 1)))
    dw = np.zeros_like(w)
    for ky in range(3):
        for kx in range(3):
            dw[:, :, ky, kx] = np.einsum("ohw,chw->oc", dzq, xp[:, ky:ky + H, kx:kx + W])
    wq = q(w)
    dxp = np.zeros((x.shape[0], H + 2, W + 2))
    for ky in range(3):
        for kx in range(3):
            dxp[:, ky:ky + H, kx:kx + W] += np.einsum("oc,ohw->chw", wq[:, :, ky, kx], dzq)
    return dxp[:, 1:-1, 1:-1], dw, db


def pool(x):
    return 0.25 * (x[:, 0::2, 0::2] + x[:, 1::2, 0::2] + x[:, 0::2, 1::2] + x[:, 1::2, 1::2])


def pool_back(g):
    return 0.25 * np.repeat(np.repeat(g, 2, axis=1), 2, axis=2)


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_back(g):
    return g[:, 0::2, 0::2] + g[:, 1::2, 0::2] + g[:, 0::2, 1::2] + g[:, 1::2, 1::2]


def forward(params, w, x, rnd=False):
    """Returns (out, cache)."""
    P = unpack(params, w)
    ch = widths(w)
    cache = {"x": x}
    k = 0
    src = x
    e = [None] * 5
    for l in range(5):
        if l:
            src = pool(e[l - 1])
            cache[f"p{l}"] = src
        a = conv_fwd(src, *P[k], True, rnd)
        k += 1
        cache[f"a{l}"] = a
        e[l] = conv_fwd(a, *P[k], True, rnd)
        k += 1
        cache[f"e{l}"] = e[l]
    below = e[4]
    for l in range(3, -1, -1):
        u = up(below)
        cat = np.concatenate([u, e[l]])
        cache[f"u{l}"], cache[f"c{l}"] = u, cat
        b = conv_fwd(cat, *P[k], True, rnd)
        k += 1
        d = conv_fwd(b, *P[k], True, rnd)
        k += 1
        cache[f"b{l}"], cache[f"d{l}"] = b, d
        below = d
    out = conv_fwd(below, *P[k], False, rnd)
    cache["out"] = out
    assert ch[0] == below.shape[0]
    return out, cache


def loss_and_grad(out, base, target, mask):
    """Masked mean squared error over the three channels, the density channel (0) compared up to
    a constant: its masked mean error is removed first.  Returns (loss, dloss/dout); the mean's
    own derivative cancels because the centred errors sum to zero."""
    e = base + out - target
    m = mask.sum()
    e[0] = e[0] - (mask * e[0]).sum() / m
    d = mask[None] * e
    n = 3.0 * m
    return float((d * d).sum() / n), 2.0 * d / n


def backward(params, w, cache, gout, rnd=False):
    """Flat gradient vector of the loss whose dL/d(out) is gout."""
    P = unpack(params, w)
    ch = widths(w)
    grads = [None] * len(P)
    k = len(P) - 1
    gx, gw_, gb = conv_bwd(cache["d0"], *P[k][:1], cache["out"], gout, False, rnd)
    grads[k] = (gw_, gb)
    k -= 1
    g_below = gx
    ge = [None] * 5
    for l in range(4):
        gx, gw_, gb = conv_bwd(cache[f"b{l}"], P[k][0], cache[f"d{l}"], g_below, True, rnd)
        grads[k] = (gw_, gb)
        k -= 1
        gcat, gw_, gb = conv_bwd(cache[f"c{l}"], P[k][0], cache[f"b{l}"], gx, True, rnd)
        grads[k] = (gw_, gb)
        k -= 1
        cu = ch[l + 1]
        ge[l] = gcat[cu:]
        g_below = up_back(gcat[:cu])
    ge[4] = g_below
    for l in range(4, -1, -1):
        ga, gw_, gb = conv_bwd(cache[f"a{l}"], P[k][0], cache[f"e{l}"], ge[l], True, rnd)
        grads[k] = (gw_, gb)
        k -= 1
        src = cache[f"p{l}"] if l else cache["x"]
        gsrc, gw_, gb = conv_bwd(src, P[k][0], cache[f"a{l}"], ga, True, rnd)
        grads[k] = (gw_, gb)
        k -= 1
        if l:
            ge[l - 1] = ge[l - 1] + pool_back(gsrc)
    return pack(grads)


def init_params(w: int, seed: int) -> np.ndarray:
    """Independent seeded initialisation for oracle-only tests (He-uniform, biases small)."""
    rng = np.random.default_rng(seed)
    parts = []
    for ci, co in conv_list(w):
        bound = np.sqrt(6.0 / (ci * 9))
        parts.append(rng.uniform(-bound, bound, size=co * ci * 9))
        parts.append(rng.uniform(-0.05, 0.05, size=co))
    return np.concatenate(parts)
