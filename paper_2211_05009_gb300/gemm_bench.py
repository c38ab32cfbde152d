"""Time the warm-start network's two BF16 GEMM back ends (tcgen05 and mma.sync) on convolution-
shaped products, and check that they agree.

  python -m paper_2211_05009_gb300.gemm_bench --pixels 65536 --cout 160 --cin 160 --reps 20
  python -m paper_2211_05009_gb300.gemm_bench --conv 256 --cout 160 --cin 160 --reps 20

The shape is the forward product of a 3x3 convolution: M = pixels, N = output channels,
K = 9 x input channels (tcgen05: pixels on the 128-row side, result stored channel-major);
mma.sync computes the same product with channels as rows.  Prints one JSON line with TFLOP/s.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import binding as B
from .build import build


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--pixels", type=int, default=65536)
    ap.add_argument("--cout", type=int, default=160)
    ap.add_argument("--cin", type=int, default=160)
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--conv", type=int, default=0, metavar="SIDE",
                    help="instead: the implicit-GEMM convolutions (gathered, and by TMA boxes over a channels-last "
                         "copy) on a SIDE x SIDE image against the same tcgen05 GEMM on its explicit im2col "
                         "(built here with torch, not timed)")
    a = ap.parse_args(argv)
    build()
    if a.conv:
        return conv_main(a)
    M, N, K = a.pixels, a.cout, (a.cin * 9 + 7) // 8 * 8
    g = torch.Generator(device="cpu").manual_seed(0)
    X = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()   # im2col rows (pixel-major)
    Wt = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()  # weights
    Y1 = torch.empty(N, M, dtype=torch.float32, device="cuda")
    Y2 = torch.empty(N, M, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()

    def tc05():
        assert B.lbm_nn_gemm_bf16_tc05(M, N, K, X, K, Wt, K, Y1, M, 0, err, 1, 1, st.cuda_stream) == B.LBM_OK

    def mma():
        assert B.lbm_nn_gemm_bf16(N, M, K, Wt, K, X, K, Y2, M, 0, 1, st.cuda_stream) == B.LBM_OK

    out = {"M": M, "N": N, "K": K}
    for name, fn in (("tcgen05", tc05), ("mma_sync", mma)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(a.reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / a.reps
        out[name] = {"us": sec * 1e6, "tflops": 2.0 * M * N * K / sec / 1e12}
    out["max_rel_diff"] = float((Y1 - Y2).abs().max() / Y2.abs().max())
    out["tcgen05_wait_error"] = int(err.item())
    print(json.dumps(out), flush=True)


def conv_main(a):
    H = W = a.conv
    P, N, C = H * W, a.cout, a.cin
    K = (C * 9 + 7) // 8 * 8
    g = torch.Generator(device="cpu").manual_seed(0)
    x = torch.randn(C, H, W, generator=g).cuda()
    Wt = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    cols = torch.nn.functional.unfold(x[None], 3, padding=1)[0]  # [C*9][P], k = ci*9 + ky*3 + kx
    A = torch.zeros(P, K, dtype=torch.bfloat16, device="cuda")
    A[:, :C * 9] = cols.t().to(torch.bfloat16)
    Y1 = torch.empty(N, P, dtype=torch.float32, device="cuda")
    Y2 = torch.empty(N, P, dtype=torch.float32, device="cuda")
    Y3 = torch.empty(N, P, dtype=torch.float32, device="cuda")
    Cp = (C + 63) // 64 * 64
    Wtap = torch.empty(N, 9 * Cp, dtype=torch.bfloat16, device="cuda")
    xs = torch.empty(P * Cp, dtype=torch.bfloat16, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    st = torch.cuda.current_stream()
    assert B.lbm_nn_weights_tap_major(Wt, K, C, N, Wtap, st.cuda_stream) == B.LBM_OK

    def tma():
        assert B.lbm_nn_conv3x3_bf16_tma(x, C, None, 0, H, W, Wtap, N, Y3, P, 0, xs, err, 1, st.cuda_stream) == B.LBM_OK

    def implicit():
        assert B.lbm_nn_conv3x3_bf16_tc05(x, C, None, 0, H, W, K, Wt, N, Y1, P, 0, err, 1, st.cuda_stream) == B.LBM_OK

    def explicit():
        assert B.lbm_nn_gemm_bf16_tc05(P, N, K, A, K, Wt, K, Y2, P, 0, err, 1, 1, st.cuda_stream) == B.LBM_OK

    out = {"H": H, "W": W, "M": P, "N": N, "K": K}
    for name, fn in (("tma_conv", tma), ("implicit_conv", implicit), ("gemm_on_explicit_im2col", explicit)):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for _ in range(a.reps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 1e3 / a.reps
        out[name] = {"us": sec * 1e6, "tflops": 2.0 * P * N * K / sec / 1e12}
    out["bitwise_equal"] = bool(torch.equal(Y1, Y2))
    # the TMA form sums the same BF16 products in another order: compare with FP64 on every 16th pixel
    rows = torch.arange(0, P, 16, device="cuda")
    As, Ws = A[rows, :C * 9].double(), Wt[:, :C * 9].double()
    ref, scale = (As @ Ws.t()).t(), (As.abs() @ Ws.abs().t()).t()
    out["tma_max_err_over_abs_sum"] = float(((Y3[:, rows].double() - ref).abs() / scale.clamp_min(1e-30)).max())
    out["explicit_max_err_over_abs_sum"] = float(((Y2[:, rows].double() - ref).abs() / scale.clamp_min(1e-30)).max())
    out["tma_conv"]["tflops_issued"] = out["tma_conv"]["tflops"] * (9 * Cp) / K
    out["bytes_tma_algorithmic"] = C * P * 4 + P * Cp * 2 + N * 9 * Cp * 2 + N * P * 4
    out["tcgen05_wait_error"] = int(err.item())
    out["bytes_implicit_algorithmic"] = C * P * 4 + N * K * 2 + N * P * 4
    out["bytes_explicit_algorithmic"] = P * K * 2 + N * K * 2 + N * P * 4
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
