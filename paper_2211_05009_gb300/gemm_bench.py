"""Time the warm-start network's two BF16 GEMM back ends (tcgen05 and mma.sync) on convolution-
shaped products, and check that they agree.

  python -m paper_2211_05009_gb300.gemm_bench --pixels 65536 --cout 160 --cin 160 --reps 20

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
    a = ap.parse_args(argv)
    build()
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


if __name__ == "__main__":
    main()
