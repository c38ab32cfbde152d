// lbm_nn_gemm.cu -- see lbm_nn_gemm.cuh.
#include "lbm_nn_gemm.cuh"

namespace lbm {
namespace nn {

namespace {

constexpr int BM = 64, BN = 64, BK = 32;
constexpr int LDS = BK + 8;  // padded shared row (80 bytes): conflict-free ldmatrix

__device__ __forceinline__ unsigned smem_u32(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// 16-byte async copy global -> shared; src_bytes = 0 fills zeros (rows or K past the matrix).
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src),
                 "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

__device__ __forceinline__ void ldmatrix_x4(unsigned (&r)[4], const void* p) {
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(smem_u32(p)));
}

__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
        "{%8, %9}, {%0, %1, %2, %3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Stage one BM x BK tile of A and one BN x BK tile of B (k0 .. k0+BK) into shared memory.
__device__ __forceinline__ void load_tiles(__nv_bfloat16 (*As)[LDS], __nv_bfloat16 (*Bs)[LDS],
                                           const __nv_bfloat16* A, int lda, const __nv_bfloat16* B,
                                           int ldb, int M, int N, int K, int m0, int n0, int k0) {
    // 64 rows x 4 chunks of 8 elements per operand = 256 chunks; 128 threads -> 2 each
#pragma unroll
    for (int c = 0; c < 2; ++c) {
        const int idx = threadIdx.x + c * 128;
        const int row = idx >> 2, ck = (idx & 3) * 8;
        const int k = k0 + ck;
        {
            const int m = m0 + row;
            const bool ok = m < M && k < K;
            const __nv_bfloat16* src = ok ? A + (long long)m * lda + k : A;
            cp_async16(&As[row][ck], src, ok ? 16 : 0);
        }
        {
            const int n = n0 + row;
            const bool ok = n < N && k < K;
            const __nv_bfloat16* src = ok ? B + (long long)n * ldb + k : B;
            cp_async16(&Bs[row][ck], src, ok ? 16 : 0);
        }
    }
}

__global__ void __launch_bounds__(128) k_gemm_bf16_nt(int M, int N, int K, const __nv_bfloat16* __restrict__ A,
                                                      int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                                                      float* __restrict__ C, int ldc, int op, int k_per_split) {
    __shared__ __align__(128) __nv_bfloat16 As[2][BM][LDS];
    __shared__ __align__(128) __nv_bfloat16 Bs[2][BN][LDS];
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;

    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[i][j][r] = 0.f;

    const int nk = (ke - kb + BK - 1) / BK;
    if (nk > 0) {
        load_tiles(As[0], Bs[0], A, lda, B, ldb, M, N, ke, m0, n0, kb);
        cp_async_commit();
    }
    for (int t = 0; t < nk; ++t) {
        const int cur = t & 1;
        if (t + 1 < nk) {
            load_tiles(As[cur ^ 1], Bs[cur ^ 1], A, lda, B, ldb, M, N, ke, m0, n0, kb + (t + 1) * BK);
            cp_async_commit();
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            unsigned af[2][4], bfr[2][4];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int row = wm + i * 16 + (lane & 7) + ((lane >> 3) & 1) * 8;
                const int col = kk + (lane >> 4) * 8;
                ldmatrix_x4(af[i], &As[cur][row][col]);
            }
#pragma unroll
            for (int j = 0; j < 2; ++j) {  // each x4 covers two n8 tiles
                const int row = wn + j * 16 + (lane & 7) + (lane >> 4) * 8;
                const int col = kk + ((lane >> 3) & 1) * 8;
                ldmatrix_x4(bfr[j], &Bs[cur][row][col]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bfr[j >> 1][(j & 1) * 2], bfr[j >> 1][(j & 1) * 2 + 1]);
        }
        __syncthreads();
    }

    // epilogue: fragment (row g, col 2t..2t+1) and (row g+8, ...)
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int m = m0 + wm + i * 16 + g + h * 8;
                if (m >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int n = n0 + wn + j * 8 + tq * 2 + e;
                    if (n >= N) continue;
                    float* c = C + (long long)m * ldc + n;
                    const float v = acc[i][j][h * 2 + e];
                    if (op == kAtomicAdd)
                        atomicAdd(c, v);
                    else if (op == kAccumulate)
                        *c += v;
                    else
                        *c = v;
                }
            }
}

}  // namespace

cudaError_t gemm_bf16_nt(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B,
                         int ldb, float* C, int ldc, GemmOp op, int split_k, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if ((K & 7) || (lda & 7) || (ldb & 7) || K <= 0) return cudaErrorInvalidValue;
    if (split_k < 1) split_k = 1;
    if (split_k > 1 && op != kAtomicAdd) return cudaErrorInvalidValue;
    int kps = (K + split_k - 1) / split_k;
    kps = (kps + BK - 1) / BK * BK;
    split_k = (K + kps - 1) / kps;
    dim3 grid((N + BN - 1) / BN, (M + BM - 1) / BM, split_k);
    k_gemm_bf16_nt<<<grid, 128, 0, st>>>(M, N, K, A, lda, B, ldb, C, ldc, (int)op, kps);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace lbm
