// lbm_nn_umma.cu -- the warm-start network's BF16 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), sm_103a.
//
//   C[M][N] (op)= sum_k A[M][K] * B[N][K]      (both K-contiguous; same contract as gemm_bf16_nt)
//
// CTA tile 128 x TN (TN = 32, 64 or 128, picked from N), K step 64 (four MMAs of K = 16), two
// shared-memory stages; optional split-K over gridDim.z (atomic accumulation) and a transposed
// store C[n][m], so a GEMM can put its long dimension (pixels) on the 128-row side.  Operands are
// staged with cp.async into the canonical no-swizzle K-major layout (8 x 8 core matrices of 128
// contiguous bytes; core matrices adjacent in K are 128 bytes apart, 8-row groups 1024 bytes
// apart) and described to the tensor core by shared-memory descriptors.  One thread issues the
// MMAs; tcgen05.commit arrives on the stage's mbarrier when they complete, which frees the stage
// for the next load.  The 128 x TN FP32 accumulator lives in TN TMEM columns; each warp reads
// its 32 lanes back with tcgen05.ld.  Every mbarrier wait is bounded (clock limit): on timeout
// the CTA records an error, still frees its TMEM and returns.  Shared memory per CTA (two stages of
// 16 KB + TN x 128 bytes) bounds residency so that the resident CTAs of one kernel never need more
// than the 512 TMEM columns of an SM (3 x 128, 4 x 64, 5 x 32); no CTA waits on another while it
// holds TMEM, so allocation can at worst wait for a neighbouring kernel's CTAs to finish.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lbm_nn_gemm.cuh"

namespace lbm {
namespace nn {

namespace {

constexpr int TM = 128, TK = 64, STAGES = 2;
constexpr int kTileA = TM * TK * 2;  // 16 KB
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s

template <int TN>
struct Cfg {
    static constexpr int kTileB = TN * TK * 2;
    static constexpr int kStage = kTileA + kTileB;
    static constexpr int kSmem = STAGES * kStage + 2048;  // + alignment slack, mbarriers, TMEM slot
    // instruction descriptor, kind::f16: FP32 accumulate, BF16 A and B, both K-major, N, M
    static constexpr uint32_t kIdesc =
        (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
};

__device__ __forceinline__ uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ __forceinline__ void cp16(uint32_t dst, const void* src, int bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(bytes));
}

// shared-memory matrix descriptor: start >> 4, LBO >> 4, SBO >> 4, version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    const long long t0 = clock64();
    while (true) {
        uint32_t done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > kWaitCycles) return false;
    }
}

// Stage rows [r0, r0 + ROWS) x K [k0, k0 + 64) of a K-contiguous matrix into the core-matrix
// layout at s (row group stride 1024 bytes, K-chunk stride 128 bytes); zero outside [0,R) x [0,ke).
template <int ROWS>
__device__ __forceinline__ void stage_rows(uint32_t s, const __nv_bfloat16* X, int ld, int R, int ke, int r0, int k0) {
    constexpr int PER = ROWS * 8 / 128;  // 16-byte chunks per thread
#pragma unroll
    for (int c = 0; c < PER; ++c) {
        const int idx = threadIdx.x + c * 128;
        const int r = idx >> 3, kc = idx & 7;
        const uint32_t off = (uint32_t)((r >> 3) * 1024 + kc * 128 + (r & 7) * 16);
        const int k = k0 + kc * 8;
        const bool ok = (r0 + r) < R && k < ke;
        cp16(s + off, ok ? (const void*)(X + (long long)(r0 + r) * ld + k) : (const void*)X, ok ? 16 : 0);
    }
}

template <int TN>
__global__ void __launch_bounds__(128, 1) k_gemm_umma(int M, int N, int K, const __nv_bfloat16* __restrict__ A, int lda,
                                                     const __nv_bfloat16* __restrict__ B, int ldb, float* __restrict__ C,
                                                     int ldc, int op, int trans_c, int k_per_split, int* err) {
    using CF = Cfg<TN>;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + STAGES * CF::kStage);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + STAGES);
    __shared__ int failed;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * TN;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    if (threadIdx.x == 0) {
        failed = 0;
        for (int s = 0; s < STAGES; ++s) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(&bars[s])));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(tmem_slot)), "r"((uint32_t)TN));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tmem_slot;

    const int nk = ke > kb ? (ke - kb + TK - 1) / TK : 0;
    auto sA = [&](int s) { return sa(base + (size_t)s * CF::kStage); };
    auto sB = [&](int s) { return sa(base + (size_t)s * CF::kStage + kTileA); };

    if (nk > 0) {
        stage_rows<TM>(sA(0), A, lda, M, ke, m0, kb);
        stage_rows<TN>(sB(0), B, ldb, N, ke, n0, kb);
        asm volatile("cp.async.commit_group;\n" ::);
    }
    for (int t = 0; t < nk; ++t) {
        const int s = t & 1;
        asm volatile("cp.async.wait_group 0;\n" ::);
        asm volatile("fence.proxy.async.shared::cta;\n" ::);  // staged tile visible to the tensor core
        __syncthreads();
        if (threadIdx.x == 0 && !failed) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const uint64_t da = smem_desc(sA(s) + kk * 256, 128, 1024);
                const uint64_t db = smem_desc(sB(s) + kk * 256, 128, 1024);
                const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(CF::kIdesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(&bars[s])));
        }
        if (t + 1 < nk) {
            const int s2 = s ^ 1;
            // the MMAs of tile t-1 read stage s2: wait for their commit before overwriting it
            if (t >= 1 && !failed && !mbar_wait(sa(&bars[s2]), ((t - 1) >> 1) & 1)) failed = 1;
            __syncthreads();
            if (!failed) {
                stage_rows<TM>(sA(s2), A, lda, M, ke, m0, kb + (t + 1) * TK);
                stage_rows<TN>(sB(s2), B, ldb, N, ke, n0, kb + (t + 1) * TK);
            }
            asm volatile("cp.async.commit_group;\n" ::);
        }
    }
    // all MMAs done: the last commit covers every earlier one of this thread
    if (nk > 0 && !failed && !mbar_wait(sa(&bars[(nk - 1) & 1]), ((nk - 1) >> 1) & 1)) failed = 1;
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);

    if (!failed && nk > 0) {
        // warp w owns TMEM lanes 32w .. 32w+31 = tile rows; 16 columns per load
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < TN; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
                "%14, %15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::);
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int n = n0 + c0 + j;
                    if (n < N) {
                        float* c = trans_c ? C + (long long)n * ldc + row : C + (long long)row * ldc + n;
                        const float f = __uint_as_float(v[j]);
                        if (op == kAtomicAdd)
                            atomicAdd(c, f);
                        else if (op == kAccumulate)
                            *c += f;
                        else
                            *c = f;
                    }
                }
            }
        }
    } else if (failed && threadIdx.x == 0) {
        atomicExch(err, 1);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)TN));
}

template <int TN>
cudaError_t launch_umma(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb, float* C,
                        int ldc, GemmOp op, bool trans_c, int split_k, int* err, cudaStream_t st) {
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_gemm_umma<TN>, cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg<TN>::kSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    int kps = (K + split_k - 1) / split_k;
    kps = (kps + TK - 1) / TK * TK;
    split_k = (K + kps - 1) / kps;
    dim3 grid((N + TN - 1) / TN, (M + TM - 1) / TM, split_k);
    k_gemm_umma<TN><<<grid, 128, Cfg<TN>::kSmem, st>>>(M, N, K, A, lda, B, ldb, C, ldc, (int)op, trans_c ? 1 : 0, kps, err);
    return cudaGetLastError();
}

}  // namespace

cudaError_t gemm_bf16_nt_umma(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                              float* C, int ldc, GemmOp op, bool trans_c, int split_k, int* err, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if ((K & 7) || (lda & 7) || (ldb & 7) || K <= 0 || !err) return cudaErrorInvalidValue;
    if (split_k < 1) split_k = 1;
    if (split_k > 1 && op != kAtomicAdd) return cudaErrorInvalidValue;
    if (N <= 32) return launch_umma<32>(M, N, K, A, lda, B, ldb, C, ldc, op, trans_c, split_k, err, st);
    if (N <= 64) return launch_umma<64>(M, N, K, A, lda, B, ldb, C, ldc, op, trans_c, split_k, err, st);
    return launch_umma<128>(M, N, K, A, lda, B, ldb, C, ldc, op, trans_c, split_k, err, st);
}

}  // namespace nn
}  // namespace lbm
