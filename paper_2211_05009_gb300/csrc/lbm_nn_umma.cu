// lbm_nn_umma.cu -- the warm-start network's BF16 GEMM on the 5th-generation tensor cores
// (tcgen05.mma, accumulator in tensor memory), sm_103a.
//
//   C[M][N] (op)= sum_k A[M][K] * B[N][K]      (both K-contiguous; same contract as gemm_bf16_nt)
//
// CTA tile 128 x TN with TN = N rounded up to 16 (N <= 256; larger N is cut into equal tiles of at
// most 256), K step 64.  Operand tiles arrive by TMA (cp.async.bulk.tensor, 128-byte swizzle,
// out-of-range rows and K filled with zeros) into a ring of 2..6 shared-memory stages, each
// guarded by a "full" mbarrier (TMA transaction bytes) and an "empty" mbarrier (tcgen05.commit of
// the MMAs that read it).  Warp 0 lane 0 issues the copies, warp 1 lane 0 the MMAs (four K = 16
// steps per stage, descriptors advanced 32 bytes inside the swizzle atom), warp 2 owns the TMEM
// allocation; after the last commit every warp reads its 32 accumulator lanes back with
// tcgen05.ld and stores them (row-major or transposed, store / accumulate / atomic add for
// split-K over gridDim.z).  Shared memory per CTA is held under 110 KB so two CTAs share an SM
// (one's epilogue overlaps the other's main loop) and their TMEM columns (<= 2 x 256) fit the
// SM's 512.  Every mbarrier wait is bounded by a clock limit: on timeout the CTA records an error,
// lets its issued copies and MMAs finish (bounded), frees its TMEM and returns.
#include <cuda.h>          // CUtensorMap and the encoder's types; the encoder itself is fetched
#include <cudaTypedefs.h>  // through the runtime's driver entry point (no link against libcuda)
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "lbm_nn_gemm.cuh"

namespace lbm {
namespace nn {

namespace {

constexpr int TM = 128, TK = 64;
constexpr int kTileA = TM * TK * 2;           // 16 KB
constexpr int kSmemBudget = 110 * 1024;       // per CTA: two CTAs per SM
constexpr int kSmemExtra = 1024 + 256;        // 1024-byte alignment slack + barriers / TMEM slot
constexpr long long kWaitCycles = 2000000000ll;  // ~1 s

struct Plan {
    int tn, tiles_n, cols, stages, smem;
};

Plan plan_for(int N) {
    Plan p{};
    p.tiles_n = (N + 255) / 256;
    p.tn = ((N + p.tiles_n - 1) / p.tiles_n + 15) / 16 * 16;  // multiple of 16, <= 256
    p.cols = 32;
    while (p.cols < p.tn) p.cols <<= 1;  // TMEM allocation: a power of two >= 32
    const int stage = kTileA + p.tn * TK * 2;
    p.stages = (kSmemBudget - kSmemExtra) / stage;
    if (p.stages > 6) p.stages = 6;
    p.smem = p.stages * stage + kSmemExtra;
    return p;
}

__device__ __forceinline__ uint32_t sa(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

// tcgen05 shared-memory descriptor, K-major operand in the 128-byte swizzle layout: start >> 4,
// leading offset 16 B (unused by this layout), stride 1024 B between 8-row groups, version 1,
// base offset 0 (stage tiles are 1024-aligned), layout type 2 = 128-byte swizzle.
__device__ __forceinline__ uint64_t desc_sw128(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)(16 >> 4) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase of the given parity; gives up early when another role aborted
// (abort != nullptr) or after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, const volatile int* abort) {
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if ((abort && *abort) || clock64() - t0 > kWaitCycles) return false;
    }
    return true;
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}

__global__ void __launch_bounds__(128, 1)
    k_gemm_tc05(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                float* __restrict__ C, int ldc, int op, int trans_c, int k_per_split, int tn, int cols, int stages,
                int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = kTileA + tn * TK * 2;
    uint64_t* full = reinterpret_cast<uint64_t*>(base + (size_t)stages * stage_bytes);
    uint64_t* empty = full + stages;
    uint64_t* done = empty + stages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * tn;
    const int kb = blockIdx.z * k_per_split;
    const int ke = min(K, kb + k_per_split);
    const int nk = ke > kb ? (ke - kb + TK - 1) / TK : 0;
    auto sA = [&](int s) { return sa(base + (size_t)s * stage_bytes); };
    auto sB = [&](int s) { return sa(base + (size_t)s * stage_bytes + kTileA); };

    if (threadIdx.x == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(&empty[s])));
        }
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(sa(done)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(sa(tmem_slot)), "r"((uint32_t)cols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = *tmem_slot;

    if (warp == 0 && lane == 0) {
        // producer: TMA copies of stage t % stages once the MMAs of t - stages released it
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmA)) : "memory");
        asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");
        int t = 0;
        for (; t < nk; ++t) {
            const int s = t % stages;
            if (t >= stages && !mbar_wait(sa(&empty[s]), ((t / stages) - 1) & 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(&full[s])), "r"(stage_bytes)
                         : "memory");
            tma_load_2d(sA(s), &tmA, kb + t * TK, m0, sa(&full[s]));
            tma_load_2d(sB(s), &tmB, kb + t * TK, n0, sa(&full[s]));
        }
        if (abort_flag)  // the copies already issued must land before the CTA may leave
            for (int u = t > stages ? t - stages : 0; u < t; ++u) mbar_wait(sa(&full[u % stages]), (u / stages) & 1, nullptr);
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: four K = 16 steps per stage, accumulate after the first
        const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(tn >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
        for (int t = 0; t < nk; ++t) {
            const int s = t % stages;
            if (!mbar_wait(sa(&full[s]), (t / stages) & 1, &abort_flag)) {
                abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
#pragma unroll
            for (int kk = 0; kk < TK / 16; ++kk) {
                const uint64_t da = desc_sw128(sA(s) + kk * 32);
                const uint64_t db = desc_sw128(sB(s) + kk * 32);
                const uint32_t acc = (t > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
                    "l"(da), "l"(db), "r"(idesc), "r"(acc));
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(&empty[s])));
        }
        // arrives once every MMA issued above has completed (at once if none was issued)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(done)));
    }
    __syncwarp();

    // epilogue: warp w reads TMEM lanes 32w .. 32w+31 (= tile rows), 16 columns per load
    const bool ok = mbar_wait(sa(done), 0, nullptr);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (ok && !abort_flag && nk > 0) {
        const int row = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < tn; c0 += 16) {
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
    }
    if (threadIdx.x == 0 && (!ok || abort_flag)) atomicExch(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"((uint32_t)cols));
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    });
    return fn;
}

// Row-major [rows][K] bfloat16 (row stride ld elements) as a 2-D tensor {K, rows}, box {64, box_rows},
// 128-byte swizzle, zero fill out of range.
bool make_map(CUtensorMap* m, const __nv_bfloat16* X, int rows, int K, int ld, int box_rows) {
    auto enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)TK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

cudaError_t gemm_bf16_nt_umma(int M, int N, int K, const __nv_bfloat16* A, int lda, const __nv_bfloat16* B, int ldb,
                              float* C, int ldc, GemmOp op, bool trans_c, int split_k, int* err, cudaStream_t st) {
    if (M <= 0 || N <= 0) return cudaSuccess;
    if ((K & 7) || (lda & 7) || (ldb & 7) || K <= 0 || !err) return cudaErrorInvalidValue;
    if (((uintptr_t)A & 15) || ((uintptr_t)B & 15)) return cudaErrorInvalidValue;  // TMA: 16-byte aligned bases
    if (split_k < 1) split_k = 1;
    if (split_k > 1 && op != kAtomicAdd) return cudaErrorInvalidValue;
    const Plan p = plan_for(N);
    CUtensorMap ma, mb;
    if (!make_map(&ma, A, M, K, lda, TM) || !make_map(&mb, B, N, K, ldb, p.tn)) return cudaErrorInvalidValue;
    {
        // opt in to the plan's dynamic shared memory: the attribute belongs to the current device,
        // so the largest size set so far is kept per device (thread-safe)
        static std::mutex mu;
        static int opted[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 64 || p.smem > opted[dev]) {
            e = cudaFuncSetAttribute(k_gemm_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
            if (e != cudaSuccess) return e;
            if (dev < 64) opted[dev] = p.smem;
        }
    }
    int kps = (K + split_k - 1) / split_k;
    kps = (kps + TK - 1) / TK * TK;
    split_k = (K + kps - 1) / kps;
    const dim3 grid(p.tiles_n, (M + TM - 1) / TM, split_k);
    k_gemm_tc05<<<grid, 128, p.smem, st>>>(ma, mb, M, N, K, C, ldc, (int)op, trans_c ? 1 : 0, kps, p.tn, p.cols,
                                            p.stages, err);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace lbm
