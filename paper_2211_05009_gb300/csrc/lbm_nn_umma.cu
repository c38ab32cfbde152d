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

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
}

// Geometry of the convolution form (CONV = true): image width W, 64-channel blocks per tap cb.
struct ConvGeo {
    int W, cb;
};

// CONV = false: the GEMM above.  CONV = true: A is a 3x3, padding-1 convolution input stored
// channels-last in BF16 ([H][W][Cp], Cp = cb * 64) and K is ordered tap-major (k = tap * Cp + c,
// tap = ky * 3 + kx).  The 128 pixels of an M tile are 128 consecutive pixels of one row (W a
// multiple of 128) or 128 / W whole rows (W dividing 128), so the A tile of K step t -- tap
// t / cb, channels (t % cb) * 64 .. +63 -- is one 3-D TMA box of that shape shifted by
// (kx - 1, ky - 1) pixels: the TMA fills the image border with zeros, and the stage lands in
// shared memory exactly as the GEMM's 128 x 64 A tile does.  No gather runs on the SM.
template <bool CONV>
__global__ void __launch_bounds__(128, 1)
    k_gemm_tc05(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N, int K,
                float* __restrict__ C, int ldc, int op, int trans_c, int k_per_split, int tn, int cols, int stages,
                int* err, ConvGeo geo) {
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
            if constexpr (CONV) {
                const int tap = t / geo.cb;
                const int c0 = (t - tap * geo.cb) * TK;
                const int x = (geo.W > TM ? m0 % geo.W : 0) + tap % 3 - 1;
                tma_load_3d(sA(s), &tmA, c0, x, m0 / geo.W + tap / 3 - 1, sa(&full[s]));
            } else {
                tma_load_2d(sA(s), &tmA, kb + t * TK, m0, sa(&full[s]));
            }
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

// ------------------------------------------------------------------ implicit-GEMM convolution
// The same product with A = the pixel-major im2col of a 3x3, padding-1 convolution input, never
// written to memory.  Per 64-wide K step the CTA first copies, with coalesced loads, the input
// window its 128 pixels need -- the (at most 8) channels of that K range, the tile's pixel rows
// plus one halo row above and below, the tile's columns plus one halo column each side, zeros
// outside the image -- into shared memory; then every thread builds one row (pixel) of the
// 128 x 64 A stage from that window (k = ci*9 + ky*3 + kx, zeros past C*9), rounds it to BF16
// exactly as the explicit im2col does, and writes it in the 128-byte swizzle layout (16-byte
// chunk c of row r at r*128 + ((c ^ (r & 7)) * 16)).  B (the weights) still arrives by TMA.  The
// "full" barrier of a stage takes 128 thread arrivals (each after a proxy fence, so the tensor
// cores see the generic-proxy stores) plus the TMA's.  The CTA moves through the K steps together
// (block barriers around the window), and every decision to stop is taken block-wide.
struct ConvIn {
    const float* x1;
    const float* x2;
    int c1, c2, H, W;
    int win_floats;  // per-channel window capacity (floats) the launch reserved
};

constexpr int kWinCh = 8;  // channels a 64-wide K range can touch (ceil(64 / 9) + 1)

__device__ __forceinline__ uint32_t bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

// Window geometry of the tile starting at pixel m0: rows wy0 .. wy0+R-1, columns wx0 .. wx0+WC-1.
__host__ __device__ inline void conv_window(int m0, int M, int W, int TMr, int& wy0, int& R, int& wx0, int& WC) {
    const int pend = (m0 + TMr < M ? m0 + TMr : M);
    const int py0 = m0 / W, py1 = (pend - 1) / W;
    wy0 = py0 - 1;
    R = py1 - py0 + 3;
    if (py0 == py1) {
        wx0 = m0 % W - 1;
        WC = pend - m0 + 2;
    } else {
        wx0 = -1;
        WC = W + 2;
    }
}

constexpr int kConvThreads = 256;  // two threads per A row (32 K values each)

__global__ void __launch_bounds__(kConvThreads, 2)
    k_conv_tc05(const ConvIn in, const __grid_constant__ CUtensorMap tmB, int N, int K, float* __restrict__ C,
                int ldc, int op, int trans_c, int tn, int cols, int stages, int* err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int stage_bytes = kTileA + tn * TK * 2;
    // two input windows (step t and the prefetch of t+1), each [kWinCh][win_floats] + a zero slot
    const int win_stride = kWinCh * in.win_floats + 4;
    float* win_base = reinterpret_cast<float*>(base + (size_t)stages * stage_bytes);
    uint64_t* full = reinterpret_cast<uint64_t*>(win_base + 2 * (size_t)win_stride);
    uint64_t* empty = full + stages;
    uint64_t* done = empty + stages;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
    __shared__ volatile int abort_flag;
    __shared__ int koff[TK];  // window offset of each K value of the step (from a pixel's corner; -1: zero)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long P = (long long)in.H * in.W;
    const int M = (int)P, W = in.W;
    const int m0 = blockIdx.y * TM, n0 = blockIdx.x * tn;
    const int nk = (K + TK - 1) / TK;
    const int C_in = in.c1 + in.c2, CK = C_in * 9;
    const int zero_slot = kWinCh * in.win_floats;  // always 0: read for K values past C*9
    auto sA = [&](int s) { return sa(base + (size_t)s * stage_bytes); };
    auto sB = [&](int s) { return sa(base + (size_t)s * stage_bytes + kTileA); };

    if (threadIdx.x == 0) {
        abort_flag = 0;
        win_base[zero_slot] = 0.f;
        win_base[win_stride + zero_slot] = 0.f;
        for (int s = 0; s < stages; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(sa(&full[s])), "r"(kConvThreads + 1));
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
    if (threadIdx.x == 0) asm volatile("prefetch.tensormap [%0];\n" ::"l"(reinterpret_cast<uint64_t>(&tmB)) : "memory");

    int wy0, R, wx0, WC;
    conv_window(m0, M, W, TM, wy0, R, wx0, WC);
    // this thread's pixel (row of A), half of the K step, and its 3x3 corner in the window
    const int r = threadIdx.x & (TM - 1), half = threadIdx.x >> 7;
    const int pm = m0 + r;
    const bool row_ok = pm < M;
    const int off0 = row_ok ? (pm / W - 1 - wy0) * WC + (pm % W - 1 - wx0) : 0;
    const bool issuer = threadIdx.x == 32;  // warp 1, lane 0
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(tn >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
    // asynchronous copy (cp.async, 4 bytes, zero fill outside the image) of the input window of
    // the channels K step tt touches into window buffer tt & 1
    auto load_window = [&](int tt) {
        const int kk0 = tt * TK, c0 = kk0 / 9;
        const int nch = min(C_in, (kk0 + TK + 8) / 9) - c0;
        float* wb = win_base + (size_t)(tt & 1) * win_stride;
        for (int q = 0; q < nch * R; ++q) {  // window rows, channel-major
            const int c = q / R, wy = q - c * R;
            const int ci = c0 + c, y = wy0 + wy;
            const float* src = ci < in.c1 ? in.x1 + (long long)ci * P : in.x2 + (long long)(ci - in.c1) * P;
            const bool yin = y >= 0 && y < in.H;
            for (int wx = threadIdx.x; wx < WC; wx += kConvThreads) {
                const int x = wx0 + wx;
                const bool inside = yin && x >= 0 && x < W;
                const float* g = inside ? src + (long long)y * W + x : in.x1;  // any valid address when empty
                asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa(wb + (size_t)c * in.win_floats + wy * WC + wx)),
                             "l"(g), "r"(inside ? 4 : 0)
                             : "memory");
            }
        }
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };
    if (nk > 0) load_window(0);
    int t = 0;
    for (; t < nk; ++t) {
        const int s = t % stages;
        // the stage is free once the MMAs of t - stages completed (thread 0 waits; the block
        // barrier passes the news on, and any failure stops every thread at the same point)
        bool bad = false;
        if (threadIdx.x == 0 && t >= stages) bad = !mbar_wait(sa(&empty[s]), ((t / stages) - 1) & 1, nullptr);
        if (__syncthreads_or(bad || abort_flag)) {
            if (threadIdx.x == 0) abort_flag = 1;
            break;
        }
        const int k0 = t * TK;
        const int ci0 = k0 / 9;
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(sa(&full[s])), "r"(tn * TK * 2)
                         : "memory");
            tma_load_2d(sB(s), &tmB, k0, n0, sa(&full[s]));
        }
        if (threadIdx.x < TK) {  // offsets of k0 .. k0+63 in the window; past C*9 the zero slot
            const int k = k0 + threadIdx.x;
            const int cl = k / 9 - ci0, tap = k % 9, ky = tap / 3;
            koff[threadIdx.x] = k < CK ? cl * in.win_floats + ky * WC + (tap - 3 * ky) : -1;
        }
        // this step's window (copied during the previous step) is in; then start the next one
        asm volatile("cp.async.wait_all;\n" ::: "memory");
        __syncthreads();
        if (t + 1 < nk) load_window(t + 1);
        const float* win = win_base + (size_t)(t & 1) * win_stride;
        // this thread's 32 K values of row r
        uint32_t w[16];
#pragma unroll
        for (int j2 = 0; j2 < 16; ++j2) {
            const int j = half * 32 + 2 * j2;
            const int kf0 = koff[j], kf1 = koff[j + 1];
            // off0 + kf stays inside the window (kf <= 7 win_floats + 2 WC + 2, off0 <= (R-3) WC + WC-3);
            // K values past C*9 and pixels past the image read the zero slot
            const float lo = win[(row_ok && kf0 >= 0) ? off0 + kf0 : zero_slot];
            const float hi = win[(row_ok && kf1 >= 0) ? off0 + kf1 : zero_slot];
            w[j2] = bf16x2(lo, hi);
        }
        unsigned char* rowp = base + (size_t)s * stage_bytes + (size_t)r * 128;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const int chunk = half * 4 + c;
            *reinterpret_cast<uint4*>(rowp + ((chunk ^ (r & 7)) << 4)) =
                make_uint4(w[4 * c], w[4 * c + 1], w[4 * c + 2], w[4 * c + 3]);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(sa(&full[s])) : "memory");
        if (issuer) {
            // MMA issuer: stage t once all rows and the weight tile are in
            if (!mbar_wait(sa(&full[s]), (t / stages) & 1, nullptr)) {
                abort_flag = 1;  // the next block-wide check stops everyone
            } else {
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
        }
    }
    if (issuer)  // arrives once every MMA issued above has completed (at once if none was issued)
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(sa(done)));
    if (threadIdx.x == 0 && abort_flag) {
        // weight copies already issued must land before the CTA may leave (bounded waits)
        for (int u = t > stages ? t - stages : 0; u < t; ++u) mbar_wait(sa(&full[u % stages]), (u / stages) & 1, nullptr);
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");  // a window prefetch in flight after an early stop
    __syncwarp();

    // epilogue, as in k_gemm_tc05, by warps 0..3 (TMEM lanes 32w .. 32w+31)
    const bool fin = mbar_wait(sa(done), 0, nullptr);
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (warp < 4 && fin && !abort_flag && nk > 0) {
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
    if (threadIdx.x == 0 && (!fin || abort_flag)) atomicExch(err, 1);
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

// Channels-last activation [H][W][Cp] bfloat16 as a 3-D tensor {Cp, W, H}, box {64, bw, bh} with
// bw * bh = 128 pixels, 128-byte swizzle, zero fill out of range (the convolution's border).
bool make_act_map(CUtensorMap* m, const __nv_bfloat16* X, int H, int W, int Cp, int bw, int bh) {
    auto enc = encoder();
    if (!enc) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)Cp, (cuuint64_t)W, (cuuint64_t)H};
    const cuuint64_t strides[2] = {(cuuint64_t)Cp * 2, (cuuint64_t)W * Cp * 2};
    const cuuint32_t box[3] = {(cuuint32_t)TK, (cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<__nv_bfloat16*>(X), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// X[p][c] = bf16(x1 ++ x2 channel c at pixel p), zero for c >= c1 + c2: one pixel and 8 channels per
// thread (reads coalesced along the pixels, one 16-byte store), rounding as the explicit im2col.
__global__ void k_channels_last_bf16(const float* __restrict__ x1, int c1, const float* __restrict__ x2, int c2,
                                     long long P, int Cp, __nv_bfloat16* __restrict__ X) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int cg = blockIdx.y * 8;
    float v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const int c = cg + j;
        v[j] = c < c1 ? x1[(long long)c * P + p] : (c < c1 + c2 ? x2[(long long)(c - c1) * P + p] : 0.f);
    }
    uint4 w;
    w.x = bf16x2(v[0], v[1]);
    w.y = bf16x2(v[2], v[3]);
    w.z = bf16x2(v[4], v[5]);
    w.w = bf16x2(v[6], v[7]);
    *reinterpret_cast<uint4*>(X + p * Cp + cg) = w;
}

// Wtap[n][tap * Cp + c] = Wt[n][c * 9 + tap] for c < C, zero for C <= c < Cp.
__global__ void k_weights_tap_major(const __nv_bfloat16* __restrict__ Wt, int ldk, int C, int N, int Cp,
                                    __nv_bfloat16* __restrict__ Wtap) {
    const long long per = 9ll * Cp;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= per * N) return;
    const int n = (int)(i / per), r = (int)(i - n * per), tap = r / Cp, c = r - tap * Cp;
    Wtap[i] = c < C ? Wt[(long long)n * ldk + c * 9 + tap] : __float2bfloat16_rn(0.f);
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
            e = cudaFuncSetAttribute(k_gemm_tc05<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
            if (e != cudaSuccess) return e;
            if (dev < 64) opted[dev] = p.smem;
        }
    }
    int kps = (K + split_k - 1) / split_k;
    kps = (kps + TK - 1) / TK * TK;
    split_k = (K + kps - 1) / kps;
    const dim3 grid(p.tiles_n, (M + TM - 1) / TM, split_k);
    k_gemm_tc05<false><<<grid, 128, p.smem, st>>>(ma, mb, M, N, K, C, ldc, (int)op, trans_c ? 1 : 0, kps, p.tn, p.cols,
                                                   p.stages, err, ConvGeo{0, 0});
    return cudaGetLastError();
}

cudaError_t conv3x3_bf16_umma(const float* x1, int c1, const float* x2, int c2, int H, int W, int K,
                              const __nv_bfloat16* Wt, int N, float* C, int ldc, GemmOp op, bool trans_c, int* err,
                              cudaStream_t st) {
    const long long P = (long long)H * W;
    if (P <= 0 || N <= 0) return cudaSuccess;
    if (!x1 || c1 < 1 || c2 < 0 || (c2 > 0 && !x2) || P > 0x7fffffffll) return cudaErrorInvalidValue;
    if ((K & 7) || K < (c1 + c2) * 9 || !err || ((uintptr_t)Wt & 15)) return cudaErrorInvalidValue;
    Plan p = plan_for(N);
    if (p.tiles_n != 1 || p.tn > 256) return cudaErrorInvalidValue;  // one N tile (N <= 256)
    // the largest input window over the tiles (floats per channel), and the stage ring that fits
    // beside it in the per-CTA budget (two CTAs per SM)
    int win = 0;
    for (long long m0 = 0; m0 < P; m0 += TM) {
        int wy0, R, wx0, WC;
        conv_window((int)m0, (int)P, W, TM, wy0, R, wx0, WC);
        win = R * WC > win ? R * WC : win;
    }
    win = (win + 3) / 4 * 4;
    const int win_bytes = 2 * (kWinCh * win + 4) * 4;  // two windows, each with its zero slot
    const int stage = kTileA + p.tn * TK * 2;
    p.stages = (kSmemBudget - kSmemExtra - win_bytes) / stage;
    if (p.stages > 6) p.stages = 6;
    if (p.stages < 2) return cudaErrorInvalidValue;  // window too wide for the budget: use the explicit im2col
    p.smem = p.stages * stage + win_bytes + kSmemExtra;
    CUtensorMap mb;
    if (!make_map(&mb, Wt, N, K, K, p.tn)) return cudaErrorInvalidValue;
    {
        static std::mutex mu;
        static int opted[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 64 || p.smem > opted[dev]) {
            e = cudaFuncSetAttribute(k_conv_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
            if (e != cudaSuccess) return e;
            if (dev < 64) opted[dev] = p.smem;
        }
    }
    const ConvIn in{x1, x2, c1, c2, H, W, win};
    const dim3 grid(1, (unsigned)((P + TM - 1) / TM), 1);
    k_conv_tc05<<<grid, kConvThreads, p.smem, st>>>(in, mb, N, K, C, ldc, (int)op, trans_c ? 1 : 0, p.tn, p.cols, p.stages, err);
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace lbm

namespace lbm {
namespace nn {

int conv_cp(int c) { return (c + TK - 1) / TK * TK; }

cudaError_t weights_tap_major(const __nv_bfloat16* Wt, int ldk, int C, int N, __nv_bfloat16* Wtap, cudaStream_t st) {
    if (N <= 0 || C <= 0) return cudaSuccess;
    if (!Wt || !Wtap || ldk < 9 * C) return cudaErrorInvalidValue;
    const long long total = 9ll * conv_cp(C) * N;
    k_weights_tap_major<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(Wt, ldk, C, N, conv_cp(C), Wtap);
    return cudaGetLastError();
}

cudaError_t conv3x3_bf16_tma(const float* x1, int c1, const float* x2, int c2, int H, int W, const __nv_bfloat16* Wtap,
                             int N, float* C, int ldc, GemmOp op, bool trans_c, __nv_bfloat16* xs, int* err,
                             cudaStream_t st) {
    const long long P = (long long)H * W;
    if (P <= 0 || N <= 0) return cudaSuccess;
    if (!x1 || c1 < 1 || c2 < 0 || (c2 > 0 && !x2) || !Wtap || !xs || !err) return cudaErrorInvalidValue;
    // tiles of 128 pixels: part of one row, or whole rows; the box's dimensions stay <= 256
    if (P % TM || !(W % TM == 0 || TM % W == 0) || H > 0x7fffffff / W) return cudaErrorInvalidValue;
    if (((uintptr_t)Wtap & 15) || ((uintptr_t)xs & 15)) return cudaErrorInvalidValue;
    const int Cp = conv_cp(c1 + c2), K = 9 * Cp;
    const Plan p = plan_for(N);
    CUtensorMap ma, mb;
    const int bw = W < TM ? W : TM;
    if (!make_act_map(&ma, xs, H, W, Cp, bw, TM / bw) || !make_map(&mb, Wtap, N, K, K, p.tn)) return cudaErrorInvalidValue;
    {
        static std::mutex mu;
        static int opted[64] = {};
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        if (dev >= 64 || p.smem > opted[dev]) {
            e = cudaFuncSetAttribute(k_gemm_tc05<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, p.smem);
            if (e != cudaSuccess) return e;
            if (dev < 64) opted[dev] = p.smem;
        }
    }
    k_channels_last_bf16<<<dim3((unsigned)((P + 255) / 256), (unsigned)(Cp / 8)), 256, 0, st>>>(x1, c1, x2, c2, P, Cp, xs);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid(p.tiles_n, (unsigned)(P / TM), 1);
    k_gemm_tc05<true><<<grid, 128, p.smem, st>>>(ma, mb, (int)P, N, K, C, ldc, (int)op, trans_c ? 1 : 0, K, p.tn, p.cols,
                                                  p.stages, err, ConvGeo{W, Cp / TK});
    return cudaGetLastError();
}

}  // namespace nn
}  // namespace lbm
