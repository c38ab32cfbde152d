// lbm_device.cuh -- device-side building blocks of the sm_103a D2Q9 cavity library.
//
// Method: Xiang & Shi (arXiv 2211.05009) Sec. 2.1 Eq. 1-3, Eq. 5 and Sec. 2.2 (i)-(iii).
// Storage: SoA f[q][ny][pitch]; rows are multiples of 512 bytes and a warp owns 32*V consecutive
// nodes of one row, so every population is read and written with one 8- or 16-byte vector access
// per thread.  The +-1 x neighbours of a pull come from the adjacent lane by warp shuffle.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbm {

// D2Q9 velocity set and weights, Sec. 2.1 (after Eq. 2), c = 1 (Sec. 3).
// Order: 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1) 6:(-1,1) 7:(-1,-1) 8:(1,-1).
__host__ __device__ constexpr int cx(int j) { return j == 1 || j == 5 || j == 8 ? 1 : (j == 3 || j == 6 || j == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int j) { return j == 2 || j == 5 || j == 6 ? 1 : (j == 4 || j == 7 || j == 8 ? -1 : 0); }
__host__ __device__ constexpr double wd(int j) { return j == 0 ? 4.0 / 9.0 : (j < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

constexpr int kMaxProbes = 4;
constexpr int kInterval = 100;  // Eq. 6 compares fields 100 steps apart

// ------------------------------------------------------------------ storage traits
// V = nodes per 16-byte vector; C = arithmetic type.
template <typename S> struct St;
template <> struct St<double> {
    static constexpr int V = 2;
    using C = double;
    __device__ static double to(double v) { return v; }
    __device__ static double from(double v) { return v; }
};
template <> struct St<float> {
    static constexpr int V = 4;
    using C = float;
    __device__ static float to(float v) { return v; }
    __device__ static float from(float v) { return v; }
};
template <> struct St<__half> {
    static constexpr int V = 8;
    using C = float;
    __device__ static float to(__half v) { return __half2float(v); }
    __device__ static __half from(float v) { return __float2half_rn(v); }
};
template <> struct St<__nv_bfloat16> {
    static constexpr int V = 8;
    using C = float;
    __device__ static float to(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
};

// LBM_Q16S: one 16-bit code per population -- sign, 2-bit exponent E, 13-bit mantissa M -- of
// h_j / S_j, with h_j = g_j - w_j rho_ref the deviation from the rest state at a reference density
// 1 + rho_ref (updated at checkpoints) and S_j a power-of-two scale per direction fixed when the
// context is created.  |h| / S = M 2^-15 for E = 0, (1 + M 2^-13) 2^(E-3) for E = 1..3: 13-bit
// precision relative to the value over [S/4, 2S), absolute spacing S 2^-15 below.  Codes are
// converted with integer operations on the FP32 bit pattern: the code's 15 magnitude bits, shifted
// left by 10, are the FP32 pattern of (|h| / S) 2^-124 (E = 0 gives FP32 subnormals, which the
// multiply by 2^124 S keeps; the library is built without flush-to-zero).
struct q16 {
    unsigned short bits;
};
template <> struct St<q16> {
    static constexpr int V = 8;
    using C = float;
};

template <typename S> inline constexpr bool kIsQ16 = false;
template <> inline constexpr bool kIsQ16<q16> = true;

struct QCodec {
    float dec[9];  // 2^124 S_j
    float enc[9];  // 2^-124 / S_j
};

// code (low 16 bits) -> h
__device__ __forceinline__ float q16_decode(unsigned code, float dec) {
    return __uint_as_float(((code & 0x7fffu) << 10) | ((code & 0x8000u) << 16)) * dec;
}
// h -> code, round to nearest with ties to even; beyond the largest code (2 - 2^-13) S the
// magnitude saturates there and *sat becomes true.  NaN saturates too.
__device__ __forceinline__ unsigned q16_encode(float h, float enc, bool& sat) {
    const unsigned b = __float_as_uint(h * enc);
    const unsigned a = b & 0x7fffffffu;
    const unsigned r = (a + 0x1ffu + ((a >> 10) & 1u)) >> 10;
    sat |= r > 0x7fffu;
    return min(r, 0x7fffu) | ((b >> 16) & 0x8000u);
}

// 16-byte vector load/store of V storage elements, converted to/from C.
template <typename S>
__device__ __forceinline__ void vload(const S* __restrict__ p, typename St<S>::C (&out)[St<S>::V]) {
    constexpr int V = St<S>::V;
    union { uint4 u; S s[V]; } b;
    b.u = __ldg(reinterpret_cast<const uint4*>(p));
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = St<S>::to(b.s[i]);
}
template <typename S>
__device__ __forceinline__ void vstore(S* __restrict__ p, const typename St<S>::C (&in)[St<S>::V]) {
    constexpr int V = St<S>::V;
    union { uint4 u; S s[V]; } b;
#pragma unroll
    for (int i = 0; i < V; ++i) b.s[i] = St<S>::from(in[i]);
    *reinterpret_cast<uint4*>(p) = b.u;
}

// ------------------------------------------------------------------ arguments
struct ProbeSet {
    int n;
    int px[kMaxProbes], py[kMaxProbes], every[kMaxProbes];
    long long start[kMaxProbes];  // global step at which the probe was added
    long long cap[kMaxProbes];
    double* series[kMaxProbes];
};

// Device-resident state shared by every launch of a context.
struct DevState {
    long long base;       // global step index of the last 100-step checkpoint
    double residual;      // Eq. 6 at the last checkpoint
    double mass;          // sum rho at the last checkpoint
    double num, den;      // Eq. 6 numerator / denominator
    long long at_step;    // global step of that checkpoint
    int valid;            // 1 once a checkpoint exists
    int pad;
    double scalar;        // result of the last on-demand reduction (mass)
    double ext[6];        // stream-function window extrema: min, imin, jmin, max, imax, jmax
    // LBM_Q16S reference density (rho_ref of the stored deviations): [0] of the current
    // populations, [1] the one the next checkpoint step stores against (from the last mass)
    double rho_ref[2];
    int q16_saturated;    // a checkpoint step stored a population beyond the LBM_Q16S range
    int pad2;
};

struct StepArgs {
    const void* src;
    void* dst;
    int nx, ny;
    long long pitch;  // elements per row
    long long plane;  // pitch * ny
    double omega;     // 1/tau
    double U;         // lid speed
    float omega_f, U_f;  // the same in FP32 (no FP64 conversion in FP32 kernels)
    int corner_moving;
    int s;            // steps since the last checkpoint (0..99) of the state being advanced
    DevState* state;
    ProbeSet probes;
    void* snap;        // [2][ny][pitch] Eq. 6 velocity snapshot, arithmetic type (REDUCE only)
    double* partials;  // [blocks][3]               (REDUCE only)
    QCodec q;          // LBM_Q16S scales (unused by the other storage types)
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace lbm
