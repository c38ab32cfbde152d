// lbm_aux.cu -- per-run and on-demand kernels around the time step: initial state, field
// import/export, mass reduction and the stream function with vortex-centre search.
//
//   init / set_moments   Sec. 2.2 (i): f = f^eq(rho, u) (Eq. 2)
//   moments              Eq. 3 of the stored post-collision populations
//   mass                 sum_x rho(x), FP64 across nodes (two-stage, fixed order -> deterministic)
//   stream_function      Psi with u_x = dPsi/dy, Psi(y = 0) = 0, trapezoid rule in y, integrated in
//                        FP64; the extrema and their nodes give the vortex strengths and centres of
//                        Table 1 / Table 2.
// Per-node arithmetic runs in the storage's arithmetic type C (FP32 for the FP32/16-bit storage
// types, FP64 for FP64); FP64 is used from the first cross-node sum on.  On this GPU FP64 issue
// rate is a small fraction of FP32's, so per-node FP64 math would dominate these kernels.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

int storage_bytes(int dtype) { return dtype == 0 ? 8 : (dtype <= 2 ? 4 : 2); }

long long row_pitch(int dtype, int nx) {
    const long long per_warp = 32ll * (16 / storage_bytes(dtype));
    return (nx + per_warp - 1) / per_warp * per_warp;
}

// Deviation equilibrium g_j = w_j (drho + rho A_j(u)) (Eq. 2), in the arithmetic type.
template <typename C>
__device__ __forceinline__ C geq_c(int j, C drho, C ux, C uy) {
    const C cu = C(cx(j)) * ux + C(cy(j)) * uy;
    const C A = cu * (C(3.0) + C(4.5) * cu) - C(1.5) * (ux * ux + uy * uy);
    return C(wd(j)) * (drho + (C(1.0) + drho) * A);
}

// LBM_Q16S reference density of the stored populations (0 for the other storage types).
template <typename S>
__device__ __forceinline__ float ref_density(const FieldArgs& a) {
    if constexpr (kIsQ16<S>) return float(__ldcg(&a.st->rho_ref[0]));
    else return 0.f;
}

// g_j = f_j - w_j of one stored population (sref: ref_density).
template <typename S, bool SHIFTED>
__device__ __forceinline__ typename St<S>::C load_g(const S* f, long long idx, int j, const QCodec& q,
                                                    float sref) {
    using C = typename St<S>::C;
    if constexpr (kIsQ16<S>) {
        return fmaf(float(wd(j)), sref, q16_decode(f[idx].bits, q.dec[j]));
    } else {
        const C v = St<S>::to(f[idx]);
        return SHIFTED ? v : v - C(wd(j));
    }
}

// Store g_j = f_j - w_j as one population.
template <typename S, bool SHIFTED>
__device__ __forceinline__ void store_g(S* f, long long idx, int j, typename St<S>::C g, const QCodec& q,
                                        float sref) {
    using C = typename St<S>::C;
    if constexpr (kIsQ16<S>) {
        bool sat = false;
        f[idx].bits = (unsigned short)q16_encode(g - float(wd(j)) * sref, q.enc[j], sat);
    } else {
        f[idx] = St<S>::from(SHIFTED ? g : g + C(wd(j)));
    }
}

// Moments (Eq. 3) of the stored populations at linear index k.
template <typename S, bool SHIFTED>
__device__ __forceinline__ void node_moments(const S* f, long long plane, long long k, const QCodec& q,
                                             float sref, typename St<S>::C& drho, typename St<S>::C& ux,
                                             typename St<S>::C& uy) {
    using C = typename St<S>::C;
    C g[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = load_g<S, SHIFTED>(f, j * plane + k, j, q, sref);
    drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const C rho = C(1.0) + drho;
    ux = ((g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7])) / rho;
    uy = ((g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8])) / rho;
}

// ------------------------------------------------------------------ init / set_moments
// d/dk of a node field along one grid line (spacing 1): central inside, three-point one-sided
// at the two ends (both exact for quadratics).  line[k * stride] is node k; n >= 3.
__device__ __forceinline__ double d_line(const double* line, long long stride, int i, int n) {
    if (i == 0) return (-3.0 * line[0] + 4.0 * line[stride] - line[2 * stride]) * 0.5;
    if (i == n - 1)
        return (3.0 * line[(n - 1) * stride] - 4.0 * line[(n - 2) * stride] + line[(n - 3) * stride]) * 0.5;
    return (line[(i + 1) * stride] - line[(i - 1) * stride]) * 0.5;
}

// neq_tau > 0 (only with given fields): add (1 - 1/tau) f^neq_j, the first-order Chapman-Enskog
// non-equilibrium part f^neq_j = -tau w_j rho / c_s^2 (c_ja c_jb - c_s^2 delta_ab) d_a u_b of BGK,
// so that the start carries the stress of its velocity field (no counterpart in the paper).
template <typename S, bool SHIFTED>
__global__ void k_init(FieldArgs a, void* snap_v, const double* rho_in, const double* ux_in,
                       const double* uy_in, double neq_tau) {
    using C = typename St<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.pitch || y >= a.ny) return;
    S* f = static_cast<S*>(a.f);
    const long long k = (long long)y * a.pitch + x;
    C drho = C(0), ux = C(0), uy = C(0);
    C dxux = C(0), dyux = C(0), dxuy = C(0), dyuy = C(0);
    const bool neq = neq_tau > 0.0 && rho_in && x < a.nx;
    if (x < a.nx) {
        if (rho_in) {
            const long long d = (long long)y * a.nx + x;
            drho = C(rho_in[d] - 1.0);
            ux = C(ux_in[d]);
            uy = C(uy_in[d]);
            if (neq) {
                const long long row = (long long)y * a.nx;
                dxux = C(d_line(ux_in + row, 1, x, a.nx));
                dxuy = C(d_line(uy_in + row, 1, x, a.nx));
                dyux = C(d_line(ux_in + x, a.nx, y, a.ny));
                dyuy = C(d_line(uy_in + x, a.nx, y, a.ny));
            }
        } else if (y == a.ny - 1 && (a.corner_moving || (x > 0 && x < a.nx - 1))) {
            ux = C(a.U);  // Sec. 2.2 (i): only the lid moves at t = 0
        }
    }
    const C tau = C(neq_tau), keep = neq ? C(1.0) - C(1.0) / tau : C(0);
    const float sref = ref_density<S>(a);
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        C g = geq_c<C>(j, drho, ux, uy);
        if (neq) {
            const C third = C(1.0 / 3.0);
            const C qxx = C(cx(j) * cx(j)) - third, qyy = C(cy(j) * cy(j)) - third, qxy = C(cx(j) * cy(j));
            const C qdu = qxx * dxux + qxy * (dxuy + dyux) + qyy * dyuy;
            g += keep * (-C(3.0) * tau * C(wd(j)) * (C(1.0) + drho) * qdu);
        }
        store_g<S, SHIFTED>(f, j * a.plane + k, j, g, a.q, sref);
    }
    if (snap_v) {
        C* snap = static_cast<C*>(snap_v);
        snap[k] = ux;
        snap[a.plane + k] = uy;
    }
}

// ------------------------------------------------------------------ export / import
template <typename S, bool SHIFTED>
__global__ void k_moments(FieldArgs a, double* rho, double* ux, double* uy) {
    using C = typename St<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    const S* f = static_cast<const S*>(a.f);
    C drho, u, v;
    node_moments<S, SHIFTED>(f, a.plane, (long long)y * a.pitch + x, a.q, ref_density<S>(a), drho, u, v);
    const long long d = (long long)y * a.nx + x;
    if (rho) rho[d] = 1.0 + double(drho);
    if (ux) ux[d] = double(u);
    if (uy) uy[d] = double(v);
}

template <typename S, bool SHIFTED>
__global__ void k_get_pop(FieldArgs a, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, j = blockIdx.z;
    if (x >= a.nx) return;
    const S* f = static_cast<const S*>(a.f);
    const long long k = j * a.plane + (long long)y * a.pitch + x;
    double v;
    if constexpr (kIsQ16<S>) v = double(load_g<S, SHIFTED>(f, k, j, a.q, ref_density<S>(a))) + wd(j);
    else v = SHIFTED ? double(St<S>::to(f[k])) + wd(j) : double(St<S>::to(f[k]));
    out[((long long)j * a.ny + y) * a.nx + x] = v;
}

template <typename S, bool SHIFTED>
__global__ void k_set_pop(FieldArgs a, const double* in) {
    using C = typename St<S>::C;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, j = blockIdx.z;
    if (x >= a.nx) return;
    S* f = static_cast<S*>(a.f);
    const double v = in[((long long)j * a.ny + y) * a.nx + x];
    const long long k = j * a.plane + (long long)y * a.pitch + x;
    if constexpr (kIsQ16<S>) store_g<S, SHIFTED>(f, k, j, C(v - wd(j)), a.q, ref_density<S>(a));
    else f[k] = St<S>::from(C(SHIFTED ? v - wd(j) : v));
}

// ------------------------------------------------------------------ mass
template <typename S, bool SHIFTED>
__global__ void __launch_bounds__(256) k_mass(FieldArgs a, double* partials) {
    using C = typename St<S>::C;
    __shared__ double sh[8];
    const S* f = static_cast<const S*>(a.f);
    const float sref = ref_density<S>(a);
    double acc = 0.0;
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x)
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            const long long k = (long long)y * a.pitch + x;
            C g[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) g[j] = load_g<S, SHIFTED>(f, j * a.plane + k, j, a.q, sref);
            acc += double(((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8]);
        }
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < 8; ++w) s += sh[w];
        partials[blockIdx.x] = s;
    }
}

__global__ void k_mass_finalize(const double* partials, int n, double nodes, DevState* st) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int b = threadIdx.x; b < n; b += 256) s += partials[b];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) st->scalar = nodes + sh[0];
}

// ------------------------------------------------------------------ stream function
// Psi(x, y) = sum_{k<=y} u(k) - u(0)/2 - u(y)/2, the trapezoid sum of (u(k-1) + u(k))/2 for
// k = 1..y.  Three passes over (128-column) x (32-row segment) blocks:
//   1. u_x of every node into a scratch field and the FP64 sum of each column segment;
//   2. each segment adds the sums of the segments below it, walks its rows in FP64, writes Psi
//      (optional) and reduces the window extrema of its block;
//   3. one block merges the block extrema in a fixed order (ties -> smaller row-major index).
constexpr int kPsiCols = 128, kPsiSeg = 32;

struct Ext {
    double vmin, vmax;
    long long imin, imax;  // linear node index y*nx + x, -1 if none
};

__device__ __forceinline__ void ext_merge(Ext& a, const Ext& b) {
    if (b.imin >= 0 && (a.imin < 0 || b.vmin < a.vmin || (b.vmin == a.vmin && b.imin < a.imin))) {
        a.vmin = b.vmin;
        a.imin = b.imin;
    }
    if (b.imax >= 0 && (a.imax < 0 || b.vmax > a.vmax || (b.vmax == a.vmax && b.imax < a.imax))) {
        a.vmax = b.vmax;
        a.imax = b.imax;
    }
}

template <typename S, bool SHIFTED>
__global__ void __launch_bounds__(kPsiCols) k_psi_seg(FieldArgs a, void* uscr_v, double* segsum) {
    using C = typename St<S>::C;
    const int x = blockIdx.x * kPsiCols + threadIdx.x;
    const int seg = blockIdx.y;
    if (x >= a.nx) return;
    const S* f = static_cast<const S*>(a.f);
    C* uscr = static_cast<C*>(uscr_v);
    const int y0 = seg * kPsiSeg, y1 = min(a.ny, y0 + kPsiSeg);
    const float sref = ref_density<S>(a);
    double s = 0.0;
    for (int y = y0; y < y1; ++y) {
        C drho, u, v;
        node_moments<S, SHIFTED>(f, a.plane, (long long)y * a.pitch + x, a.q, sref, drho, u, v);
        uscr[(long long)y * a.nx + x] = u;
        s += double(u);
    }
    segsum[(long long)seg * a.nx + x] = s;
}

template <typename C>
__global__ void __launch_bounds__(kPsiCols) k_psi_walk(int nx, int ny, const C* __restrict__ uscr,
                                                      const double* __restrict__ segsum, double* psi,
                                                      int i0, int i1, int j0, int j1, double* part) {
    __shared__ Ext ex[kPsiCols];
    const int x = blockIdx.x * kPsiCols + threadIdx.x;
    const int seg = blockIdx.y;
    Ext e{INFINITY, -INFINITY, -1, -1};
    if (x < nx) {
        double run = 0.0;
        for (int k = 0; k < seg; ++k) run += segsum[(long long)k * nx + x];
        const double u0 = double(uscr[x]);
        const bool colin = x >= i0 && x < i1;
        const int y0 = seg * kPsiSeg, y1 = min(ny, y0 + kPsiSeg);
        for (int y = y0; y < y1; ++y) {
            const double u = double(uscr[(long long)y * nx + x]);
            run += u;
            const double p = y == 0 ? 0.0 : run - 0.5 * u0 - 0.5 * u;
            if (psi) psi[(long long)y * nx + x] = p;
            if (colin && y >= j0 && y < j1) {
                const long long id = (long long)y * nx + x;
                if (e.imin < 0 || p < e.vmin) { e.vmin = p; e.imin = id; }
                if (e.imax < 0 || p > e.vmax) { e.vmax = p; e.imax = id; }
            }
        }
    }
    ex[threadIdx.x] = e;
    __syncthreads();
    for (int o = kPsiCols / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) ext_merge(ex[threadIdx.x], ex[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        part[4 * b + 0] = ex[0].vmin;
        part[4 * b + 1] = (double)ex[0].imin;
        part[4 * b + 2] = ex[0].vmax;
        part[4 * b + 3] = (double)ex[0].imax;
    }
}

__global__ void k_psi_finalize(const double* part, int nblocks, int nx, DevState* st) {
    __shared__ Ext ex[256];
    Ext e{INFINITY, -INFINITY, -1, -1};
    for (int b = threadIdx.x; b < nblocks; b += 256) {
        const Ext o{part[4ll * b], part[4ll * b + 2], (long long)part[4ll * b + 1], (long long)part[4ll * b + 3]};
        ext_merge(e, o);
    }
    ex[threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) ext_merge(ex[threadIdx.x], ex[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        e = ex[0];
        st->ext[0] = e.vmin;
        st->ext[1] = e.imin < 0 ? -1.0 : (double)(e.imin % nx);
        st->ext[2] = e.imin < 0 ? -1.0 : (double)(e.imin / nx);
        st->ext[3] = e.vmax;
        st->ext[4] = e.imax < 0 ? -1.0 : (double)(e.imax % nx);
        st->ext[5] = e.imax < 0 ? -1.0 : (double)(e.imax / nx);
    }
}

size_t psi_scratch_doubles(int nx, int ny) {
    const size_t nseg = (ny + kPsiSeg - 1) / kPsiSeg;
    const size_t ncb = (nx + kPsiCols - 1) / kPsiCols;
    return (size_t)nx * ny + nseg * nx + 4 * nseg * ncb;
}

// ------------------------------------------------------------------ dispatch
#define LBM_DISPATCH(dtype, CALL)                                                      \
    switch (dtype) {                                                                   \
        case 0: { using S = double; constexpr bool SH = true; CALL; } break;          \
        case 1: { using S = float; constexpr bool SH = false; CALL; } break;          \
        case 2: { using S = float; constexpr bool SH = true; CALL; } break;           \
        case 3: { using S = __half; constexpr bool SH = true; CALL; } break;          \
        case 4: { using S = __nv_bfloat16; constexpr bool SH = true; CALL; } break;   \
        case 5: { using S = q16; constexpr bool SH = true; CALL; } break;             \
        default: return cudaErrorInvalidValue;                                         \
    }

cudaError_t launch_init(int dtype, const FieldArgs& a, void* snap, cudaStream_t st) {
    dim3 grid((unsigned)((a.pitch + 127) / 128), a.ny);
    LBM_DISPATCH(dtype, (k_init<S, SH><<<grid, 128, 0, st>>>(a, snap, nullptr, nullptr, nullptr, 0.0)));
    return cudaGetLastError();
}

cudaError_t launch_set_moments(int dtype, const FieldArgs& a, const double* rho, const double* ux,
                               const double* uy, void* snap, double neq_tau, cudaStream_t st) {
    dim3 grid((unsigned)((a.pitch + 127) / 128), a.ny);
    LBM_DISPATCH(dtype, (k_init<S, SH><<<grid, 128, 0, st>>>(a, snap, rho, ux, uy, neq_tau)));
    return cudaGetLastError();
}

cudaError_t launch_moments(int dtype, const FieldArgs& a, double* rho, double* ux, double* uy,
                           cudaStream_t st) {
    dim3 grid((unsigned)((a.nx + 127) / 128), a.ny);
    LBM_DISPATCH(dtype, (k_moments<S, SH><<<grid, 128, 0, st>>>(a, rho, ux, uy)));
    return cudaGetLastError();
}

cudaError_t launch_get_populations(int dtype, const FieldArgs& a, double* out, cudaStream_t st) {
    dim3 grid((unsigned)((a.nx + 127) / 128), a.ny, 9);
    LBM_DISPATCH(dtype, (k_get_pop<S, SH><<<grid, 128, 0, st>>>(a, out)));
    return cudaGetLastError();
}

cudaError_t launch_set_populations(int dtype, const FieldArgs& a, const double* in, cudaStream_t st) {
    dim3 grid((unsigned)((a.nx + 127) / 128), a.ny, 9);
    LBM_DISPATCH(dtype, (k_set_pop<S, SH><<<grid, 128, 0, st>>>(a, in)));
    return cudaGetLastError();
}

cudaError_t launch_mass(int dtype, const FieldArgs& a, double* partials, int max_partials,
                        DevState* state, cudaStream_t st) {
    const int g = a.ny < max_partials ? a.ny : max_partials;
    LBM_DISPATCH(dtype, (k_mass<S, SH><<<g, 256, 0, st>>>(a, partials)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_mass_finalize<<<1, 256, 0, st>>>(partials, g, (double)a.nx * (double)a.ny, state);
    return cudaGetLastError();
}

cudaError_t launch_stream_function(int dtype, const FieldArgs& a, double* psi, int i0, int i1,
                                   int j0, int j1, double* scratch, DevState* state,
                                   cudaStream_t st) {
    const int ncb = (a.nx + kPsiCols - 1) / kPsiCols;
    const int nseg = (a.ny + kPsiSeg - 1) / kPsiSeg;
    double* uscr = scratch;                            // nx*ny values of the arithmetic type
    double* segsum = scratch + (size_t)a.nx * a.ny;    // nseg * nx
    double* part = segsum + (size_t)nseg * a.nx;       // 4 per walk block
    dim3 grid(ncb, nseg);
    LBM_DISPATCH(dtype, (k_psi_seg<S, SH><<<grid, kPsiCols, 0, st>>>(a, uscr, segsum)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    LBM_DISPATCH(dtype, (k_psi_walk<typename St<S>::C><<<grid, kPsiCols, 0, st>>>(
                             a.nx, a.ny, reinterpret_cast<const typename St<S>::C*>(uscr), segsum, psi,
                             i0, i1, j0, j1, part)));
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_psi_finalize<<<1, 256, 0, st>>>(part, ncb * nseg, a.nx, state);
    return cudaGetLastError();
}

}  // namespace lbm
