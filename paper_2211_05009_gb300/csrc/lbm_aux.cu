// lbm_aux.cu -- per-run and on-demand kernels around the time step: initial state, field
// import/export, FP64 mass reduction and the FP64 stream function with vortex-centre search.
//
//   init / set_moments   Sec. 2.2 (i): f = f^eq(rho, u) (Eq. 2)
//   moments              Eq. 3 of the stored post-collision populations
//   mass                 sum_x rho(x) in FP64 (two-stage, fixed order -> deterministic)
//   stream_function      Psi with u_x = dPsi/dy, Psi(y = 0) = 0, trapezoid rule in y; the extrema
//                        and their nodes give the vortex strengths and centres of Table 1 / 2.
#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

int storage_bytes(int dtype) { return dtype == 0 ? 8 : (dtype <= 2 ? 4 : 2); }

long long row_pitch(int dtype, int nx) {
    const long long per_warp = 32ll * (16 / storage_bytes(dtype));
    return (nx + per_warp - 1) / per_warp * per_warp;
}

// Deviation equilibrium in FP64: g_j = w_j (drho + rho A_j(u)) (Eq. 2).
__device__ __forceinline__ double geq_d(int j, double drho, double rho, double ux, double uy) {
    const double cu = cx(j) * ux + cy(j) * uy;
    const double A = 3.0 * cu + 4.5 * cu * cu - 1.5 * (ux * ux + uy * uy);
    return wd(j) * (drho + rho * A);
}

template <typename S, bool SHIFTED>
__device__ __forceinline__ void store_dev(S* f, long long idx, int j, double g) {
    f[idx] = St<S>::from(typename St<S>::C(SHIFTED ? g : g + wd(j)));
}

template <typename S, bool SHIFTED>
__device__ __forceinline__ double load_dev(const S* f, long long idx, int j) {
    const double v = double(St<S>::to(f[idx]));
    return SHIFTED ? v : v - wd(j);
}

// Moments (Eq. 3) of the stored populations at linear index k, in FP64.
template <typename S, bool SHIFTED>
__device__ __forceinline__ void node_moments(const S* f, long long plane, long long k, double& drho,
                                             double& ux, double& uy) {
    double g[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) g[j] = load_dev<S, SHIFTED>(f, j * plane + k, j);
    drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
    const double rho = 1.0 + drho;
    ux = ((g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7])) / rho;
    uy = ((g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8])) / rho;
}

// ------------------------------------------------------------------ init / set_moments
template <typename S, bool SHIFTED>
__global__ void k_init(FieldArgs a, double* snap, const double* rho_in, const double* ux_in,
                       const double* uy_in) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.pitch || y >= a.ny) return;
    S* f = static_cast<S*>(a.f);
    const long long k = (long long)y * a.pitch + x;
    double drho = 0.0, ux = 0.0, uy = 0.0;
    if (x < a.nx) {
        if (rho_in) {
            const long long d = (long long)y * a.nx + x;
            drho = rho_in[d] - 1.0;
            ux = ux_in[d];
            uy = uy_in[d];
        } else if (y == a.ny - 1 && (a.corner_moving || (x > 0 && x < a.nx - 1))) {
            ux = a.U;  // Sec. 2.2 (i): only the lid moves at t = 0
        }
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) store_dev<S, SHIFTED>(f, j * a.plane + k, j, geq_d(j, drho, 1.0 + drho, ux, uy));
    if (snap) {
        snap[k] = ux;
        snap[a.plane + k] = uy;
    }
}

// ------------------------------------------------------------------ export / import
template <typename S, bool SHIFTED>
__global__ void k_moments(FieldArgs a, double* rho, double* ux, double* uy) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x >= a.nx) return;
    const S* f = static_cast<const S*>(a.f);
    double drho, u, v;
    node_moments<S, SHIFTED>(f, a.plane, (long long)y * a.pitch + x, drho, u, v);
    const long long d = (long long)y * a.nx + x;
    if (rho) rho[d] = 1.0 + drho;
    if (ux) ux[d] = u;
    if (uy) uy[d] = v;
}

template <typename S, bool SHIFTED>
__global__ void k_get_pop(FieldArgs a, double* out) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, j = blockIdx.z;
    if (x >= a.nx) return;
    const S* f = static_cast<const S*>(a.f);
    out[((long long)j * a.ny + y) * a.nx + x] = load_dev<S, SHIFTED>(f, j * a.plane + (long long)y * a.pitch + x, j) + wd(j);
}

template <typename S, bool SHIFTED>
__global__ void k_set_pop(FieldArgs a, const double* in) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y, j = blockIdx.z;
    if (x >= a.nx) return;
    S* f = static_cast<S*>(a.f);
    store_dev<S, SHIFTED>(f, j * a.plane + (long long)y * a.pitch + x, j,
                          in[((long long)j * a.ny + y) * a.nx + x] - wd(j));
}

// ------------------------------------------------------------------ mass
template <typename S, bool SHIFTED>
__global__ void __launch_bounds__(256) k_mass(FieldArgs a, double* partials) {
    __shared__ double sh[8];
    const S* f = static_cast<const S*>(a.f);
    double acc = 0.0;
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x)
        for (int x = threadIdx.x; x < a.nx; x += blockDim.x) {
            const long long k = (long long)y * a.pitch + x;
#pragma unroll
            for (int j = 0; j < 9; ++j) acc += load_dev<S, SHIFTED>(f, j * a.plane + k, j);
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
// Block (32 columns) x (32 chunks of rows).  Psi(x, y) = sum_{k<=y} u(k) - u(0)/2 - u(y)/2,
// which is the trapezoid sum of (u(k-1) + u(k))/2 for k = 1..y.
constexpr int kPsiCols = 32, kPsiChunks = 32;

struct Ext {
    double vmin, vmax;
    long long imin, imax;  // linear node index y*nx + x (ties -> smaller index)
};

__device__ __forceinline__ void ext_merge(Ext& a, const Ext& b) {
    if (b.vmin < a.vmin || (b.vmin == a.vmin && b.imin < a.imin)) { a.vmin = b.vmin; a.imin = b.imin; }
    if (b.vmax > a.vmax || (b.vmax == a.vmax && b.imax < a.imax)) { a.vmax = b.vmax; a.imax = b.imax; }
}

template <typename S, bool SHIFTED>
__device__ __forceinline__ double node_ux(const S* f, const FieldArgs& a, int x, int y) {
    double drho, u, v;
    node_moments<S, SHIFTED>(f, a.plane, (long long)y * a.pitch + x, drho, u, v);
    return u;
}

template <typename S, bool SHIFTED>
__global__ void __launch_bounds__(kPsiCols * kPsiChunks) k_psi(FieldArgs a, double* psi, int i0, int i1, int j0,
                                                              int j1, double* part) {
    __shared__ double csum[kPsiChunks][kPsiCols + 1];
    __shared__ Ext ex[kPsiChunks * kPsiCols];
    const S* f = static_cast<const S*>(a.f);
    const int tx = threadIdx.x, c = threadIdx.y;
    const int x = blockIdx.x * kPsiCols + tx;
    const int ch = (a.ny + kPsiChunks - 1) / kPsiChunks;
    const int y0 = c * ch, y1 = min(a.ny, y0 + ch);
    double s = 0.0;
    if (x < a.nx)
        for (int y = y0; y < y1; ++y) s += node_ux<S, SHIFTED>(f, a, x, y);
    csum[c][tx] = s;
    __syncthreads();
    Ext e{INFINITY, -INFINITY, -1, -1};
    if (x < a.nx) {
        double run = 0.0;
        for (int k = 0; k < c; ++k) run += csum[k][tx];
        const double u0 = node_ux<S, SHIFTED>(f, a, x, 0);
        const bool colin = x >= i0 && x < i1;
        for (int y = y0; y < y1; ++y) {
            const double u = node_ux<S, SHIFTED>(f, a, x, y);
            run += u;
            const double p = y == 0 ? 0.0 : run - 0.5 * u0 - 0.5 * u;
            if (psi) psi[(long long)y * a.nx + x] = p;
            if (colin && y >= j0 && y < j1) {
                const long long id = (long long)y * a.nx + x;
                if (p < e.vmin) { e.vmin = p; e.imin = id; }
                if (p > e.vmax) { e.vmax = p; e.imax = id; }
            }
        }
    }
    const int t = c * kPsiCols + tx;
    ex[t] = e;
    __syncthreads();
    for (int o = kPsiCols * kPsiChunks / 2; o > 0; o >>= 1) {
        if (t < o) ext_merge(ex[t], ex[t + o]);
        __syncthreads();
    }
    if (t == 0) {
        part[4ll * blockIdx.x + 0] = ex[0].vmin;
        part[4ll * blockIdx.x + 1] = (double)ex[0].imin;
        part[4ll * blockIdx.x + 2] = ex[0].vmax;
        part[4ll * blockIdx.x + 3] = (double)ex[0].imax;
    }
}

__global__ void k_psi_finalize(const double* part, int nblocks, int nx, DevState* st) {
    if (threadIdx.x != 0) return;
    Ext e{INFINITY, -INFINITY, -1, -1};
    for (int b = 0; b < nblocks; ++b) {
        Ext o{part[4ll * b], part[4ll * b + 2], (long long)part[4ll * b + 1], (long long)part[4ll * b + 3]};
        if (o.imin < 0) o.vmin = INFINITY;
        if (o.imax < 0) o.vmax = -INFINITY;
        if (o.imin >= 0 && (e.imin < 0 || o.vmin < e.vmin || (o.vmin == e.vmin && o.imin < e.imin))) { e.vmin = o.vmin; e.imin = o.imin; }
        if (o.imax >= 0 && (e.imax < 0 || o.vmax > e.vmax || (o.vmax == e.vmax && o.imax < e.imax))) { e.vmax = o.vmax; e.imax = o.imax; }
    }
    st->ext[0] = e.vmin;
    st->ext[1] = e.imin < 0 ? -1.0 : (double)(e.imin % nx);
    st->ext[2] = e.imin < 0 ? -1.0 : (double)(e.imin / nx);
    st->ext[3] = e.vmax;
    st->ext[4] = e.imax < 0 ? -1.0 : (double)(e.imax % nx);
    st->ext[5] = e.imax < 0 ? -1.0 : (double)(e.imax / nx);
}

size_t psi_scratch_doubles(int nx, int ny) {
    (void)ny;
    return 4ull * ((nx + kPsiCols - 1) / kPsiCols);
}

// ------------------------------------------------------------------ dispatch
#define LBM_DISPATCH(dtype, CALL)                                   \
    switch (dtype) {                                                \
        case 0: { using S = double; constexpr bool SH = false; CALL; } break;          \
        case 1: { using S = float; constexpr bool SH = false; CALL; } break;           \
        case 2: { using S = float; constexpr bool SH = true; CALL; } break;            \
        case 3: { using S = __half; constexpr bool SH = true; CALL; } break;           \
        case 4: { using S = __nv_bfloat16; constexpr bool SH = true; CALL; } break;    \
        default: return cudaErrorInvalidValue;                      \
    }

cudaError_t launch_init(int dtype, const FieldArgs& a, double* snap, cudaStream_t st) {
    dim3 grid((unsigned)((a.pitch + 127) / 128), a.ny);
    LBM_DISPATCH(dtype, (k_init<S, SH><<<grid, 128, 0, st>>>(a, snap, nullptr, nullptr, nullptr)));
    return cudaGetLastError();
}

cudaError_t launch_set_moments(int dtype, const FieldArgs& a, const double* rho, const double* ux,
                               const double* uy, double* snap, cudaStream_t st) {
    dim3 grid((unsigned)((a.pitch + 127) / 128), a.ny);
    LBM_DISPATCH(dtype, (k_init<S, SH><<<grid, 128, 0, st>>>(a, snap, rho, ux, uy)));
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
    const int nb = (a.nx + kPsiCols - 1) / kPsiCols;
    dim3 block(kPsiCols, kPsiChunks);
    LBM_DISPATCH(dtype, (k_psi<S, SH><<<nb, block, 0, st>>>(a, psi, i0, i1, j0, j1, scratch)));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_psi_finalize<<<1, 32, 0, st>>>(scratch, nb, a.nx, state);
    return cudaGetLastError();
}

}  // namespace lbm
