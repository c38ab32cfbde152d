// lbm_step_kernel.cuh -- the fused D2Q9 stream + collide + wall kernel (one launch per time step).
//
// Per node (Xiang & Shi, arXiv 2211.05009):
//   streaming   pull f_j(x - c_j) from the previous post-collision field        Eq. 1 (left)
//   moments     rho = sum f_j, rho u = sum c_j f_j                               Eq. 3
//   collision   f*_j = f_j + (f^eq_j - f_j)/tau                                   Eq. 1, Eq. 2
//   walls       ring nodes pull at their inner neighbour x_f instead and store
//               f^eq(rho_f, u_w) + (1 - 1/tau)(f(x_f) - f^eq(rho_f, u_f))           Sec. 2.2 (ii)
//               -- the non-equilibrium extrapolation rebuilt and collided in one go (the
//               rebuilt node has moments (rho_f, u_w), so its BGK step is this closed form).
// All arithmetic runs on deviations g_j = f_j - w_j, which keeps rounding relative to the flow
// rather than to the weights.  Every REDUCE launch (the 100th step of a checkpoint interval) also
// forms sum(rho - 1) and the two sums of Eq. 6 against the snapshot of 100 steps before, and writes
// the new snapshot: per node in the arithmetic type, per thread over its few nodes, and in FP64
// from the warp level up (FP64 throughput on this part is a small fraction of FP32's).
//
// Thread mapping: blockDim = (32, BY); each lane owns V consecutive nodes of R consecutive rows,
// a warp 32*V nodes per row.  All R rows are pulled before any is collided, so a thread has
// 9*R vector loads in flight.  The row pitch is a multiple of 32*V for every launch shape, so all
// vector accesses are in bounds; padding nodes (x >= nx) store the rest state.
#pragma once

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

static constexpr unsigned kFull = 0xffffffffu;

template <int BYTES> struct Raw;
template <> struct Raw<16> { using T = uint4; };
template <> struct Raw<8> { using T = uint2; };
template <> struct Raw<4> { using T = unsigned int; };

template <typename S, int V>
__device__ __forceinline__ void vload_n(const S* __restrict__ p, typename St<S>::C (&out)[V]) {
    using T = typename Raw<V * sizeof(S)>::T;
    union { T u; S s[V]; } b;
    b.u = __ldg(reinterpret_cast<const T*>(p));
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = St<S>::to(b.s[i]);
}

template <typename S, int V>
__device__ __forceinline__ void vstore_n(S* __restrict__ p, const typename St<S>::C (&in)[V]) {
    using T = typename Raw<V * sizeof(S)>::T;
    union { T u; S s[V]; } b;
#pragma unroll
    for (int i = 0; i < V; ++i) b.s[i] = St<S>::from(in[i]);
    *reinterpret_cast<T*>(p) = b.u;
}

// Pull one population row segment: out[i] = value at (x0 + i - DX), DX = c_x of the direction.
template <typename S, bool SHIFTED, int V, int DX>
__device__ __forceinline__ void pull_row(const S* __restrict__ p, int lane, int x0, long long pitch,
                                         typename St<S>::C wj, typename St<S>::C (&out)[V]) {
    using C = typename St<S>::C;
    C v[V];
    vload_n<S, V>(p, v);
    if constexpr (DX == 0) {
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = v[i];
    } else if constexpr (DX == 1) {
        C left = __shfl_up_sync(kFull, v[V - 1], 1);
        if (lane == 0) left = (x0 > 0) ? St<S>::to(p[-1]) : v[0];
        out[0] = left;
#pragma unroll
        for (int i = 1; i < V; ++i) out[i] = v[i - 1];
    } else {
        C right = __shfl_down_sync(kFull, v[0], 1);
        if (lane == 31) right = (x0 + V < pitch) ? St<S>::to(p[V]) : v[V - 1];
#pragma unroll
        for (int i = 0; i < V - 1; ++i) out[i] = v[i + 1];
        out[V - 1] = right;
    }
    if constexpr (!SHIFTED) {
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] -= wj;
    }
}

// Deviation equilibrium g^eq_j = w_j (drho + rho A_j), A_j = 3 c.u + 9/2 (c.u)^2 - 3/2 u.u (Eq. 2).
template <typename C>
__device__ __forceinline__ void geq9(C drho, C rho, C ux, C uy, C (&e)[9]) {
    const C usq = C(1.5) * (ux * ux + uy * uy);
    const C w0 = C(4.0 / 9.0), w1 = C(1.0 / 9.0), w5 = C(1.0 / 36.0);
    auto A = [&](C cu) { return cu * (C(3.0) + C(4.5) * cu) - usq; };
    const C up = ux + uy, um = ux - uy;
    e[0] = w0 * (drho - rho * usq);
    e[1] = w1 * (drho + rho * A(ux));
    e[2] = w1 * (drho + rho * A(uy));
    e[3] = w1 * (drho + rho * A(-ux));
    e[4] = w1 * (drho + rho * A(-uy));
    e[5] = w5 * (drho + rho * A(up));
    e[6] = w5 * (drho + rho * A(-um));
    e[7] = w5 * (drho + rho * A(-up));
    e[8] = w5 * (drho + rho * A(um));
}

template <typename C>
__device__ __forceinline__ C rcp(C v);
template <> __device__ __forceinline__ float rcp<float>(float v) { return __frcp_rn(v); }
template <> __device__ __forceinline__ double rcp<double>(double v) { return __drcp_rn(v); }

// Streamed populations of one row segment (V nodes) of row y, walls folded in: wall rows gather
// at their inner row, the left/right wall nodes take the populations of x_f = 1 / nx - 2.
template <typename S, bool SHIFTED, int V>
__device__ __forceinline__ void pull_segment(const S* __restrict__ src, int lane, int x0, int y, int nx,
                                             int ny, long long pitch, long long plane,
                                             typename St<S>::C (&f)[9][V]) {
    using C = typename St<S>::C;
    const int yc = min(max(y, 1), ny - 2);  // gather centre row
    const S* pc = src + (long long)yc * pitch + x0;
    const S* ps = pc - pitch;  // row yc - 1: source of c_y = +1
    const S* pn = pc + pitch;  // row yc + 1: source of c_y = -1
    pull_row<S, SHIFTED, V, 0>(pc + 0 * plane, lane, x0, pitch, C(4.0 / 9.0), f[0]);
    pull_row<S, SHIFTED, V, 1>(pc + 1 * plane, lane, x0, pitch, C(1.0 / 9.0), f[1]);
    pull_row<S, SHIFTED, V, 0>(ps + 2 * plane, lane, x0, pitch, C(1.0 / 9.0), f[2]);
    pull_row<S, SHIFTED, V, -1>(pc + 3 * plane, lane, x0, pitch, C(1.0 / 9.0), f[3]);
    pull_row<S, SHIFTED, V, 0>(pn + 4 * plane, lane, x0, pitch, C(1.0 / 9.0), f[4]);
    pull_row<S, SHIFTED, V, 1>(ps + 5 * plane, lane, x0, pitch, C(1.0 / 36.0), f[5]);
    pull_row<S, SHIFTED, V, -1>(ps + 6 * plane, lane, x0, pitch, C(1.0 / 36.0), f[6]);
    pull_row<S, SHIFTED, V, -1>(pn + 7 * plane, lane, x0, pitch, C(1.0 / 36.0), f[7]);
    pull_row<S, SHIFTED, V, 1>(pn + 8 * plane, lane, x0, pitch, C(1.0 / 36.0), f[8]);
    if (x0 == 0) {
#pragma unroll
        for (int j = 0; j < 9; ++j) f[j][0] = f[j][1];
    }
    const int sR = nx - 1 - x0;  // slot of the right wall node in this lane, if any
#pragma unroll
    for (int i = 1; i < V; ++i)
        if (sR == i) {
#pragma unroll
            for (int j = 0; j < 9; ++j) f[j][i] = f[j][i - 1];
        }
    if (sR == 0) {  // x_f = nx - 2 belongs to the previous lane: pull it directly
        const long long xf = nx - 2;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            const C v = St<S>::to(src[j * plane + (long long)(yc - cy(j)) * pitch + (xf - cx(j))]);
            f[j][0] = SHIFTED ? v : v - C(wd(j));
        }
    }
}

template <typename S, bool SHIFTED, bool REDUCE, int V, int R, int BY, int MINB>
__global__ void __launch_bounds__(32 * BY, MINB) k_step(const StepArgs a) {
    using C = typename St<S>::C;
    const int lane = threadIdx.x;
    const int x0 = (blockIdx.x * 32 + lane) * V;
    const int yb = (blockIdx.y * BY + threadIdx.y) * R;
    const int nx = a.nx, ny = a.ny;
    const long long pitch = a.pitch, plane = a.plane;
    const S* __restrict__ src = static_cast<const S*>(a.src);
    S* __restrict__ dst = static_cast<S*>(a.dst);
    const C omega = C(a.omega);
    const C keep = C(1.0) - omega;  // 1 - 1/tau (wall nodes)
    const C Ulid = C(a.U);

    C acc_drho = C(0), acc_num = C(0), acc_den = C(0);

    // all R rows are loaded first (rows past the top are clamped for loading and not stored)
    C f[R][9][V];
#pragma unroll
    for (int r = 0; r < R; ++r) pull_segment<S, SHIFTED, V>(src, lane, x0, min(yb + r, ny - 1), nx, ny, pitch, plane, f[r]);

#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int y = yb + r;
        if (y >= ny) break;  // uniform across the warp
        // observing points on this row segment (Sec. 3.3)
        unsigned pmask = 0;
        for (int q = 0; q < a.probes.n; ++q)
            if (a.probes.py[q] == y && a.probes.px[q] >= x0 && a.probes.px[q] < x0 + V) pmask |= 1u << q;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const int x = x0 + i;
            C g[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) g[j] = f[r][j][i];
            const C drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
            const C rho = C(1.0) + drho;
            const C jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
            const C jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
            const C inv = rcp<C>(rho);
            const C ux = jx * inv, uy = jy * inv;
            C e[9];
            geq9<C>(drho, rho, ux, uy, e);
            const bool wall = (y == 0) | (y == ny - 1) | (x == 0) | (x >= nx - 1);
            C uox = ux, uoy = uy;
            if (wall) {
                const bool lid = (y == ny - 1) && (a.corner_moving || (x > 0 && x < nx - 1));
                uox = lid ? Ulid : C(0.0);
                uoy = C(0.0);
                C ew[9];
                geq9<C>(drho, rho, uox, uoy, ew);
#pragma unroll
                for (int j = 0; j < 9; ++j) f[r][j][i] = ew[j] + keep * (g[j] - e[j]);
            } else {
                // BGK as an increment d_j = (f^eq_j - f_j)/tau added to the pulled value.  The
                // increment must carry no momentum; in FP32 the rounding of f^eq breaks that by a
                // few ulps in the same direction every step, so the x and y momentum of d is
                // removed from the (1,3) and (2,4) pairs (a rounding-level change).
                C d[9];
#pragma unroll
                for (int j = 0; j < 9; ++j) d[j] = omega * (e[j] - g[j]);
                if constexpr (sizeof(C) == 4) {
                    const C mx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
                    const C my = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
                    d[1] -= C(0.5) * mx;
                    d[3] += C(0.5) * mx;
                    d[2] -= C(0.5) * my;
                    d[4] += C(0.5) * my;
                }
#pragma unroll
                for (int j = 0; j < 9; ++j) f[r][j][i] = g[j] + d[j];
            }
            if (x >= nx) {
#pragma unroll
                for (int j = 0; j < 9; ++j) f[r][j][i] = C(0.0);
            }
            if constexpr (REDUCE) {
                if (x < nx) {
                    C* snap = static_cast<C*>(a.snap);
                    const long long k = (long long)y * pitch + x;
                    const C sx = snap[k], sy = snap[plane + k];
                    const C dx = uox - sx, dy = uoy - sy;  // exact when close (Sterbenz)
                    acc_drho += drho;
                    acc_num += dx * dx + dy * dy;
                    acc_den += sx * sx + sy * sy;
                    snap[k] = uox;
                    snap[plane + k] = uoy;
                }
            }
            if (pmask) {
                for (int q = 0; q < a.probes.n; ++q) {
                    if (((pmask >> q) & 1u) && a.probes.px[q] == x) {
                        const long long t = a.state->base + a.s + 1;
                        const int ev = a.probes.every[q];
                        if (t % ev == 0) {
                            long long k = t / ev - a.probes.start[q] / ev - 1;
                            if (k >= 0) {
                                k %= a.probes.cap[q];
                                a.probes.series[q][2 * k] = double(uox);
                                a.probes.series[q][2 * k + 1] = double(uoy);
                            }
                        }
                    }
                }
            }
        }

        S* pd = dst + (long long)y * pitch + x0;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            if constexpr (!SHIFTED) {
#pragma unroll
                for (int i = 0; i < V; ++i) f[r][j][i] += C(wd(j));
            }
            vstore_n<S, V>(pd + j * plane, f[r][j]);
        }
    }

    if constexpr (REDUCE) {
        __shared__ double red[3][BY];
        const double s0 = warp_sum(double(acc_drho));
        const double s1 = warp_sum(double(acc_num));
        const double s2 = warp_sum(double(acc_den));
        if (lane == 0) {
            red[0][threadIdx.y] = s0;
            red[1][threadIdx.y] = s1;
            red[2][threadIdx.y] = s2;
        }
        __syncthreads();
        if (threadIdx.y == 0 && lane < 3) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < BY; ++w) s += red[lane][w];
            a.partials[3ll * (blockIdx.y * gridDim.x + blockIdx.x) + lane] = s;
        }
    }
}

// Launch shape (nodes per lane V, rows per thread R, warps per block BY, min blocks per SM).
// Every shape computes bitwise-identical populations; only speed differs.
template <typename S, bool SHIFTED, int V, int R, int BY, int MINB>
static cudaError_t launch_step_shape(const StepArgs& a, bool reduce, cudaStream_t st) {
    dim3 block(32, BY);
    dim3 grid((unsigned)(a.pitch / (32 * V)), (unsigned)((a.ny + BY * R - 1) / (BY * R)));
    if (reduce)
        k_step<S, SHIFTED, true, V, R, BY, MINB><<<grid, block, 0, st>>>(a);
    else
        k_step<S, SHIFTED, false, V, R, BY, MINB><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

// The shape tables; step_shape() in lbm_step.cu mirrors them.
template <typename S, bool SHIFTED>
static cudaError_t launch_step_cfg(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    if constexpr (sizeof(S) == 8) {
        switch (cfg) {
            case 0: return launch_step_shape<S, SHIFTED, 2, 1, 4, 1>(a, reduce, st);
            case 1: return launch_step_shape<S, SHIFTED, 2, 2, 2, 1>(a, reduce, st);
            case 2: return launch_step_shape<S, SHIFTED, 2, 1, 8, 1>(a, reduce, st);
            case 3: return launch_step_shape<S, SHIFTED, 2, 2, 4, 1>(a, reduce, st);
            case 4: return launch_step_shape<S, SHIFTED, 2, 1, 2, 1>(a, reduce, st);
            case 5: return launch_step_shape<S, SHIFTED, 2, 1, 4, 4>(a, reduce, st);
            default: return cudaErrorInvalidValue;
        }
    } else if constexpr (sizeof(S) == 4) {
        switch (cfg) {
            case 0: return launch_step_shape<S, SHIFTED, 4, 2, 2, 1>(a, reduce, st);
            case 1: return launch_step_shape<S, SHIFTED, 4, 1, 4, 1>(a, reduce, st);
            case 2: return launch_step_shape<S, SHIFTED, 4, 2, 4, 1>(a, reduce, st);
            case 3: return launch_step_shape<S, SHIFTED, 4, 1, 8, 1>(a, reduce, st);
            case 4: return launch_step_shape<S, SHIFTED, 2, 2, 4, 1>(a, reduce, st);
            case 5: return launch_step_shape<S, SHIFTED, 4, 2, 1, 1>(a, reduce, st);
            default: return cudaErrorInvalidValue;
        }
    } else {
        switch (cfg) {
            case 0: return launch_step_shape<S, SHIFTED, 4, 2, 2, 1>(a, reduce, st);
            case 1: return launch_step_shape<S, SHIFTED, 8, 1, 4, 1>(a, reduce, st);
            case 2: return launch_step_shape<S, SHIFTED, 4, 2, 4, 1>(a, reduce, st);
            case 3: return launch_step_shape<S, SHIFTED, 4, 1, 4, 1>(a, reduce, st);
            case 4: return launch_step_shape<S, SHIFTED, 2, 2, 4, 1>(a, reduce, st);
            case 5: return launch_step_shape<S, SHIFTED, 8, 2, 2, 1>(a, reduce, st);
            default: return cudaErrorInvalidValue;
        }
    }
}

}  // namespace lbm
