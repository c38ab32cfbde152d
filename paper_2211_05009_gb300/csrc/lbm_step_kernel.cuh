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
// Thread mapping: blockDim = (32, BY); each lane owns V consecutive nodes (V = 2: a 16-byte vector
// for FP64, 8 bytes for FP32; V = 4: 8 bytes for 16-bit storage) of R consecutive rows, a warp
// 32*V nodes per row.  The row pitch is a multiple of 32*V for every launch shape, so all vector
// accesses are in bounds; padding nodes (x >= nx) store the rest state.
#pragma once

#include <type_traits>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

static constexpr unsigned kFull = 0xffffffffu;

template <int BYTES> struct Raw;
template <> struct Raw<16> { using T = uint4; };
template <> struct Raw<8> { using T = uint2; };
template <> struct Raw<4> { using T = unsigned int; };

// Vector load.  HINT 0: read-only path; 1: read-only with an L2 256-byte prefetch, no L1
// allocation; 2: coherent L2 load (ld.global.cg) for kernels that also write the array they read
// from across a grid barrier (the read-only path may serve stale lines there); 3: weak load cached
// in L1 (ld.global.ca) for the same kernels -- coherent because the loads follow the barrier's
// acquire, which discards the SM's stale L1 lines; spelled out in asm so that the compiler cannot
// turn it into a read-only-path load.
template <typename T, int HINT>
__device__ __forceinline__ T ldg_vec(const T* p) {
    if constexpr (HINT == 0) {
        return __ldg(p);
    } else if constexpr (HINT == 2) {
        return __ldcg(p);
    } else if constexpr (HINT == 3) {
        if constexpr (sizeof(T) == 16) {
            uint4 r;
            asm volatile("ld.global.ca.v4.u32 {%0, %1, %2, %3}, [%4];"
                         : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
            return r;
        } else if constexpr (sizeof(T) == 8) {
            uint2 r;
            asm volatile("ld.global.ca.v2.u32 {%0, %1}, [%2];" : "=r"(r.x), "=r"(r.y) : "l"(p));
            return r;
        } else {
            unsigned int r;
            asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(r) : "l"(p));
            return r;
        }
    } else if constexpr (sizeof(T) == 16) {
        uint4 r;
        asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0, %1, %2, %3}, [%4];"
                     : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w) : "l"(p));
        return r;
    } else if constexpr (sizeof(T) == 8) {
        uint2 r;
        asm volatile("ld.global.nc.L1::no_allocate.L2::256B.v2.u32 {%0, %1}, [%2];"
                     : "=r"(r.x), "=r"(r.y) : "l"(p));
        return r;
    } else {
        unsigned int r;
        asm volatile("ld.global.nc.L1::no_allocate.L2::256B.u32 %0, [%1];" : "=r"(r) : "l"(p));
        return r;
    }
}

template <typename S, int V, int HINT = 0>
__device__ __forceinline__ void vload_n(const S* __restrict__ p, typename St<S>::C (&out)[V]) {
    using T = typename Raw<V * sizeof(S)>::T;
    union { T u; S s[V]; } b;
    b.u = ldg_vec<T, HINT>(reinterpret_cast<const T*>(p));
#pragma unroll
    for (int i = 0; i < V; ++i) out[i] = St<S>::to(b.s[i]);
}

// V values of a plain arithmetic-type array (the Eq. 6 snapshot), in 16-byte pieces.
template <typename C, int V, bool COHERENT = false>
__device__ __forceinline__ void cload(const C* p, C (&out)[V]) {
    constexpr int B = V * sizeof(C) < 16 ? V * sizeof(C) : 16;
    constexpr int PER = B / sizeof(C);
    using T = typename Raw<B>::T;
#pragma unroll
    for (int k = 0; k < V; k += PER) {
        union { T u; C c[PER]; } b;
        if constexpr (COHERENT)
            b.u = __ldcg(reinterpret_cast<const T*>(p + k));
        else
            b.u = *reinterpret_cast<const T*>(p + k);
#pragma unroll
        for (int i = 0; i < PER; ++i) out[k + i] = b.c[i];
    }
}
template <typename C, int V>
__device__ __forceinline__ void cstore(C* p, const C (&in)[V]) {
    constexpr int B = V * sizeof(C) < 16 ? V * sizeof(C) : 16;
    constexpr int PER = B / sizeof(C);
    using T = typename Raw<B>::T;
#pragma unroll
    for (int k = 0; k < V; k += PER) {
        union { T u; C c[PER]; } b;
#pragma unroll
        for (int i = 0; i < PER; ++i) b.c[i] = in[k + i];
        *reinterpret_cast<T*>(p + k) = b.u;
    }
}

template <typename S, int V>
__device__ __forceinline__ void vstore_n(S* __restrict__ p, const typename St<S>::C (&in)[V]) {
    using T = typename Raw<V * sizeof(S)>::T;
    union { T u; S s[V]; } b;
#pragma unroll
    for (int i = 0; i < V; ++i) b.s[i] = St<S>::from(in[i]);
    *reinterpret_cast<T*>(p) = b.u;
}

// Scalar load of one storage element, coherent at L2 when HINT == 2, L1-cached weak when 3.
template <typename S, int HINT>
__device__ __forceinline__ typename St<S>::C lds(const S* p) {
    if constexpr (HINT == 3) {
        if constexpr (sizeof(S) == 8) {
            unsigned long long r;
            asm volatile("ld.global.ca.u64 %0, [%1];" : "=l"(r) : "l"(p));
            union { unsigned long long u; S s; } b;
            b.u = r;
            return St<S>::to(b.s);
        } else if constexpr (sizeof(S) == 4) {
            unsigned int r;
            asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(r) : "l"(p));
            union { unsigned int u; S s; } b;
            b.u = r;
            return St<S>::to(b.s);
        } else {
            unsigned short r;
            asm volatile("ld.global.ca.u16 %0, [%1];" : "=h"(r) : "l"(p));
            union { unsigned short u; S s; } b;
            b.u = r;
            return St<S>::to(b.s);
        }
    } else if constexpr (HINT == 2) {
        if constexpr (sizeof(S) == 8) return St<S>::to(__ldcg(reinterpret_cast<const double*>(p)));
        else if constexpr (sizeof(S) == 4) return St<S>::to(__ldcg(reinterpret_cast<const float*>(p)));
        else {
            union { unsigned short u; S s; } b;
            b.u = __ldcg(reinterpret_cast<const unsigned short*>(p));
            return St<S>::to(b.s);
        }
    } else {
        return St<S>::to(*p);
    }
}

// One raw 16-bit element with the load path of HINT (see ldg_vec / lds).
template <int HINT>
__device__ __forceinline__ unsigned raw16(const void* p) {
    if constexpr (HINT == 3) {
        unsigned short r;
        asm volatile("ld.global.ca.u16 %0, [%1];" : "=h"(r) : "l"(p));
        return r;
    } else if constexpr (HINT == 2) {
        return __ldcg(static_cast<const unsigned short*>(p));
    } else {
        return *static_cast<const unsigned short*>(p);
    }
}

// One population value in the arithmetic type; qd = the LBM_Q16S decode scale of its direction.
template <typename S, int HINT>
__device__ __forceinline__ typename St<S>::C ld1(const S* p, float qd) {
    if constexpr (kIsQ16<S>) return q16_decode(raw16<HINT>(p), qd);
    else return lds<S, HINT>(p);
}

// V values of one direction: load (decoding LBM_Q16S codes with qd) / store (encoding with qe).
template <typename S, int V, int HINT>
__device__ __forceinline__ void vload_g(const S* __restrict__ p, float qd, typename St<S>::C (&out)[V]) {
    if constexpr (kIsQ16<S>) {
        using T = typename Raw<V * 2>::T;
        union { T u; unsigned short c[V]; } b;
        b.u = ldg_vec<T, HINT>(reinterpret_cast<const T*>(p));
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = q16_decode(b.c[i], qd);
    } else {
        vload_n<S, V, HINT>(p, out);
    }
}
template <typename S, int V>
__device__ __forceinline__ void vstore_g(S* __restrict__ p, float qe, const typename St<S>::C (&in)[V], bool& sat) {
    if constexpr (kIsQ16<S>) {
        using T = typename Raw<V * 2>::T;
        union { T u; unsigned short c[V]; } b;
#pragma unroll
        for (int i = 0; i < V; ++i) b.c[i] = (unsigned short)q16_encode(in[i], qe, sat);
        *reinterpret_cast<T*>(p) = b.u;
    } else {
        vstore_n<S, V>(p, in);
    }
}

// Pull one population row segment: out[i] = value at (x0 + i - DX), DX = c_x of the direction.
template <typename S, bool SHIFTED, int V, int DX, int HINT>
__device__ __forceinline__ void pull_row(const S* __restrict__ p, int lane, int x0, long long pitch,
                                         typename St<S>::C wj, float qd, typename St<S>::C (&out)[V]) {
    using C = typename St<S>::C;
    C v[V];
    vload_g<S, V, HINT>(p, qd, v);
    if constexpr (DX == 0) {
#pragma unroll
        for (int i = 0; i < V; ++i) out[i] = v[i];
    } else if constexpr (DX == 1) {
        C left = __shfl_up_sync(kFull, v[V - 1], 1);
        if (lane == 0) left = (x0 > 0) ? ld1<S, HINT>(p - 1, qd) : v[0];
        out[0] = left;
#pragma unroll
        for (int i = 1; i < V; ++i) out[i] = v[i - 1];
    } else {
        C right = __shfl_down_sync(kFull, v[0], 1);
        if (lane == 31) right = (x0 + V < pitch) ? ld1<S, HINT>(p + V, qd) : v[V - 1];
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

// BGK collision of a fluid node, f*_j = g_j + omega (g^eq_j - g_j) with g^eq_j = w_j (drho + rho A_j)
// (Eq. 1, Eq. 2), written per opposite pair (j, jbar): A = c2 +- 3 c.u with c2 = 9/2 (c.u)^2 - usq,
// so a pair shares c2, drho + rho c2 and 3 rho c.u.  About 50 operations per node instead of the
// 65 of forming all nine g^eq and then relaxing towards them.  ow = omega w for the three weights.
template <typename C>
__device__ __forceinline__ void collide_pairs(C drho, C rho, C ux, C uy, C omega, C ow0, C ow1, C ow5,
                                              const C (&g)[9], C (&out)[9]) {
    const C usq = C(1.5) * (ux * ux + uy * uy);
    const C r3 = C(3.0) * rho;
    out[0] = fma(ow0, fma(-rho, usq, drho), fma(-omega, g[0], g[0]));
    auto pair = [&](int a, int b, C cu, C ow) {
        const C c2 = fma(C(4.5) * cu, cu, -usq);
        const C base = fma(rho, c2, drho);
        const C sft = r3 * cu;
        out[a] = fma(ow, base + sft, fma(-omega, g[a], g[a]));
        out[b] = fma(ow, base - sft, fma(-omega, g[b], g[b]));
    };
    pair(1, 3, ux, ow1);
    pair(2, 4, uy, ow1);
    pair(5, 7, ux + uy, ow5);
    pair(8, 6, ux - uy, ow5);
}

template <typename C>
__device__ __forceinline__ C rcp(C v);
// FP32: hardware reciprocal estimate refined by one Newton-Raphson step r + r(1 - v r) (error
// below one ulp for the densities rho ~ 1 met here; no subnormals).  The IEEE-rounded reciprocal
// costs several times the instructions in a kernel that is partly issue-bound.
template <> __device__ __forceinline__ float rcp<float>(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    const float e = fmaf(-v, r, 1.0f);
    return fmaf(r, e, r);
}
template <> __device__ __forceinline__ double rcp<double>(double v) { return __drcp_rn(v); }

// Streamed populations of one row segment (V nodes) of row y, walls folded in: wall rows gather
// at their inner row, the left/right wall nodes take the populations of x_f = 1 / nx - 2.
template <typename S, bool SHIFTED, int V, int HINT>
__device__ __forceinline__ void pull_segment(const S* __restrict__ src, int lane, int x0, int y, int nx,
                                             int ny, long long pitch, long long plane, const QCodec& q,
                                             typename St<S>::C (&f)[9][V]) {
    using C = typename St<S>::C;
    const int yc = min(max(y, 1), ny - 2);  // gather centre row
    const S* pc = src + (long long)yc * pitch + x0;
    const S* ps = pc - pitch;  // row yc - 1: source of c_y = +1
    const S* pn = pc + pitch;  // row yc + 1: source of c_y = -1
    pull_row<S, SHIFTED, V, 0, HINT>(pc + 0 * plane, lane, x0, pitch, C(4.0 / 9.0), q.dec[0], f[0]);
    pull_row<S, SHIFTED, V, 1, HINT>(pc + 1 * plane, lane, x0, pitch, C(1.0 / 9.0), q.dec[1], f[1]);
    pull_row<S, SHIFTED, V, 0, HINT>(ps + 2 * plane, lane, x0, pitch, C(1.0 / 9.0), q.dec[2], f[2]);
    pull_row<S, SHIFTED, V, -1, HINT>(pc + 3 * plane, lane, x0, pitch, C(1.0 / 9.0), q.dec[3], f[3]);
    pull_row<S, SHIFTED, V, 0, HINT>(pn + 4 * plane, lane, x0, pitch, C(1.0 / 9.0), q.dec[4], f[4]);
    pull_row<S, SHIFTED, V, 1, HINT>(ps + 5 * plane, lane, x0, pitch, C(1.0 / 36.0), q.dec[5], f[5]);
    pull_row<S, SHIFTED, V, -1, HINT>(ps + 6 * plane, lane, x0, pitch, C(1.0 / 36.0), q.dec[6], f[6]);
    pull_row<S, SHIFTED, V, -1, HINT>(pn + 7 * plane, lane, x0, pitch, C(1.0 / 36.0), q.dec[7], f[7]);
    pull_row<S, SHIFTED, V, 1, HINT>(pn + 8 * plane, lane, x0, pitch, C(1.0 / 36.0), q.dec[8], f[8]);
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
            const C v = ld1<S, HINT>(src + j * plane + (long long)(yc - cy(j)) * pitch + (xf - cx(j)), q.dec[j]);
            f[j][0] = SHIFTED ? v : v - C(wd(j));
        }
    }
}

// Observing points as the row step sees them: the up-to-four probes of a single cavity
// (kernel parameter space) or the one probe of a batched cavity (registers).
struct ProbeList {
    const ProbeSet& p;
    __device__ int n() const { return p.n; }
    __device__ int px(int q) const { return p.px[q]; }
    __device__ int py(int q) const { return p.py[q]; }
    __device__ int every(int q) const { return p.every[q]; }
    __device__ long long start(int q) const { return p.start[q]; }
    __device__ long long cap(int q) const { return p.cap[q]; }
    __device__ double* series(int q) const { return p.series[q]; }
};
struct ProbeOne {
    int n_, px_, py_, every_;
    long long start_, cap_;
    double* series_;
    __device__ int n() const { return n_; }
    __device__ int px(int) const { return px_; }
    __device__ int py(int) const { return py_; }
    __device__ int every(int) const { return every_; }
    __device__ long long start(int) const { return start_; }
    __device__ long long cap(int) const { return cap_; }
    __device__ double* series(int) const { return series_; }
};

// Geometry and parameters of one cavity as the row step sees them.
template <typename C>
struct CavityView {
    int nx, ny;
    long long pitch, plane;
    C omega, Ulid;
    int corner_moving;
    QCodec q;        // LBM_Q16S only
    C sref, sref_w;  // LBM_Q16S only: rho_ref the populations are read against / stored against
};

// One time step for the V nodes of lane `lane` in row y (x0 = first node): pull, moments,
// collision or wall closure, optional Eq. 6 accumulation and probe sampling, store.
// step_time() = global index of the step being produced (called only when a probe sits in this
// segment).
// EDGE_ALWAYS: run every warp through the node code with the wall tests instead of giving
// all-interior warps their own copy (the batch kernel's choice for 16-bit storage, below).
template <typename S, bool SHIFTED, bool REDUCE, int V, int HINT, bool EDGE_ALWAYS, typename Probes, typename TimeFn>
__device__ __forceinline__ void step_row(const S* __restrict__ src, S* __restrict__ dst,
                                         const CavityView<typename St<S>::C>& cv, int lane, int x0,
                                         int y, typename St<S>::C* snap, const Probes& probes,
                                         TimeFn step_time,
                                         typename St<S>::C& acc_drho, typename St<S>::C& acc_num,
                                         typename St<S>::C& acc_den) {
    using C = typename St<S>::C;
    const int nx = cv.nx, ny = cv.ny;
    const long long pitch = cv.pitch, plane = cv.plane;
    const C omega = cv.omega;
    const C keep = C(1.0) - omega;  // 1 - 1/tau (wall nodes)
    const C ow0 = omega * C(4.0 / 9.0), ow1 = omega * C(1.0 / 9.0), ow5 = omega * C(1.0 / 36.0);
    C f[9][V];
    pull_segment<S, SHIFTED, V, HINT>(src, lane, x0, y, nx, ny, pitch, plane, cv.q, f);
    // LBM_Q16S works on h = g - w rho_ref: BGK and the wall closure keep their form in h with
    // rho = 1 + rho_ref + sum h (sum w = 1, sum c w = 0); other storage types have rho_ref = 0
    const C one_ref = kIsQ16<S> ? C(1.0) + cv.sref : C(1.0);
    C sx[V], sy[V];
    if constexpr (REDUCE) {
        cload<C, V, HINT == 2>(snap + (long long)y * pitch + x0, sx);
        cload<C, V, HINT == 2>(snap + plane + (long long)y * pitch + x0, sy);
    }
    // observing points on this row segment (Sec. 3.3)
    unsigned pmask = 0;
    for (int q = 0; q < probes.n(); ++q)
        if (probes.py(q) == y && probes.px(q) >= x0 && probes.px(q) < x0 + V) pmask |= 1u << q;
    // Per node.  EDGE = false: every segment of the warp is interior (no wall, lid or padding
    // node), the case of all but the first and last warps of a row, so the wall tests compile
    // away; the arithmetic is the same either way.  The choice is made per warp (a per-lane choice
    // would run both copies of the node code in a warp that holds a wall lane).  With EDGE_ALWAYS
    // there is one copy: the batch kernel's 16-bit instantiations measured faster that way (half
    // the warps of a 500-wide cavity hold a wall lane; 45-cavity batch, f16s 131.4 -> 135.3 GLUPS),
    // while the single-cavity 16-bit kernel gains from the split (4096^2 f16s 171.4 -> 177.6).
    auto node = [&](auto edge_c, int i) {
        constexpr bool EDGE = decltype(edge_c)::value;
        const int x = x0 + i;
        C g[9];
#pragma unroll
        for (int j = 0; j < 9; ++j) g[j] = f[j][i];
        const C drho = ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7])) + g[8];
        const C rho = one_ref + drho;
        const C jx = (g[1] - g[3]) + (g[5] - g[6]) + (g[8] - g[7]);
        const C jy = (g[2] - g[4]) + (g[5] + g[6]) - (g[7] + g[8]);
        const C inv = rcp<C>(rho);
        const C ux = jx * inv, uy = jy * inv;
        const bool wall = EDGE && ((y == 0) | (y == ny - 1) | (x == 0) | (x >= nx - 1));
        C uox = ux, uoy = uy;
        if (wall) {
            const bool lid = (y == ny - 1) && (cv.corner_moving || (x > 0 && x < nx - 1));
            uox = lid ? cv.Ulid : C(0.0);
            uoy = C(0.0);
            C e[9], ew[9];
            geq9<C>(drho, rho, ux, uy, e);
            geq9<C>(drho, rho, uox, uoy, ew);
#pragma unroll
            for (int j = 0; j < 9; ++j) f[j][i] = ew[j] + keep * (g[j] - e[j]);
        } else if constexpr (sizeof(C) == 4 && (sizeof(S) == 4 || kIsQ16<S>)) {
            // FP32 and LBM_Q16S storage: BGK as an increment d_j = (f^eq_j - f_j)/tau added to
            // the pulled value.  The increment must carry no momentum; in FP32 the rounding of
            // f^eq breaks that by a few ulps in the same direction every step, so the x and y
            // momentum of d is removed from the (1,3) and (2,4) pairs (a rounding-level change).
            // LBM_Q16S rounds its stores to nearest, which passes such a bias on unchanged on
            // average, so it needs the correction as much as FP32 storage does.
            C e[9];
            geq9<C>(drho, rho, ux, uy, e);
            C d[9];
#pragma unroll
            for (int j = 0; j < 9; ++j) d[j] = omega * (e[j] - g[j]);
            const C mx = (d[1] - d[3]) + (d[5] - d[6]) + (d[8] - d[7]);
            const C my = (d[2] - d[4]) + (d[5] + d[6]) - (d[7] + d[8]);
            d[1] -= C(0.5) * mx;
            d[3] += C(0.5) * mx;
            d[2] -= C(0.5) * my;
            d[4] += C(0.5) * my;
#pragma unroll
            for (int j = 0; j < 9; ++j) f[j][i] = g[j] + d[j];
        } else {
            // FP64 storage (bound by the FP64 pipe) and binary16 / bfloat16 storage (bound by
            // instruction issue; their stored rounding swamps an FP32 bias): the pairwise form
            // with fewer operations.
            C out[9];
            collide_pairs<C>(drho, rho, ux, uy, omega, ow0, ow1, ow5, g, out);
#pragma unroll
            for (int j = 0; j < 9; ++j) f[j][i] = out[j];
        }
        if (EDGE && x >= nx) {
#pragma unroll
            for (int j = 0; j < 9; ++j) f[j][i] = C(0.0);
        }
        if constexpr (REDUCE) {
            if (!EDGE || x < nx) {
                const C dx = uox - sx[i], dy = uoy - sy[i];  // exact when close (Sterbenz)
                acc_drho += kIsQ16<S> ? drho + cv.sref : drho;
                acc_num += dx * dx + dy * dy;
                acc_den += sx[i] * sx[i] + sy[i] * sy[i];
            }
            sx[i] = (!EDGE || x < nx) ? uox : C(0);
            sy[i] = (!EDGE || x < nx) ? uoy : C(0);
        }
        if (pmask) {
            for (int q = 0; q < probes.n(); ++q) {
                if (((pmask >> q) & 1u) && probes.px(q) == x) {
                    const long long t = step_time();
                    const int ev = probes.every(q);
                    if (t % ev == 0) {
                        long long k = t / ev - probes.start(q) / ev - 1;
                        if (k >= 0) {
                            k %= probes.cap(q);
                            probes.series(q)[2 * k] = double(uox);
                            probes.series(q)[2 * k + 1] = double(uoy);
                        }
                    }
                }
            }
        }
    };
    if (EDGE_ALWAYS || __any_sync(kFull, (y == 0) | (y == ny - 1) | (x0 == 0) | (x0 + V >= nx))) {
#pragma unroll
        for (int i = 0; i < V; ++i) node(std::true_type{}, i);
    } else {
#pragma unroll
        for (int i = 0; i < V; ++i) node(std::false_type{}, i);
    }

    S* pd = dst + (long long)y * pitch + x0;
    bool sat = false;
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        if constexpr (!SHIFTED) {
#pragma unroll
            for (int i = 0; i < V; ++i) f[j][i] += C(wd(j));
        }
        if constexpr (kIsQ16<S> && REDUCE) {  // re-reference to the next rho_ref
            const C shift = C(wd(j)) * (cv.sref - cv.sref_w);
#pragma unroll
            for (int i = 0; i < V; ++i)
                if (x0 + i < nx) f[j][i] += shift;
        }
        vstore_g<S, V>(pd + j * plane, cv.q.enc[j], f[j], sat);
    }
    if constexpr (kIsQ16<S> && REDUCE) {
        if (sat) acc_num += C(NAN);  // a saturated code: the checkpoint reports non-finite
    }
    if constexpr (REDUCE) {
        cstore<C, V>(snap + (long long)y * pitch + x0, sx);
        cstore<C, V>(snap + plane + (long long)y * pitch + x0, sy);
    }
}

// Sum of three per-thread values over the block's warps into partials[3*block .. 3*block+2].
template <int BY, typename C>
__device__ __forceinline__ void block_partials(C a0, C a1, C a2, double* partials, long long block) {
    __shared__ double red[3][BY];
    const double s0 = warp_sum(double(a0));
    const double s1 = warp_sum(double(a1));
    const double s2 = warp_sum(double(a2));
    if (threadIdx.x == 0) {
        red[0][threadIdx.y] = s0;
        red[1][threadIdx.y] = s1;
        red[2][threadIdx.y] = s2;
    }
    __syncthreads();
    if (threadIdx.y == 0 && threadIdx.x < 3) {
        double s = 0.0;
#pragma unroll
        for (int w = 0; w < BY; ++w) s += red[threadIdx.x][w];
        partials[3 * block + threadIdx.x] = s;
    }
}

// Resident blocks per SM the register budget is sized for.  binary16 / bfloat16 storage: 32 warps
// per SM (64 registers, a few spilled to L1).  Left to itself the compiler takes 80 and leaves 24
// warps, and these kernels wait on memory latency: f16s 163 -> 170 GLUPS at 4096^2 (bf16s 161 ->
// 168).  0 (no bound) for the rest -- a bound of 1 is not the same as none, it lets the compiler
// take more registers; LBM_Q16S, bound by its integer code conversions, lost 4 % at 2048^2 under
// the same cap.
template <typename S, int BY>
inline constexpr int kStepMinBlocks = (sizeof(S) == 2 && !kIsQ16<S>) ? 32 / BY : 0;

template <typename S, bool SHIFTED, bool REDUCE, int V, int R, int BY, int HINT>
__global__ void __launch_bounds__(32 * BY, (kStepMinBlocks<S, BY>)) k_step(const StepArgs a) {
    using C = typename St<S>::C;
    const int lane = threadIdx.x;
    const int x0 = (blockIdx.x * 32 + lane) * V;
    const int yb = (blockIdx.y * BY + threadIdx.y) * R;
    CavityView<C> cv;
    cv.nx = a.nx;
    cv.ny = a.ny;
    cv.pitch = a.pitch;
    cv.plane = a.plane;
    cv.omega = sizeof(C) == 4 ? C(a.omega_f) : C(a.omega);
    cv.Ulid = sizeof(C) == 4 ? C(a.U_f) : C(a.U);
    cv.corner_moving = a.corner_moving;
    cv.sref = cv.sref_w = C(0);
    if constexpr (kIsQ16<S>) {
        cv.q = a.q;
        cv.sref = C(__ldcg(&a.state->rho_ref[0]));
        cv.sref_w = REDUCE ? C(__ldcg(&a.state->rho_ref[1])) : cv.sref;
    }
    const S* __restrict__ src = static_cast<const S*>(a.src);
    S* __restrict__ dst = static_cast<S*>(a.dst);
    C acc_drho = C(0), acc_num = C(0), acc_den = C(0);
#pragma unroll 1
    for (int r = 0; r < R; ++r) {
        const int y = yb + r;
        if (y >= a.ny) break;  // uniform across the warp
        step_row<S, SHIFTED, REDUCE, V, HINT, kIsQ16<S>>(
            src, dst, cv, lane, x0, y, static_cast<C*>(a.snap), ProbeList{a.probes},
            [&]() { return a.state->base + a.s + 1; }, acc_drho, acc_num, acc_den);
    }
    if constexpr (REDUCE) block_partials<BY>(acc_drho, acc_num, acc_den, a.partials, (long long)blockIdx.y * gridDim.x + blockIdx.x);
}

// Launch shape (nodes per lane V, rows per thread R, warps per block BY, load hint).  Every shape
// computes bitwise-identical populations; only speed differs.
template <typename S, bool SHIFTED, int V, int R, int BY, int HINT>
static cudaError_t launch_step_shape(const StepArgs& a, bool reduce, cudaStream_t st) {
    dim3 block(32, BY);
    dim3 grid((unsigned)(a.pitch / (32 * V)), (unsigned)((a.ny + BY * R - 1) / (BY * R)));
    if (reduce)
        k_step<S, SHIFTED, true, V, R, BY, HINT><<<grid, block, 0, st>>>(a);
    else
        k_step<S, SHIFTED, false, V, R, BY, HINT><<<grid, block, 0, st>>>(a);
    return cudaGetLastError();
}

// The shape tables; kShapes* in lbm_step.cu mirror them.
template <typename S, bool SHIFTED>
static cudaError_t launch_step_cfg(int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    // nodes per lane: 2 for FP64 and FP32 storage (16- and 8-byte vectors; for FP32 the smaller
    // register footprint buys more resident warps, measured faster than 4), 4 for 16-bit storage
    constexpr int V = sizeof(S) == 2 ? 4 : 2;
    switch (cfg) {
        case 0: return launch_step_shape<S, SHIFTED, V, 2, 2, 0>(a, reduce, st);
        case 1: return launch_step_shape<S, SHIFTED, V, 1, 4, 0>(a, reduce, st);
        case 2: return launch_step_shape<S, SHIFTED, V, 2, 2, 1>(a, reduce, st);
        case 3: return launch_step_shape<S, SHIFTED, V, 4, 1, 0>(a, reduce, st);
        case 4: return launch_step_shape<S, SHIFTED, V, 2, 4, 0>(a, reduce, st);
        case 5: return launch_step_shape<S, SHIFTED, V, 4, 2, 1>(a, reduce, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbm
