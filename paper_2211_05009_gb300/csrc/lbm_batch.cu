// lbm_batch.cu -- a sweep of independent cavities of uneven sizes (each its own nx, ny, Re, U) in
// one persistent kernel: the batched form of the step of Xiang & Shi (arXiv 2211.05009) Sec. 2,
// used for the Re x Ar state survey of Sec. 3.3 (Fig. 17).
//
// Work decomposition: every cavity is cut into items of one warp-wide column strip (32*V nodes)
// by R rows; items of all active cavities are numbered consecutively and the warps of the grid
// take them round-robin, so small and large cavities share the GPU.  A launch runs up to one
// checkpoint interval (the plain steps, then the checkpoint step as a second launch of the
// REDUCE variant, which keeps the plain variant's register budget small); steps are separated by
// a grid barrier.  The launch is
// cooperative (all blocks resident) and every barrier wait is bounded by a clock limit: when it
// runs out the kernel sets an error word and returns, and the host reports LBM_ETIMEOUT.
// At each checkpoint (Sec. 2.2 iii) every cavity gets its own Eq. 6 residual and mass (fixed-order
// FP64 sums of per-item partials), cavities whose residual fell below tol -- or that reached the
// step cap -- retire, and the active list is compacted so retired cavities cost nothing.
// The populations of both pools are read and written within one launch, so no load of them takes
// the read-only path: they are either L2 loads (ld.global.cg) or weak L1-cached loads, which are
// coherent here because every read of a pool follows the grid barrier after its last write.
//
// Tile shape: rows per work item (1, 2, 4) x load path (L2 / L1); lbm_batch_autotune times each
// on the batch's own state and keeps the fastest.  Whole checkpoint intervals (the plain launch
// and the checkpoint launch) are captured once in a CUDA graph and replayed.
#include <cuda/atomic>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_step_kernel.cuh"

namespace lbm {

constexpr int kBatchThreads = 128;
static_assert((kBatchThreads & (kBatchThreads - 1)) == 0, "tree reductions assume a power of two");

// Tile shapes: rows per work item x load hint (2: ld.global.cg, 3: ld.global.ca) x resident
// blocks per SM the register budget is sized for (5: 96 registers, 4: 128, 8: 64).  The 8-block
// shapes are for 16-bit storage, whose kernels fit 64 registers without spilling and wait on
// memory latency (45-cavity batch, f16s 124.8 -> 136.5 GLUPS); FP32 spills there and FP64 wants
// the 4-block budget, and the autotuner keeps whichever is fastest.
struct BatchShape {
    int rows, hint, minb;
};
constexpr BatchShape kBatchShapes[LBM_BATCH_SHAPES] = {{2, 2, 5}, {1, 2, 5}, {4, 2, 5}, {2, 3, 5}, {1, 3, 5},
                                                       {4, 3, 5}, {2, 3, 4}, {4, 3, 4}, {2, 2, 8}, {4, 3, 8}};

struct BatchCav {
    long long off;       // population offset (storage elements) in each pool
    long long snap_off;  // snapshot offset (arithmetic-type elements)
    long long pitch, plane;
    int nx, ny;
    double omega, U;
    float omega_f, U_f;
    int corner_moving;
    int strips, items, item0;  // items = strips x ceil(ny / rows) for the current tile shape
    // one observing point per cavity (Sec. 3.3)
    int px, py, every;
    long long cap;
    double* series;
};

struct BatchState {
    long long step;  // global step of the active cavities
    int n_active;
    int err;         // 1: a barrier wait ran out
    unsigned bar_count, bar_gen;
    unsigned claim;  // work-item tickets drawn in the current launch (0 between launches)
    double tol;          // retire when residual < tol (tol <= 0: never)
    long long max_step;  // retire a cavity at this global step (<= 0: never)
    int active[LBM_BATCH_MAX];
    int prefix[LBM_BATCH_MAX + 1];  // exclusive prefix of item counts over the active list
    long long done_at[LBM_BATCH_MAX];  // global step of a retired cavity's state (-1: active)
    long long probe_start[LBM_BATCH_MAX];
    double residual[LBM_BATCH_MAX], mass[LBM_BATCH_MAX];
    int status[LBM_BATCH_MAX];  // 0 active, 1 converged, 2 step cap, 3 non-finite
};

struct BatchArgs {
    void* pool[2];
    void* snap;
    const BatchCav* cavs;
    BatchState* st;
    double* partials;  // 3 per item, full numbering
    int nsteps;
    int rows;             // rows per work item
    int no_probe;         // 1: do not sample the observing points (autotuning trials)
    long long spin_limit; // barrier wait limit in clock cycles
    int absent_block;     // test hook: this block leaves at the first barrier (-1: none)
};

// Grid barrier with a bounded wait.  Returns false (and sets st->err) if the wait ran out or any
// block reported a timeout; callers then return.  The block's writes reach thread 0 through the
// block barrier, and thread 0's device-scope fence and release publish them (fences are
// cumulative), so one fence per block suffices.
__device__ __forceinline__ bool grid_barrier(BatchState* st, long long limit) {
    __shared__ int ok_sh;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int ok = 1;
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> gen(st->bar_gen);
        cuda::atomic_ref<unsigned, cuda::thread_scope_device> cnt(st->bar_count);
        cuda::atomic_ref<int, cuda::thread_scope_device> err(st->err);
        const unsigned g = gen.load(cuda::memory_order_acquire);
        const unsigned arrived = cnt.fetch_add(1u, cuda::memory_order_acq_rel) + 1u;
        if (arrived == gridDim.x) {
            cnt.store(0u, cuda::memory_order_relaxed);
            gen.store(g + 1u, cuda::memory_order_release);
        } else {
            const long long t0 = clock64();
            while (gen.load(cuda::memory_order_acquire) == g) {
                if (err.load(cuda::memory_order_relaxed) || clock64() - t0 > limit) {
                    err.store(1, cuda::memory_order_relaxed);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        if (err.load(cuda::memory_order_acquire)) ok = 0;
        __threadfence();
        ok_sh = ok;
    }
    __syncthreads();
    return ok_sh != 0;
}

// REDUCE = false: a.nsteps plain steps (none of them a checkpoint step).  REDUCE = true: exactly
// one step, the checkpoint step, followed by the per-cavity reduction and the compaction.
template <typename S, bool SHIFTED, int V, bool REDUCE, int HINT, int MINB>
__global__ void __launch_bounds__(kBatchThreads, MINB) k_batch(const BatchArgs a) {
    using C = typename St<S>::C;
    __shared__ int s_active[LBM_BATCH_MAX];
    __shared__ int s_prefix[LBM_BATCH_MAX + 1];
    __shared__ int s_n;
    BatchState* st = a.st;
    const int lane = threadIdx.x & 31;
    constexpr int W = kBatchThreads / 32;
    const unsigned nwarps = gridDim.x * W;
    const long long step0 = __ldcg(&st->step);
    unsigned ticket0 = 0;  // the claim counter's value at the start of the current step

    for (int s = 0; s < a.nsteps; ++s) {
        const long long step = step0 + s;
        // the active list (changes only at checkpoints, behind barriers)
        if (threadIdx.x == 0) s_n = __ldcg(&st->n_active);
        __syncthreads();
        const int n = s_n;
        for (int k = threadIdx.x; k <= n; k += blockDim.x) {
            if (k < n) s_active[k] = __ldcg(&st->active[k]);
            s_prefix[k] = __ldcg(&st->prefix[k]);
        }
        __syncthreads();
        const int n_items = s_prefix[n];
        // a select, not a[step & 1]: a dynamic index into the parameter array would copy the
        // whole argument block to local memory
        const bool odd = (step & 1) != 0;
        const S* src_pool = static_cast<const S*>(odd ? a.pool[1] : a.pool[0]);
        S* dst_pool = static_cast<S*>(odd ? a.pool[0] : a.pool[1]);
        // Work items are drawn one at a time from a grid-wide ticket counter, so that a warp which
        // drew cheaper items (interior strips, no wall path) takes more of them; a static
        // round-robin gave every warp the same strip of every cavity whenever the warp count was
        // a multiple of the strips per row.  The next ticket is drawn during the item's last row,
        // which hides the atomic's latency.  Each warp draws exactly one ticket past the end per
        // step, so a step consumes n_items + nwarps tickets.
        unsigned t = 0;
        if (lane == 0) t = atomicAdd(&st->claim, 1u);
        // unsigned: a counter left over from an aborted launch can only skip items, never index below 0
        unsigned item = __shfl_sync(kFull, t, 0) - ticket0;
        while (item < (unsigned)n_items) {
            int lo = 0, hi = n - 1;  // largest k with prefix[k] <= item
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if ((unsigned)s_prefix[mid] <= item) lo = mid; else hi = mid - 1;
            }
            const BatchCav& cd = a.cavs[s_active[lo]];
            const int local = (int)(item - s_prefix[lo]);
            const int strip = local % cd.strips, rg = local / cd.strips;
            CavityView<C> cv;
            cv.nx = cd.nx;
            cv.ny = cd.ny;
            cv.pitch = cd.pitch;
            cv.plane = cd.plane;
            cv.omega = sizeof(C) == 4 ? C(cd.omega_f) : C(cd.omega);
            cv.Ulid = sizeof(C) == 4 ? C(cd.U_f) : C(cd.U);
            cv.corner_moving = cd.corner_moving;
            cv.sref = cv.sref_w = C(0);  // reference density: LBM_Q16S only, which batches do not take
            ProbeOne pr;
            pr.n_ = (cd.series && !a.no_probe) ? 1 : 0;
            pr.px_ = cd.px;
            pr.py_ = cd.py;
            pr.every_ = cd.every > 0 ? cd.every : 1;
            pr.start_ = cd.series ? __ldcg(&st->probe_start[s_active[lo]]) : 0;
            pr.cap_ = cd.cap > 0 ? cd.cap : 1;
            pr.series_ = cd.series;
            const S* src = src_pool + cd.off;
            S* dst = dst_pool + cd.off;
            C* snap = static_cast<C*>(a.snap) + cd.snap_off;
            const int x0 = (strip * 32 + lane) * V;
            C a0 = C(0), a1 = C(0), a2 = C(0);
            unsigned next = 0;
#pragma unroll 1
            for (int r = 0; r < a.rows; ++r) {
                const int y = rg * a.rows + r;
                if (y >= cd.ny) break;
                if (lane == 0 && (r == a.rows - 1 || y + 1 == cd.ny)) next = atomicAdd(&st->claim, 1u);
                step_row<S, SHIFTED, REDUCE, V, HINT, (sizeof(S) < 4)>(src, dst, cv, lane, x0, y, snap, pr,
                                                   [step]() { return step + 1; }, a0, a1, a2);
            }
            if constexpr (REDUCE) {
                const double p0 = warp_sum(double(a0)), p1 = warp_sum(double(a1)), p2 = warp_sum(double(a2));
                if (lane == 0) {
                    double* p = a.partials + 3ll * (cd.item0 + local);
                    p[0] = p0;
                    p[1] = p1;
                    p[2] = p2;
                }
            }
            item = __shfl_sync(kFull, next, 0) - ticket0;
        }
        ticket0 += (unsigned)n_items + nwarps;
        if (a.absent_block == (int)blockIdx.x && s == 0) return;  // test hook: never arrives
        if (!grid_barrier(st, a.spin_limit)) return;
        if constexpr (!REDUCE) continue;

        // checkpoint: per-cavity Eq. 6 and mass, in a fixed order
        __shared__ double red[3][kBatchThreads];
        const double tol = __ldcg(&st->tol);
        const long long max_step = __ldcg(&st->max_step);
        for (int k = blockIdx.x; k < n; k += gridDim.x) {
            const int c = s_active[k];
            const BatchCav& cd = a.cavs[c];
            double q0 = 0.0, q1 = 0.0, q2 = 0.0;
            for (int i = threadIdx.x; i < cd.items; i += blockDim.x) {
                const double* p = a.partials + 3ll * (cd.item0 + i);
                q0 += __ldcg(p);
                q1 += __ldcg(p + 1);
                q2 += __ldcg(p + 2);
            }
            red[0][threadIdx.x] = q0;
            red[1][threadIdx.x] = q1;
            red[2][threadIdx.x] = q2;
            __syncthreads();
            for (int o = kBatchThreads / 2; o > 0; o >>= 1) {
                if (threadIdx.x < o)
                    for (int m = 0; m < 3; ++m) red[m][threadIdx.x] += red[m][threadIdx.x + o];
                __syncthreads();
            }
            if (threadIdx.x == 0) {
                const double r = sqrt(red[1][0] / red[2][0]);
                const double mass = (double)cd.nx * cd.ny + red[0][0];
                st->residual[c] = r;
                st->mass[c] = mass;
                int status = 0;
                if (!isfinite(r) || !isfinite(mass)) status = 3;
                else if (tol > 0.0 && r < tol) status = 1;
                else if (max_step > 0 && step + 1 >= max_step) status = 2;
                st->status[c] = status;
                if (status) st->done_at[c] = step + 1;
            }
            __syncthreads();
        }
        if (!grid_barrier(st, a.spin_limit)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {  // compact the active list
            int m = 0, acc = 0;
            for (int k = 0; k < n; ++k) {
                const int c = s_active[k];
                if (__ldcg(&st->status[c]) == 0) {
                    st->active[m] = c;
                    st->prefix[m] = acc;
                    acc += a.cavs[c].items;
                    ++m;
                }
            }
            st->prefix[m] = acc;
            st->n_active = m;
        }
        if (!grid_barrier(st, a.spin_limit)) return;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {  // every ticket of this launch was drawn before its last barrier
        st->step = step0 + a.nsteps;
        st->claim = 0u;
    }
}

template <typename S, bool SHIFTED, int HINT, int MINB>
static cudaError_t launch_batch_h(const BatchArgs& a, bool reduce, int blocks, cudaStream_t st) {
    constexpr int V = sizeof(S) == 8 ? 2 : 4;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(kBatchThreads);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (reduce) return cudaLaunchKernelEx(&cfg, k_batch<S, SHIFTED, V, true, HINT, MINB>, a);
    return cudaLaunchKernelEx(&cfg, k_batch<S, SHIFTED, V, false, HINT, MINB>, a);
}

template <typename S, bool SHIFTED>
static cudaError_t launch_batch_t(const BatchShape& sh, const BatchArgs& a, bool reduce, int blocks, cudaStream_t st) {
    if (sh.hint == 2 && sh.minb == 5) return launch_batch_h<S, SHIFTED, 2, 5>(a, reduce, blocks, st);
    if (sh.hint == 3 && sh.minb == 5) return launch_batch_h<S, SHIFTED, 3, 5>(a, reduce, blocks, st);
    if (sh.hint == 3 && sh.minb == 4) return launch_batch_h<S, SHIFTED, 3, 4>(a, reduce, blocks, st);
    if (sh.hint == 2 && sh.minb == 8) return launch_batch_h<S, SHIFTED, 2, 8>(a, reduce, blocks, st);
    if (sh.hint == 3 && sh.minb == 8) return launch_batch_h<S, SHIFTED, 3, 8>(a, reduce, blocks, st);
    return cudaErrorInvalidValue;
}

template <typename S, bool SHIFTED, int HINT, int MINB>
static int batch_blocks_h() {
    constexpr int V = sizeof(S) == 8 ? 2 : 4;
    int dev = 0, sms = 0, p0 = 0, p1 = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p0, k_batch<S, SHIFTED, V, false, HINT, MINB>, kBatchThreads, 0) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&p1, k_batch<S, SHIFTED, V, true, HINT, MINB>, kBatchThreads, 0) != cudaSuccess) return 0;
    return (p0 < p1 ? p0 : p1) * sms;  // one grid size that fits both variants
}

template <typename S, bool SHIFTED>
static int batch_blocks_t(const BatchShape& sh) {
    if (sh.hint == 2 && sh.minb == 5) return batch_blocks_h<S, SHIFTED, 2, 5>();
    if (sh.hint == 3 && sh.minb == 5) return batch_blocks_h<S, SHIFTED, 3, 5>();
    if (sh.hint == 3 && sh.minb == 4) return batch_blocks_h<S, SHIFTED, 3, 4>();
    if (sh.hint == 2 && sh.minb == 8) return batch_blocks_h<S, SHIFTED, 2, 8>();
    if (sh.hint == 3 && sh.minb == 8) return batch_blocks_h<S, SHIFTED, 3, 8>();
    return 0;
}

#define LBM_BATCH_DISPATCH(dtype, CALL)                                              \
    switch (dtype) {                                                                 \
        case 0: { using S = double; constexpr bool SH = true; CALL; }               \
        case 1: { using S = float; constexpr bool SH = false; CALL; }               \
        case 2: { using S = float; constexpr bool SH = true; CALL; }                \
        case 3: { using S = __half; constexpr bool SH = true; CALL; }               \
        case 4: { using S = __nv_bfloat16; constexpr bool SH = true; CALL; }        \
        default: break;                                                              \
    }

static cudaError_t launch_batch(int dtype, const BatchShape& sh, const BatchArgs& a, bool reduce, int blocks, cudaStream_t st) {
    LBM_BATCH_DISPATCH(dtype, return (launch_batch_t<S, SH>(sh, a, reduce, blocks, st)));
    return cudaErrorInvalidValue;
}

static int batch_blocks(int dtype, const BatchShape& sh) {
    LBM_BATCH_DISPATCH(dtype, return (batch_blocks_t<S, SH>(sh)));
    return 0;
}

}  // namespace lbm

using namespace lbm;

namespace {
std::string bfmt(const char* f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}
thread_local std::string g_batch_create_error;
}  // namespace

struct lbm_batch {
    int n = 0, dtype = 0;
    std::vector<BatchCav> cavs;
    std::vector<double> tau;
    void* pool[2] = {nullptr, nullptr};
    size_t pool_bytes = 0;
    void* snap = nullptr;
    BatchCav* d_cavs = nullptr;
    BatchState* d_state = nullptr;
    BatchState* h_state = nullptr;  // pinned
    double* partials = nullptr;      // sized for one row per item (the most items)
    int total_items = 0;             // items at one row per item
    double* psi_scratch = nullptr;
    size_t psi_doubles = 0;
    DevState* d_ext = nullptr;  // stream-function results
    DevState* h_ext = nullptr;  // pinned
    int shape = 0;              // index into kBatchShapes
    int blocks = 0;
    long long step = 0;  // host mirror of the active step
    double spin_limit_s = 2.0;
    int absent_block = -1;
    double dev_tol = 0.0;       // the values last written to d_state->tol / max_step
    long long dev_max_step = 0;
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream for graph capture
    cudaGraphExec_t gexec = nullptr;    // one checkpoint interval
    long long graph_key = -1;
    long long graph_launches = 0;
    bool graph_broken = false;
    size_t device_bytes = 0;
    std::string err;

    int fail(int code, const std::string& m) {
        err = m;
        return code;
    }
    int cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return LBM_OK;
        err = bfmt("%s: %s", what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
    void* dalloc(size_t bytes) {
        void* p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        device_bytes += bytes;
        return p;
    }
    int sync() { return cuda(cudaStreamSynchronize(stream), "stream synchronize"); }

    long long cavity_step(int i) const {
        const long long d = h_state->done_at[i];
        return d >= 0 ? d : step;
    }
    FieldArgs field(int i) const {
        FieldArgs a{};
        const BatchCav& c = cavs[i];
        const size_t es = storage_bytes(dtype);
        a.f = (char*)pool[cavity_step(i) & 1] + c.off * es;
        a.nx = c.nx;
        a.ny = c.ny;
        a.pitch = c.pitch;
        a.plane = c.plane;
        a.U = c.U;
        a.corner_moving = c.corner_moving;
        return a;
    }
    long long spin_limit_cycles() const {
        int dev = 0, khz = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
        return (long long)(spin_limit_s * (khz > 0 ? khz : 2000000) * 1000.0);
    }
    BatchArgs args(int nsteps) const {
        BatchArgs a{};
        a.pool[0] = pool[0];
        a.pool[1] = pool[1];
        a.snap = snap;
        a.cavs = d_cavs;
        a.st = d_state;
        a.partials = partials;
        a.nsteps = nsteps;
        a.rows = kBatchShapes[shape].rows;
        a.no_probe = 0;
        a.spin_limit = spin_limit_cycles();
        a.absent_block = -1;
        return a;
    }
    cudaError_t launch(const BatchArgs& a, bool reduce, cudaStream_t st) const {
        return launch_batch(dtype, kBatchShapes[shape], a, reduce, blocks, st);
    }

    // Cut every cavity into items of the shape's row count and rebuild the prefix of the active
    // list.  Needs a current h_state (after pull_state); leaves the upload queued on the stream.
    int relayout(int s) {
        const int rows = kBatchShapes[s].rows;
        const int nb = batch_blocks(dtype, kBatchShapes[s]);
        if (nb <= 0) return fail(LBM_ECUDA, "batch kernel occupancy query failed");
        int item0 = 0;
        for (BatchCav& c : cavs) {
            c.items = c.strips * ((c.ny + rows - 1) / rows);
            c.item0 = item0;
            item0 += c.items;
        }
        BatchState* h = h_state;
        int acc = 0;
        for (int k = 0; k < h->n_active; ++k) {
            h->prefix[k] = acc;
            acc += cavs[h->active[k]].items;
        }
        h->prefix[h->n_active] = acc;
        int rc = cuda(cudaMemcpyAsync(d_cavs, cavs.data(), sizeof(BatchCav) * n, cudaMemcpyHostToDevice, stream), "descriptor upload");
        if (!rc) rc = cuda(cudaMemcpyAsync(d_state->prefix, h->prefix, sizeof(int) * (h->n_active + 1), cudaMemcpyHostToDevice, stream), "prefix upload");
        if (!rc) rc = sync();  // h_state is pinned and the source of the copy above
        if (rc) return rc;
        shape = s;
        blocks = nb;
        return LBM_OK;
    }

    // Retirement rule of the coming launches, kept in device memory so that a captured graph
    // does not depend on it.
    int set_retire(double tol, long long max_step) {
        if (tol == dev_tol && max_step == dev_max_step) return LBM_OK;
        struct { double t; long long m; } v{tol, max_step};
        static_assert(offsetof(BatchState, max_step) == offsetof(BatchState, tol) + sizeof(double), "layout");
        int rc = cuda(cudaMemcpyAsync(&d_state->tol, &v, sizeof v, cudaMemcpyHostToDevice, stream), "retire rule upload");
        if (!rc) rc = sync();
        if (rc) return rc;
        dev_tol = tol;
        dev_max_step = max_step;
        return LBM_OK;
    }

    // One checkpoint interval (the plain launch of kInterval - 1 steps and the checkpoint launch),
    // captured once per tile shape and barrier limit.  A capture the driver refuses leaves
    // graph_broken set and the intervals are launched directly.
    int ensure_graph() {
        const long long key = shape * 1000003LL + (long long)(spin_limit_s * 1e6);
        if (gexec && key == graph_key) return LBM_OK;
        if (gexec) cudaGraphExecDestroy(gexec);
        gexec = nullptr;
        int rc = LBM_OK;
        if (!cap_stream) rc = cuda(cudaStreamCreateWithFlags(&cap_stream, cudaStreamNonBlocking), "capture stream");
        if (rc) return rc;
        BatchArgs a = args(kInterval - 1);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            cudaError_t e1 = launch(a, false, cap_stream);
            a.nsteps = 1;
            if (e1 == cudaSuccess) e1 = launch(a, true, cap_stream);
            e = cudaStreamEndCapture(cap_stream, &g);
            if (e1 != cudaSuccess) e = e1;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, g, 0);
        if (g) cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            cudaGetLastError();
            gexec = nullptr;
            graph_broken = true;
            err = bfmt("graph capture of the batch interval failed (%s); launching directly", cudaGetErrorString(e));
            return LBM_OK;
        }
        graph_key = key;
        return LBM_OK;
    }

    // Advance every active cavity by n steps (retiring per tol / max_step at checkpoints).
    int run(long long n, double tol, long long max_step) {
        int rc = set_retire(tol, max_step);
        while (n > 0 && !rc) {
            if (step % kInterval == 0 && n >= kInterval && absent_block < 0 && !graph_broken) {
                rc = ensure_graph();
                if (rc) return rc;
                if (gexec) {
                    rc = cuda(cudaGraphLaunch(gexec, stream), "batch graph launch");
                    if (rc) return rc;
                    ++graph_launches;
                    step += kInterval;
                    n -= kInterval;
                    continue;
                }
            }
            const long long chunk = std::min<long long>(n, kInterval - step % kInterval);
            BatchArgs a = args((int)chunk);
            a.absent_block = absent_block;
            // plain steps first; a chunk that ends on a checkpoint ends with the REDUCE launch
            const bool ends_on_checkpoint = (step + chunk) % kInterval == 0;
            const long long plain = ends_on_checkpoint ? chunk - 1 : chunk;
            if (plain > 0) {
                a.nsteps = (int)plain;
                rc = cuda(launch(a, false, stream), "batch kernel launch");
                if (rc) return rc;
                a.absent_block = -1;
            }
            if (ends_on_checkpoint) {
                a.nsteps = 1;
                rc = cuda(launch(a, true, stream), "batch checkpoint launch");
                if (rc) return rc;
            }
            absent_block = -1;
            step += chunk;
            n -= chunk;
        }
        return rc;
    }

    int pull_state() {
        int rc = cuda(cudaMemcpyAsync(h_state, d_state, sizeof(BatchState), cudaMemcpyDeviceToHost, stream), "state copy");
        if (!rc) rc = sync();
        if (!rc && h_state->err) {
            // re-arm the barrier so the batch can be used again; the populations of the
            // interrupted launch are partly advanced and must not be trusted
            h_state->err = 0;
            h_state->bar_count = 0;
            h_state->claim = 0;
            cudaMemcpyAsync(&d_state->err, &h_state->err, sizeof(int), cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(&d_state->bar_count, &h_state->bar_count, sizeof(unsigned), cudaMemcpyHostToDevice, stream);
            cudaMemcpyAsync(&d_state->claim, &h_state->claim, sizeof(unsigned), cudaMemcpyHostToDevice, stream);
            sync();
            step = h_state->step;
            return fail(LBM_ETIMEOUT, "a grid barrier wait of the batch kernel ran out");
        }
        if (!rc) step = h_state->step;
        return rc;
    }

    // Time every tile shape on the current state for `steps` plain steps (probes off), then put
    // the state back: the current pool is saved first and restored afterwards, the other pool is
    // rewritten by the next step anyway, retired cavities are never touched.
    int autotune(int steps, int* chosen, float* ms_out) {
        int rc = pull_state();
        if (rc) return rc;
        const int cur = shape;
        float ms[LBM_BATCH_SHAPES];
        for (int s = 0; s < LBM_BATCH_SHAPES; ++s) ms[s] = -1.f;
        if (h_state->n_active == 0) {
            if (chosen) *chosen = cur;
            if (ms_out) std::copy(ms, ms + LBM_BATCH_SHAPES, ms_out);
            return LBM_OK;
        }
        void* backup = nullptr;
        if (cudaMalloc(&backup, pool_bytes) != cudaSuccess) {
            cudaGetLastError();
            return fail(LBM_ENOMEM, bfmt("autotune needs a %zu-byte copy of the populations", pool_bytes));
        }
        const long long step0 = step;
        void* live = pool[step0 & 1];
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        rc = cuda(cudaMemcpyAsync(backup, live, pool_bytes, cudaMemcpyDeviceToDevice, stream), "population backup");
        if (!rc) rc = cuda(cudaEventCreate(&e0), "event");
        if (!rc) rc = cuda(cudaEventCreate(&e1), "event");
        int best = -1;
        for (int s = 0; s < LBM_BATCH_SHAPES && !rc; ++s) {
            rc = relayout(s);
            if (rc) break;
            BatchArgs a = args(2);
            a.no_probe = 1;
            rc = cuda(launch(a, false, stream), "autotune warm-up");
            a.nsteps = steps;
            if (!rc) rc = cuda(cudaEventRecord(e0, stream), "event");
            if (!rc) rc = cuda(launch(a, false, stream), "autotune trial");
            if (!rc) rc = cuda(cudaEventRecord(e1, stream), "event");
            if (!rc) rc = sync();
            if (!rc) rc = cuda(cudaEventElapsedTime(&ms[s], e0, e1), "event time");
            if (!rc) {
                rc = pull_state();  // a barrier timeout surfaces here
                if (!rc && (best < 0 || ms[s] < ms[best])) best = s;
            }
        }
        // Among the shapes within 2 % of the fastest, keep the one with the fewest rows per item:
        // the trials run with every cavity active, and as cavities retire the finer items keep
        // more warps busy (45 FP64 cavities 128 wide to Eq. 6 < 1e-9: 37.0 s with 1-row items
        // against 46.8 s with 4-row items whose trial had been 0.7 % faster).
        if (!rc && best >= 0) {
            int pick = best;
            for (int s = 0; s < LBM_BATCH_SHAPES; ++s) {
                if (ms[s] < 0.f || ms[s] > 1.02f * ms[best]) continue;
                const int rs = kBatchShapes[s].rows, rp = kBatchShapes[pick].rows;
                if (rs < rp || (rs == rp && ms[s] < ms[pick])) pick = s;
            }
            best = pick;
        }
        // restore: populations, the step counter, the chosen layout
        int rc2 = cuda(cudaMemcpyAsync(live, backup, pool_bytes, cudaMemcpyDeviceToDevice, stream), "population restore");
        if (!rc2) {
            h_state->step = step0;
            rc2 = cuda(cudaMemcpyAsync(&d_state->step, &h_state->step, sizeof(long long), cudaMemcpyHostToDevice, stream), "step restore");
        }
        if (!rc2) rc2 = sync();
        step = step0;
        if (!rc2) rc2 = relayout(rc || best < 0 ? cur : best);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(backup);
        if (rc) return rc;
        if (rc2) return rc2;
        if (chosen) *chosen = best;
        if (ms_out) std::copy(ms, ms + LBM_BATCH_SHAPES, ms_out);
        return LBM_OK;
    }
};

extern "C" int lbm_batch_create(int n, const int* nx, const int* ny, const double* Re, const double* U,
                                lbm_dtype dtype, lbm_batch** out) {
    g_batch_create_error.clear();
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    auto bad = [&](const std::string& m) {
        g_batch_create_error = m;
        return LBM_EINVAL;
    };
    if (n < 1 || n > LBM_BATCH_MAX) return bad(bfmt("batch of %d cavities: need 1..%d", n, LBM_BATCH_MAX));
    if (!nx || !ny || !Re || !U) return bad("NULL parameter array");
    if ((int)dtype < 0 || (int)dtype > 5) return bad("unknown dtype");
    if ((int)dtype == kDtypeQ16S) return bad("LBM_Q16S storage is for single cavities only");
    for (int i = 0; i < n; ++i) {
        if (nx[i] < 3 || ny[i] < 3) return bad(bfmt("cavity %d: grid %d x %d, need >= 3", i, nx[i], ny[i]));
        const double tau = 3.0 * U[i] * nx[i] / Re[i] + 0.5;
        if (!(Re[i] > 0) || !(tau > 0.5) || !std::isfinite(tau)) return bad(bfmt("cavity %d: Re/U give tau = %g", i, tau));
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        g_batch_create_error = "no CUDA device available (the library has no CPU path)";
        return LBM_ECUDA;
    }
    lbm_batch* b = new lbm_batch();
    b->n = n;
    b->dtype = (int)dtype;
    const int V = storage_bytes(b->dtype) == 8 ? 2 : 4;
    long long off = 0, soff = 0;
    int item0 = 0;
    size_t max_psi = 0;
    for (int i = 0; i < n; ++i) {
        BatchCav c{};
        c.nx = nx[i];
        c.ny = ny[i];
        c.pitch = row_pitch(b->dtype, nx[i]);
        c.plane = c.pitch * ny[i];
        const double tau = 3.0 * U[i] * nx[i] / Re[i] + 0.5;  // Re = U nx / nu, Eq. 5
        b->tau.push_back(tau);
        c.omega = 1.0 / tau;
        c.U = U[i];
        c.omega_f = (float)c.omega;
        c.U_f = (float)U[i];
        c.off = off;
        c.snap_off = soff;
        c.strips = (int)(c.pitch / (32 * V));
        c.items = c.strips * ny[i];  // one row per item: the largest item count of any shape
        c.item0 = item0;
        c.series = nullptr;
        off += 9 * c.plane;
        off = (off + 63) / 64 * 64;  // keep every cavity 512-byte aligned
        soff += 2 * c.plane;
        item0 += c.items;
        max_psi = std::max(max_psi, psi_scratch_doubles(nx[i], ny[i]));
        b->cavs.push_back(c);
    }
    b->total_items = item0;
    auto fail = [&](int code, const std::string& m) {
        g_batch_create_error = m.empty() ? b->err : m;
        lbm_batch_destroy(b);
        return code;
    };
    const size_t es = storage_bytes(b->dtype);
    b->pool_bytes = (size_t)off * es;
    for (int p = 0; p < 2; ++p)
        if (!(b->pool[p] = b->dalloc(b->pool_bytes))) return fail(LBM_ENOMEM, bfmt("population pool of %zu bytes", b->pool_bytes));
    b->snap = b->dalloc((size_t)soff * arith_bytes(b->dtype));
    b->d_cavs = (BatchCav*)b->dalloc(sizeof(BatchCav) * n);
    b->d_state = (BatchState*)b->dalloc(sizeof(BatchState));
    b->partials = (double*)b->dalloc(sizeof(double) * 3 * (size_t)b->total_items);
    b->psi_doubles = max_psi;
    b->psi_scratch = (double*)b->dalloc(sizeof(double) * max_psi);
    b->d_ext = (DevState*)b->dalloc(sizeof(DevState));
    if (!b->snap || !b->d_cavs || !b->d_state || !b->partials || !b->psi_scratch || !b->d_ext) return fail(LBM_ENOMEM, "batch scratch allocation");
    int rc = b->cuda(cudaMallocHost(&b->h_state, sizeof(BatchState)), "pinned host allocation");
    if (!rc) rc = b->cuda(cudaMallocHost(&b->h_ext, sizeof(DevState)), "pinned host allocation");
    if (rc) return fail(rc, "");
    // initial state (Sec. 2.2 i) for every cavity, in both pools
    for (int i = 0; i < n && !rc; ++i)
        for (int p = 0; p < 2 && !rc; ++p) {
            FieldArgs a{};
            a.f = (char*)b->pool[p] + b->cavs[i].off * es;
            a.nx = nx[i];
            a.ny = ny[i];
            a.pitch = b->cavs[i].pitch;
            a.plane = b->cavs[i].plane;
            a.U = U[i];
            a.corner_moving = 0;
            void* sp = (char*)b->snap + b->cavs[i].snap_off * arith_bytes(b->dtype);
            rc = b->cuda(launch_init(b->dtype, a, sp, b->stream), "init kernel launch");
        }
    if (rc) return fail(rc, "");
    BatchState* h = b->h_state;
    memset(h, 0, sizeof(BatchState));
    h->n_active = n;
    int acc = 0;
    for (int i = 0; i < n; ++i) {
        h->active[i] = i;
        h->prefix[i] = acc;
        acc += b->cavs[i].items;
        h->done_at[i] = -1;
    }
    h->prefix[n] = acc;
    rc = b->cuda(cudaMemcpyAsync(b->d_cavs, b->cavs.data(), sizeof(BatchCav) * n, cudaMemcpyHostToDevice, b->stream), "descriptor upload");
    if (!rc) rc = b->cuda(cudaMemcpyAsync(b->d_state, h, sizeof(BatchState), cudaMemcpyHostToDevice, b->stream), "state upload");
    if (!rc) rc = b->sync();
    if (!rc) rc = b->relayout(0);
    if (rc) return fail(rc, "");
    *out = b;
    return LBM_OK;
}

extern "C" void lbm_batch_destroy(lbm_batch* b) {
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    for (void* p : {b->pool[0], b->pool[1], b->snap, (void*)b->d_cavs, (void*)b->d_state, (void*)b->partials, (void*)b->psi_scratch, (void*)b->d_ext})
        if (p) cudaFree(p);
    if (b->h_state) cudaFreeHost(b->h_state);
    if (b->h_ext) cudaFreeHost(b->h_ext);
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    delete b;
}

extern "C" const char* lbm_batch_last_error(const lbm_batch* b) {
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

extern "C" int lbm_batch_set_stream(lbm_batch* b, void* stream) {
    if (!b) return LBM_EINVAL;
    int rc = b->sync();
    b->stream = (cudaStream_t)stream;
    return rc;
}

extern "C" int lbm_batch_step(lbm_batch* b, long n) {
    if (!b) return LBM_EINVAL;
    NvtxRange r("lbm_batch_step");
    if (n < 0) return b->fail(LBM_EINVAL, "n < 0");
    int rc = b->run(n, -1.0, 0);
    if (!rc) rc = b->pull_state();
    return rc;
}

extern "C" int lbm_batch_run_to_residual(lbm_batch* b, double tol, long max_steps, long* steps_done) {
    if (!b) return LBM_EINVAL;
    NvtxRange r("lbm_batch_run_to_residual");
    if (!(tol > 0) || max_steps < 0) return b->fail(LBM_EINVAL, "need tol > 0 and max_steps >= 0");
    const long long start = b->step;
    const long long cap = start + max_steps;
    int rc = LBM_OK;
    // run in chunks of 10 checkpoint intervals, stopping early once every cavity retired
    while (!rc && b->step < cap) {
        const long long chunk = std::min<long long>(cap - b->step, 10 * kInterval);
        rc = b->run(chunk, tol, cap);
        if (!rc) rc = b->pull_state();
        if (!rc && b->h_state->n_active == 0) break;
    }
    if (rc) return rc;
    bool all = true;
    for (int i = 0; i < b->n; ++i) {
        const long long d = b->h_state->done_at[i];
        if (steps_done) steps_done[i] = (long)((d >= 0 ? d : b->step) - start);
        if (b->h_state->status[i] == 3) return b->fail(LBM_EDIVERGED, bfmt("cavity %d diverged", i));
        if (b->h_state->status[i] != 1) all = false;
    }
    return all ? LBM_OK : b->fail(LBM_ENOTREADY, "some cavities did not reach tol within max_steps");
}

extern "C" int lbm_batch_residual(lbm_batch* b, double* r, int* status) {
    if (!b || !r) return LBM_EINVAL;
    int rc = b->pull_state();
    if (rc) return rc;
    for (int i = 0; i < b->n; ++i) {
        r[i] = b->h_state->residual[i];
        if (status) status[i] = b->h_state->status[i];
    }
    return LBM_OK;
}

extern "C" int lbm_batch_cavity_steps(lbm_batch* b, long* steps) {
    if (!b || !steps) return LBM_EINVAL;
    int rc = b->pull_state();
    if (rc) return rc;
    for (int i = 0; i < b->n; ++i) steps[i] = (long)b->cavity_step(i);
    return LBM_OK;
}

extern "C" int lbm_batch_moments(lbm_batch* b, int i, double* rho, double* ux, double* uy) {
    if (!b || i < 0 || i >= b->n) return b ? b->fail(LBM_EINVAL, "no such cavity") : LBM_EINVAL;
    int rc = b->pull_state();
    if (rc) return rc;
    const size_t bytes = (size_t)b->cavs[i].nx * b->cavs[i].ny * sizeof(double);
    double* outs[3] = {rho, ux, uy};
    for (int k = 0; k < 3; ++k) {
        if (!outs[k]) continue;
        cudaPointerAttributes at{};
        cudaError_t e = cudaPointerGetAttributes(&at, outs[k]);
        if (e != cudaSuccess) cudaGetLastError();
        if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)))
            return b->fail(LBM_EINVAL, "lbm_batch_moments needs device buffers");
    }
    (void)bytes;
    rc = b->cuda(launch_moments(b->dtype, b->field(i), rho, ux, uy, b->stream), "moments launch");
    if (!rc) rc = b->sync();
    return rc;
}

extern "C" int lbm_batch_get_populations(lbm_batch* b, int i, double* f) {
    if (!b || i < 0 || i >= b->n || !f) return b ? b->fail(LBM_EINVAL, "bad arguments") : LBM_EINVAL;
    int rc = b->pull_state();
    if (rc) return rc;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, f);
    if (e != cudaSuccess) cudaGetLastError();
    if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)))
        return b->fail(LBM_EINVAL, "lbm_batch_get_populations needs a device buffer");
    rc = b->cuda(launch_get_populations(b->dtype, b->field(i), f, b->stream), "get_populations launch");
    if (!rc) rc = b->sync();
    return rc;
}

extern "C" int lbm_batch_stream_function(lbm_batch* b, int i, double* psi, double* psi_min, double* xc, double* yc) {
    if (!b || i < 0 || i >= b->n) return b ? b->fail(LBM_EINVAL, "no such cavity") : LBM_EINVAL;
    int rc = b->pull_state();
    if (rc) return rc;
    const BatchCav& c = b->cavs[i];
    if (psi) {
        cudaPointerAttributes at{};
        cudaError_t e = cudaPointerGetAttributes(&at, psi);
        if (e != cudaSuccess) cudaGetLastError();
        if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)))
            return b->fail(LBM_EINVAL, "lbm_batch_stream_function needs a device psi buffer");
    }
    rc = b->cuda(launch_stream_function(b->dtype, b->field(i), psi, 0, c.nx, 0, c.ny, b->psi_scratch, b->d_ext, b->stream), "stream function launch");
    if (!rc) rc = b->cuda(cudaMemcpyAsync(b->h_ext, b->d_ext, sizeof(DevState), cudaMemcpyDeviceToHost, b->stream), "extrema copy");
    if (!rc) rc = b->sync();
    if (rc) return rc;
    if (psi_min) *psi_min = b->h_ext->ext[0];
    if (xc) *xc = b->h_ext->ext[1] / c.nx;
    if (yc) *yc = b->h_ext->ext[2] / c.nx;
    return std::isfinite(b->h_ext->ext[0]) ? LBM_OK : b->fail(LBM_EDIVERGED, "non-finite stream function");
}

extern "C" int lbm_batch_probe(lbm_batch* b, const double* x, const double* y, int every, double* dev_series, long cap) {
    if (!b || !x || !y || !dev_series || every < 1 || cap < 1) return b ? b->fail(LBM_EINVAL, "bad probe arguments") : LBM_EINVAL;
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, dev_series);
    if (e != cudaSuccess) cudaGetLastError();
    if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)))
        return b->fail(LBM_EINVAL, "probe series must be device memory");
    int rc = b->pull_state();
    if (rc) return rc;
    for (int i = 0; i < b->n; ++i) {
        BatchCav& c = b->cavs[i];
        int px = (int)std::floor(x[i] * c.nx + 0.5), py = (int)std::floor(y[i] * c.nx + 0.5);
        c.px = px < 0 ? 0 : (px >= c.nx ? c.nx - 1 : px);
        c.py = py < 0 ? 0 : (py >= c.ny ? c.ny - 1 : py);
        c.every = every;
        c.cap = cap;
        c.series = dev_series + 2ll * cap * i;
        b->h_state->probe_start[i] = b->cavity_step(i);
    }
    rc = b->cuda(cudaMemcpyAsync(b->d_cavs, b->cavs.data(), sizeof(BatchCav) * b->n, cudaMemcpyHostToDevice, b->stream), "descriptor upload");
    if (!rc) rc = b->cuda(cudaMemcpyAsync(b->d_state->probe_start, b->h_state->probe_start, sizeof(long long) * b->n, cudaMemcpyHostToDevice, b->stream), "probe start upload");
    if (!rc) rc = b->sync();
    return rc;
}

extern "C" int lbm_batch_info(lbm_batch* b, int i, lbm_info* info) {
    if (!b || !info || i < 0 || i >= b->n) return LBM_EINVAL;
    const BatchCav& c = b->cavs[i];
    info->nx = c.nx;
    info->ny = c.ny;
    info->pitch = (long)c.pitch;
    info->tau = b->tau[i];
    info->nu = (b->tau[i] - 0.5) / 3.0;
    info->U = c.U;
    info->Re = c.U * c.nx / info->nu;
    info->dtype = b->dtype;
    info->flags = 0;
    info->step = (long)b->cavity_step(i);
    info->device_bytes = b->device_bytes;
    info->launch_config = b->shape;
    return LBM_OK;
}

extern "C" int lbm_batch_set_shape(lbm_batch* b, int shape) {
    if (!b) return LBM_EINVAL;
    if (shape < 0 || shape >= LBM_BATCH_SHAPES) return b->fail(LBM_EINVAL, bfmt("tile shape %d: need 0..%d", shape, LBM_BATCH_SHAPES - 1));
    int rc = b->pull_state();
    if (!rc) rc = b->relayout(shape);
    return rc;
}

extern "C" int lbm_batch_autotune(lbm_batch* b, int steps, int* chosen, float* ms) {
    if (!b) return LBM_EINVAL;
    NvtxRange r("lbm_batch_autotune");
    if (steps < 1 || steps > 10000) return b->fail(LBM_EINVAL, "autotune: need 1 <= steps <= 10000");
    return b->autotune(steps, chosen, ms);
}

extern "C" int lbm_batch_launch_info(lbm_batch* b, int* shape, int* rows_per_item, int* blocks, long* graph_launches) {
    if (!b) return LBM_EINVAL;
    if (shape) *shape = b->shape;
    if (rows_per_item) *rows_per_item = kBatchShapes[b->shape].rows;
    if (blocks) *blocks = b->blocks;
    if (graph_launches) *graph_launches = (long)b->graph_launches;
    return b->graph_broken ? b->fail(LBM_ECUDA, b->err) : LBM_OK;
}

extern "C" int lbm_batch_set_barrier_limit(lbm_batch* b, double seconds, int absent_block) {
    if (!b || !(seconds > 0)) return LBM_EINVAL;
    b->spin_limit_s = seconds;
    b->absent_block = absent_block;
    return LBM_OK;
}

extern "C" int lbm_batch_set_moments(lbm_batch* b, int i, const double* rho, const double* ux, const double* uy) {
    return lbm_batch_set_moments_ex(b, i, rho, ux, uy, 0);
}

extern "C" int lbm_batch_set_moments_ex(lbm_batch* b, int i, const double* rho, const double* ux, const double* uy,
                                        int flags) {
    if (!b || i < 0 || i >= b->n || !rho || !ux || !uy) return b ? b->fail(LBM_EINVAL, "bad arguments") : LBM_EINVAL;
    if (flags & ~LBM_INIT_NEQ) return b->fail(LBM_EINVAL, "unknown lbm_batch_set_moments_ex flag");
    int rc = b->pull_state();
    if (rc) return rc;
    for (const double* p : {rho, ux, uy}) {
        cudaPointerAttributes at{};
        cudaError_t e = cudaPointerGetAttributes(&at, p);
        if (e != cudaSuccess) cudaGetLastError();
        if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)))
            return b->fail(LBM_EINVAL, "lbm_batch_set_moments needs device buffers");
    }
    if (b->h_state->done_at[i] >= 0 || b->step % kInterval != 0)
        return b->fail(LBM_EINVAL, "cavity retired, or the batch is not at a checkpoint boundary");
    const BatchCav& c = b->cavs[i];
    void* sp = (char*)b->snap + c.snap_off * arith_bytes(b->dtype);
    rc = b->cuda(launch_set_moments(b->dtype, b->field(i), rho, ux, uy, sp, (flags & LBM_INIT_NEQ) ? b->tau[i] : 0.0,
                                    b->stream), "set_moments launch");
    if (!rc) rc = b->sync();
    return rc;
}
