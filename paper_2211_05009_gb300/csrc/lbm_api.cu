// lbm_api.cu -- host side of the C ABI declared in include/lbm.h: context lifetime, the time loop
// (single launches and 100-step CUDA graphs), checkpointing of Eq. 6 results, field import and
// export through caller buffers, probes and save/load.  All compute runs in the kernels of
// lbm_step.cu and lbm_aux.cu; nothing here touches population values on the CPU.
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>

#include "lbm.h"
#include "lbm_internal.h"

using namespace lbm;

namespace {

thread_local std::string g_create_error;

void* (*g_alloc)(size_t, void*) = nullptr;
void (*g_release)(void*, void*) = nullptr;
void* g_alloc_user = nullptr;

std::string fmt(const char* f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}

}  // namespace

struct lbm_ctx {
    int nx = 0, ny = 0;
    long long pitch = 0, plane = 0;
    double tau = 0, U = 0;
    int dtype = 0;
    unsigned flags = 0;
    long long step = 0;  // global time step of the current state

    // allocator used for this context's device memory
    void* (*alloc)(size_t, void*) = nullptr;
    void (*release)(void*, void*) = nullptr;
    void* alloc_user = nullptr;
    size_t device_bytes = 0;

    void* buf[2] = {nullptr, nullptr};  // populations, ping-pong; current = buf[step & 1]
    void* snap = nullptr;               // [2][ny][pitch] Eq. 6 snapshot (arithmetic type)
    double* partials = nullptr;         // reduction partials
    int npartials = 0;
    double* psi_scratch = nullptr;
    DevState* d_state = nullptr;
    DevState* h_state = nullptr;  // pinned, two slots (alternating checkpoints)
    void* stage = nullptr;        // device staging for host buffers
    size_t stage_bytes = 0;

    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t chunk[2] = {nullptr, nullptr};
    cudaEvent_t ev[2] = {nullptr, nullptr};

    ProbeSet probes{};
    int cfg = 0;  // launch shape of the step kernel
    QCodec q{};   // LBM_Q16S scales (from U at creation)
    StepGeometry geo{};
    std::string err;

    int fail(int code, const std::string& m) {
        err = m;
        return code;
    }
    int cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return LBM_OK;
        err = fmt("%s: %s", what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }

    void* dalloc(size_t bytes) {
        void* p = nullptr;
        if (alloc) {
            p = alloc(bytes, alloc_user);
        } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
        if (p) device_bytes += bytes;
        return p;
    }
    void dfree(void* p) {
        if (!p) return;
        if (release)
            release(p, alloc_user);
        else
            cudaFree(p);
    }

    FieldArgs field(int which) const {
        FieldArgs a{};
        a.f = buf[which];
        a.nx = nx;
        a.ny = ny;
        a.pitch = pitch;
        a.plane = plane;
        a.U = U;
        a.corner_moving = (flags & LBM_FLAG_LID_CORNERS_MOVING) ? 1 : 0;
        a.q = q;
        a.st = d_state;
        return a;
    }
    FieldArgs cur() const { return field((int)(step & 1)); }

    StepArgs step_args(long long gstep, int s) const {
        StepArgs a{};
        a.src = buf[gstep & 1];
        a.dst = buf[(gstep + 1) & 1];
        a.nx = nx;
        a.ny = ny;
        a.pitch = pitch;
        a.plane = plane;
        a.omega = 1.0 / tau;
        a.U = U;
        a.omega_f = (float)a.omega;
        a.U_f = (float)U;
        a.corner_moving = (flags & LBM_FLAG_LID_CORNERS_MOVING) ? 1 : 0;
        a.s = s;
        a.state = d_state;
        a.probes = probes;
        a.snap = snap;
        a.partials = partials;
        a.q = q;
        return a;
    }

    void invalidate_graphs() {
        for (auto& g : chunk)
            if (g) {
                cudaGraphExecDestroy(g);
                g = nullptr;
            }
    }

    // Enqueue the kernels of one time step from global step gstep on stream st.
    int enqueue_step(long long gstep, cudaStream_t st) {
        const int s = (int)(gstep % kInterval);
        const bool reduce = (gstep + 1) % kInterval == 0;
        int rc = cuda(launch_step(dtype, cfg, step_args(gstep, s), reduce, st), "step kernel launch");
        if (rc) return rc;
        if (reduce) {
            rc = cuda(launch_finalize_checkpoint(partials, geo.blocks, (double)nx * ny, d_state, st),
                      "checkpoint reduction launch");
            if (rc) return rc;
            const int slot = (int)(((gstep + 1) / kInterval) & 1);
            rc = cuda(cudaMemcpyAsync(&h_state[slot], d_state, sizeof(DevState),
                                      cudaMemcpyDeviceToHost, st),
                      "checkpoint copy");
        }
        return rc;
    }

    // 100-step graph for chunks that start at an aligned step; slot = parity of the checkpoint.
    int ensure_graph(int slot) {
        if (chunk[slot]) return LBM_OK;
        cudaGraph_t g = nullptr;
        int rc = cuda(cudaStreamBeginCapture(cap_stream, cudaStreamCaptureModeThreadLocal),
                      "begin graph capture");
        if (rc) return rc;
        // the chunk ends at a checkpoint of parity `slot`; its first step is a multiple of 100
        const long long g0 = slot == 1 ? 0 : kInterval;
        for (int s = 0; s < kInterval && !rc; ++s) rc = enqueue_step(g0 + s, cap_stream);
        cudaError_t e = cudaStreamEndCapture(cap_stream, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        rc = cuda(e, "end graph capture");
        if (rc) return rc;
        rc = cuda(cudaGraphInstantiate(&chunk[slot], g, 0), "graph instantiate");
        cudaGraphDestroy(g);
        return rc;
    }

    int advance(long long n) {
        int rc = LBM_OK;
        while (n > 0 && !rc) {
            if (step % kInterval == 0 && n >= kInterval) {
                const int slot = (int)(((step + kInterval) / kInterval) & 1);
                rc = ensure_graph(slot);
                if (rc) return rc;
                rc = cuda(cudaGraphLaunch(chunk[slot], stream), "graph launch");
                if (rc) return rc;
                step += kInterval;
                n -= kInterval;
            } else {
                rc = enqueue_step(step, stream);
                if (rc) return rc;
                step += 1;
                n -= 1;
            }
        }
        return rc;
    }

    // Resolve a caller buffer: device pointers are used directly, host pointers go through
    // the staging buffer.  Returns the device pointer to use, or null on failure.
    double* device_view(const void* p, size_t bytes, size_t offset, bool* staged) {
        cudaPointerAttributes at{};
        cudaError_t e = cudaPointerGetAttributes(&at, p);
        if (e != cudaSuccess) cudaGetLastError();
        if (e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)) {
            *staged = false;
            return (double*)const_cast<void*>(p);
        }
        *staged = true;
        if (stage_bytes < offset + bytes) return nullptr;
        return (double*)((char*)stage + offset);
    }
    // Device address of page-locked host memory mapped into the device's address space (pinned
    // allocations under unified addressing), or null: such buffers are read or written by the
    // kernels directly over the host link instead of through the staging buffer and a copy.
    static double* mapped_host(const void* p) {
        cudaPointerAttributes at{};
        if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        return at.type == cudaMemoryTypeHost ? static_cast<double*>(at.devicePointer) : nullptr;
    }
    int ensure_stage(size_t bytes) {
        if (stage_bytes >= bytes) return LBM_OK;
        if (stage) {
            cudaStreamSynchronize(stream);
            dfree(stage);
            device_bytes -= stage_bytes;
        }
        stage = dalloc(bytes);
        stage_bytes = stage ? bytes : 0;
        return stage ? LBM_OK : fail(LBM_ENOMEM, fmt("staging buffer of %zu bytes", bytes));
    }

    int sync() { return cuda(cudaStreamSynchronize(stream), "stream synchronize"); }
};

// ------------------------------------------------------------------ lifetime
extern "C" int lbm_set_allocator(void* (*alloc)(size_t, void*), void (*release)(void*, void*), void* user) {
    if ((alloc == nullptr) != (release == nullptr)) return LBM_EINVAL;
    g_alloc = alloc;
    g_release = release;
    g_alloc_user = user;
    return LBM_OK;
}

extern "C" void lbm_destroy(lbm_ctx* c) {
    if (!c) return;
    if (c->stream || c->cap_stream) cudaStreamSynchronize(c->stream);
    c->invalidate_graphs();
    for (auto& e : c->ev)
        if (e) cudaEventDestroy(e);
    c->dfree(c->buf[0]);
    c->dfree(c->buf[1]);
    c->dfree(c->snap);
    c->dfree(c->partials);
    c->dfree(c->psi_scratch);
    c->dfree(c->d_state);
    c->dfree(c->stage);
    if (c->h_state) cudaFreeHost(c->h_state);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    delete c;
}

static int create_fail(lbm_ctx* c, int code, const std::string& m) {
    g_create_error = m.empty() && c ? c->err : m;
    lbm_destroy(c);
    return code;
}

extern "C" int lbm_create_ex(int nx, int ny, double tau, double U, lbm_dtype dtype, unsigned flags,
                             lbm_ctx** out) {
    g_create_error.clear();
    if (!out) return create_fail(nullptr, LBM_EINVAL, "out is NULL");
    *out = nullptr;
    if (nx < 3 || ny < 3) return create_fail(nullptr, LBM_EINVAL, fmt("grid %d x %d: need nx, ny >= 3", nx, ny));
    if (!(tau > 0.5) || !std::isfinite(tau)) return create_fail(nullptr, LBM_EINVAL, fmt("tau = %g: need tau > 1/2", tau));
    if (!std::isfinite(U)) return create_fail(nullptr, LBM_EINVAL, "U is not finite");
    if ((int)dtype < 0 || (int)dtype > 5) return create_fail(nullptr, LBM_EINVAL, fmt("unknown dtype %d", (int)dtype));
    if (flags & ~LBM_FLAG_LID_CORNERS_MOVING) return create_fail(nullptr, LBM_EINVAL, "unknown flags");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return create_fail(nullptr, LBM_ECUDA, "no CUDA device available (the library has no CPU path)");
    }

    lbm_ctx* c = new lbm_ctx();
    c->nx = nx;
    c->ny = ny;
    c->tau = tau;
    c->U = U;
    c->dtype = (int)dtype;
    c->flags = flags;
    c->alloc = g_alloc;
    c->release = g_release;
    c->alloc_user = g_alloc_user;
    c->pitch = row_pitch(c->dtype, nx);
    c->q = q16_codec(U);
    c->plane = c->pitch * (long long)ny;
    c->cfg = default_step_config(c->dtype);
    c->geo = step_geometry(c->dtype, c->cfg, ny, c->pitch);
    int max_blocks = 0;
    for (int k = 0; k < kStepConfigs; ++k) {
        const int b = step_geometry(c->dtype, k, ny, c->pitch).blocks;
        max_blocks = b > max_blocks ? b : max_blocks;
    }

    const size_t pop_bytes = 9ull * (size_t)c->plane * (size_t)storage_bytes(c->dtype);
    int rc;
    for (int b = 0; b < 2; ++b) {
        c->buf[b] = c->dalloc(pop_bytes);
        if (!c->buf[b]) return create_fail(c, LBM_ENOMEM, fmt("population buffer of %zu bytes", pop_bytes));
    }
    c->snap = c->dalloc(2ull * (size_t)c->plane * arith_bytes(c->dtype));
    c->npartials = 3 * max_blocks > 4096 ? 3 * max_blocks : 4096;
    c->partials = (double*)c->dalloc((size_t)c->npartials * sizeof(double));
    c->psi_scratch = (double*)c->dalloc(psi_scratch_doubles(nx, ny) * sizeof(double));
    c->d_state = (DevState*)c->dalloc(sizeof(DevState));
    if (!c->snap || !c->partials || !c->psi_scratch || !c->d_state)
        return create_fail(c, LBM_ENOMEM, "device allocation of snapshot/scratch failed");
    if ((rc = c->cuda(cudaMallocHost(&c->h_state, 2 * sizeof(DevState)), "pinned host allocation")))
        return create_fail(c, rc, "");
    memset(c->h_state, 0, 2 * sizeof(DevState));
    if ((rc = c->cuda(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "stream create")))
        return create_fail(c, rc, "");
    for (auto& e : c->ev)
        if ((rc = c->cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "event create")))
            return create_fail(c, rc, "");
    // the device state first: the LBM_Q16S initial state is stored against its reference density
    if ((rc = c->cuda(cudaMemsetAsync(c->d_state, 0, sizeof(DevState), c->stream), "state reset")))
        return create_fail(c, rc, "");
    // both buffers hold the initial state, so padding is defined in either
    for (int b = 0; b < 2; ++b)
        if ((rc = c->cuda(launch_init(c->dtype, c->field(b), c->snap, c->stream), "init kernel launch")))
            return create_fail(c, rc, "");
    if ((rc = c->sync())) return create_fail(c, rc, "");
    *out = c;
    return LBM_OK;
}

extern "C" int lbm_create_flags(int nx, int ny, double Re, double U, lbm_dtype dtype, unsigned flags,
                                lbm_ctx** out) {
    if (!(Re > 0.0) || !std::isfinite(Re)) {
        g_create_error = fmt("Re = %g: need Re > 0", Re);
        if (out) *out = nullptr;
        return LBM_EINVAL;
    }
    const double nu = U * nx / Re;  // Re = U L / nu with L = nx
    const double tau = 3.0 * nu + 0.5;  // Eq. 5 with c_s^2 = 1/3, dt = 1
    return lbm_create_ex(nx, ny, tau, U, dtype, flags, out);
}

extern "C" int lbm_create(int nx, int ny, double Re, double U, lbm_dtype dtype, lbm_ctx** out) {
    return lbm_create_flags(nx, ny, Re, U, dtype, 0u, out);
}

extern "C" const char* lbm_last_error(const lbm_ctx* c) {
    if (!c) return g_create_error.c_str();
    return c->err.c_str();
}

extern "C" int lbm_set_stream(lbm_ctx* c, void* stream) {
    if (!c) return LBM_EINVAL;
    int rc = c->sync();
    if (rc) return rc;
    c->stream = (cudaStream_t)stream;
    return LBM_OK;
}

extern "C" int lbm_get_info(const lbm_ctx* c, lbm_info* info) {
    if (!c || !info) return LBM_EINVAL;
    info->nx = c->nx;
    info->ny = c->ny;
    info->pitch = (long)c->pitch;
    info->tau = c->tau;
    info->nu = (c->tau - 0.5) / 3.0;
    info->U = c->U;
    info->Re = info->nu > 0 ? c->U * c->nx / info->nu : 0.0;
    info->dtype = c->dtype;
    info->flags = c->flags;
    info->step = (long)c->step;
    info->device_bytes = c->device_bytes;
    info->launch_config = c->cfg;
    return LBM_OK;
}

extern "C" int lbm_launch_config_count(void) { return kStepConfigs; }

extern "C" int lbm_set_launch_config(lbm_ctx* c, int cfg) {
    if (!c) return LBM_EINVAL;
    if (cfg < 0 || cfg >= kStepConfigs) return c->fail(LBM_EINVAL, fmt("launch config %d out of range", cfg));
    int rc = c->sync();
    if (rc) return rc;
    c->cfg = cfg;
    c->geo = step_geometry(c->dtype, cfg, c->ny, c->pitch);
    c->invalidate_graphs();
    return LBM_OK;
}

extern "C" int lbm_autotune(lbm_ctx* c, int steps_per_trial, int* best, double* best_glups) {
    NvtxRange r("lbm_autotune");
    if (!c || steps_per_trial < 2) return c ? c->fail(LBM_EINVAL, "steps_per_trial < 2") : LBM_EINVAL;
    // trials run on a scratch context of the same shape so the caller's state is untouched
    void* (*sa)(size_t, void*) = g_alloc;
    void (*sr)(void*, void*) = g_release;
    void* su = g_alloc_user;
    g_alloc = c->alloc;
    g_release = c->release;
    g_alloc_user = c->alloc_user;
    lbm_ctx* t = nullptr;
    int rc = lbm_create_ex(c->nx, c->ny, c->tau, c->U, (lbm_dtype)c->dtype, c->flags, &t);
    g_alloc = sa;
    g_release = sr;
    g_alloc_user = su;
    if (rc) return c->fail(rc, std::string("autotune scratch context: ") + lbm_last_error(nullptr));
    t->stream = c->stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    rc = c->cuda(cudaEventCreate(&e0), "event create");
    if (!rc) rc = c->cuda(cudaEventCreate(&e1), "event create");
    // Three rounds over all shapes (drift in clocks or temperature affects every shape alike);
    // each shape's cost is its best plain-step time x 99 plus its best checkpoint-step time, the
    // mix of a 100-step interval.
    cudaEvent_t e2 = nullptr;
    if (!rc) rc = c->cuda(cudaEventCreate(&e2), "event create");
    float plain[kStepConfigs], red[kStepConfigs];
    for (int k = 0; k < kStepConfigs; ++k) plain[k] = red[k] = 1e30f;
    for (int round = 0; round < 3 && !rc; ++round) {
        for (int k = 0; k < kStepConfigs && !rc; ++k) {
            if (round == 0)  // warm-up
                for (int s = 0; s < steps_per_trial && !rc; ++s)
                    rc = c->cuda(launch_step(t->dtype, k, t->step_args(s & 1, s % 98), false, t->stream), "autotune launch");
            if (!rc) rc = c->cuda(cudaEventRecord(e0, t->stream), "event record");
            // steps 0..97 of a checkpoint interval never reduce
            for (int s = 0; s < steps_per_trial && !rc; ++s)
                rc = c->cuda(launch_step(t->dtype, k, t->step_args(s & 1, s % 98), false, t->stream), "autotune launch");
            if (!rc) rc = c->cuda(cudaEventRecord(e1, t->stream), "event record");
            for (int s = 0; s < 2 && !rc; ++s)
                rc = c->cuda(launch_step(t->dtype, k, t->step_args(s & 1, 99), true, t->stream), "autotune launch");
            if (!rc) rc = c->cuda(cudaEventRecord(e2, t->stream), "event record");
            if (!rc) rc = c->cuda(cudaEventSynchronize(e2), "event synchronize");
            float a = 0.f, b = 0.f;
            if (!rc) rc = c->cuda(cudaEventElapsedTime(&a, e0, e1), "event time");
            if (!rc) rc = c->cuda(cudaEventElapsedTime(&b, e1, e2), "event time");
            if (!rc) {
                plain[k] = std::min(plain[k], a / steps_per_trial);
                red[k] = std::min(red[k], b / 2);
            }
        }
    }
    if (e2) cudaEventDestroy(e2);
    int arg = -1;
    float best_ms = 0.f;  // per step, interval mix
    for (int k = 0; k < kStepConfigs && !rc; ++k) {
        const float per_step = (99.f * plain[k] + red[k]) / 100.f;
        if (arg < 0 || per_step < best_ms) {
            arg = k;
            best_ms = per_step;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    lbm_destroy(t);
    if (rc) return rc;
    if (best) *best = arg;
    if (best_glups) *best_glups = (double)c->nx * c->ny / (best_ms * 1e-3) / 1e9;
    return lbm_set_launch_config(c, arg);
}

// ------------------------------------------------------------------ stepping
extern "C" int lbm_step(lbm_ctx* c, long n) {
    if (!c) return LBM_EINVAL;
    NvtxRange r("lbm_step");
    if (n < 0) return c->fail(LBM_EINVAL, "n < 0");
    return c->advance(n);
}

static int read_checkpoint(lbm_ctx* c, long long at, double* r) {
    const DevState& h = c->h_state[(at / kInterval) & 1];
    if (!h.valid || h.at_step != at) return c->fail(LBM_ECUDA, "checkpoint result missing");
    *r = h.residual;
    if (!std::isfinite(h.residual) || !std::isfinite(h.mass))
        return c->fail(LBM_EDIVERGED, fmt("non-finite residual/mass at step %lld", at));
    return LBM_OK;
}

extern "C" int lbm_residual(lbm_ctx* c, double* r) {
    if (!c || !r) return LBM_EINVAL;
    if (c->step < kInterval) return c->fail(LBM_ENOTREADY, "no Eq. 6 residual before step 100");
    int rc = c->sync();
    if (rc) return rc;
    const long long at = c->step / kInterval * kInterval;
    rc = read_checkpoint(c, at, r);
    if (rc == LBM_EDIVERGED) *r = NAN;
    return rc;
}

extern "C" int lbm_run_to_residual(lbm_ctx* c, double tol, long max_steps, long* steps_done) {
    NvtxRange r("lbm_run_to_residual");
    if (!c || max_steps < 0 || !(tol >= 0)) return c ? c->fail(LBM_EINVAL, "bad tol/max_steps") : LBM_EINVAL;
    long long taken = 0;
    int rc = LBM_OK;
    // align to a checkpoint boundary with single steps
    while (c->step % kInterval != 0 && taken < max_steps && !rc) {
        rc = c->advance(1);
        ++taken;
    }
    long long pending = -1;  // checkpoint step whose result is not read yet
    bool converged = false;
    while (!rc && taken + kInterval <= max_steps) {
        rc = c->advance(kInterval);
        if (rc) break;
        taken += kInterval;
        const long long at = c->step;
        rc = c->cuda(cudaEventRecord(c->ev[(at / kInterval) & 1], c->stream), "event record");
        if (rc) break;
        if (pending >= 0) {
            rc = c->cuda(cudaEventSynchronize(c->ev[(pending / kInterval) & 1]), "event synchronize");
            double r = 0;
            if (!rc) rc = read_checkpoint(c, pending, &r);
            if (!rc && r < tol) {
                // converged one chunk ago; the state returned must satisfy it too
                rc = c->cuda(cudaEventSynchronize(c->ev[(at / kInterval) & 1]), "event synchronize");
                if (!rc) rc = read_checkpoint(c, at, &r);
                if (!rc && r < tol) {
                    converged = true;
                    break;
                }
            }
        }
        pending = at;
    }
    if (!rc && !converged) {
        long long rest = max_steps - taken;
        if (rest > 0) {
            rc = c->advance(rest);
            taken += rest;
        }
        if (!rc && pending >= 0) {
            rc = c->sync();
            double r = 0;
            if (!rc) rc = read_checkpoint(c, pending, &r);
            if (!rc && r < tol) converged = true;
        }
    }
    if (steps_done) *steps_done = (long)taken;
    if (rc) return rc;
    if (!converged) return c->fail(LBM_ENOTREADY, "max_steps reached before the residual fell below tol");
    return LBM_OK;
}

// ------------------------------------------------------------------ fields
extern "C" int lbm_mass(lbm_ctx* c, double* m) {
    if (!c || !m) return LBM_EINVAL;
    int rc = c->cuda(launch_mass(c->dtype, c->cur(), c->partials, c->npartials, c->d_state, c->stream), "mass launch");
    if (!rc) rc = c->cuda(cudaMemcpyAsync(&c->h_state[0].scalar, &c->d_state->scalar, sizeof(double), cudaMemcpyDeviceToHost, c->stream), "mass copy");
    if (!rc) rc = c->sync();
    if (rc) return rc;
    *m = c->h_state[0].scalar;
    if (!std::isfinite(*m)) return c->fail(LBM_EDIVERGED, "non-finite mass");
    return LBM_OK;
}

extern "C" int lbm_moments(lbm_ctx* c, double* rho, double* ux, double* uy) {
    if (!c) return LBM_EINVAL;
    const size_t n = (size_t)c->nx * c->ny, bytes = n * sizeof(double);
    double* outs[3] = {rho, ux, uy};
    double* dv[3] = {nullptr, nullptr, nullptr};
    double* mapped[3] = {nullptr, nullptr, nullptr};
    bool st[3] = {false, false, false};
    size_t need = 0;
    bool host = false;
    for (int i = 0; i < 3; ++i)
        if (outs[i]) {
            cudaPointerAttributes at{};
            cudaError_t e = cudaPointerGetAttributes(&at, outs[i]);
            if (e != cudaSuccess) cudaGetLastError();
            if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged))) {
                host = true;
                mapped[i] = lbm_ctx::mapped_host(outs[i]);
                if (!mapped[i]) need += bytes;
            }
        }
    int rc = c->ensure_stage(need);
    if (rc) return rc;
    size_t off = 0;
    for (int i = 0; i < 3; ++i)
        if (outs[i] && mapped[i]) {
            dv[i] = mapped[i];
        } else if (outs[i]) {
            dv[i] = c->device_view(outs[i], bytes, off, &st[i]);
            if (st[i]) off += bytes;
        }
    rc = c->cuda(launch_moments(c->dtype, c->cur(), dv[0], dv[1], dv[2], c->stream), "moments launch");
    for (int i = 0; i < 3 && !rc; ++i)
        if (outs[i] && st[i])
            rc = c->cuda(cudaMemcpyAsync(outs[i], dv[i], bytes, cudaMemcpyDeviceToHost, c->stream), "moments copy");
    if (!rc && host) rc = c->sync();
    return rc;
}

extern "C" int lbm_set_moments(lbm_ctx* c, const double* rho, const double* ux, const double* uy) {
    return lbm_set_moments_ex(c, rho, ux, uy, 0);
}

extern "C" int lbm_set_moments_ex(lbm_ctx* c, const double* rho, const double* ux, const double* uy, int flags) {
    if (!c || !rho || !ux || !uy) return c ? c->fail(LBM_EINVAL, "NULL field") : LBM_EINVAL;
    if (flags & ~LBM_INIT_NEQ) return c->fail(LBM_EINVAL, "unknown lbm_set_moments_ex flag");
    const size_t bytes = (size_t)c->nx * c->ny * sizeof(double);
    const double* ins[3] = {rho, ux, uy};
    double* mapped[3];
    size_t need = 0;
    for (int i = 0; i < 3; ++i) {
        mapped[i] = lbm_ctx::mapped_host(ins[i]);
        cudaPointerAttributes at{};
        const cudaError_t e = cudaPointerGetAttributes(&at, ins[i]);
        if (e != cudaSuccess) cudaGetLastError();
        const bool dev = e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged);
        if (!dev && !mapped[i]) need += bytes;
    }
    int rc = c->ensure_stage(need);
    if (rc) return rc;
    double* dv[3];
    size_t off = 0;
    bool host = false;  // a host buffer the caller may reuse once this returns
    for (int i = 0; i < 3 && !rc; ++i) {
        if (mapped[i]) {
            dv[i] = mapped[i];
            host = true;
            continue;
        }
        bool staged = false;
        dv[i] = c->device_view(ins[i], bytes, off, &staged);
        if (staged) {
            rc = c->cuda(cudaMemcpyAsync(dv[i], ins[i], bytes, cudaMemcpyHostToDevice, c->stream), "moments upload");
            off += bytes;
            host = true;
        }
    }
    if (rc) return rc;
    c->step = 0;
    // the captured 100-step graphs hold the probe set by value and nothing else that this call
    // changes (the step counter picks a graph, the state lives in device memory): keep them unless
    // a probe's start step moves, so that re-seeding the field every 100 steps costs no capture
    bool probes_moved = false;
    for (int q = 0; q < c->probes.n; ++q) {
        probes_moved |= c->probes.start[q] != 0;
        c->probes.start[q] = 0;
    }
    if (probes_moved) c->invalidate_graphs();
    // the state reset comes first: the LBM_Q16S populations are stored against its reference density
    rc = c->cuda(cudaMemsetAsync(c->d_state, 0, sizeof(DevState), c->stream), "state reset");
    if (!rc)
        rc = c->cuda(launch_set_moments(c->dtype, c->cur(), dv[0], dv[1], dv[2], c->snap,
                                        (flags & LBM_INIT_NEQ) ? c->tau : 0.0, c->stream), "set_moments launch");
    if (!rc && host) rc = c->sync();  // the host input may be reused after return
    return rc;
}

extern "C" int lbm_get_populations(lbm_ctx* c, double* f) {
    if (!c || !f) return c ? c->fail(LBM_EINVAL, "NULL buffer") : LBM_EINVAL;
    const size_t bytes = 9ull * c->nx * c->ny * sizeof(double);
    bool staged = false;
    double* dv = c->device_view(f, bytes, 0, &staged);
    if (staged) {
        int rc = c->ensure_stage(bytes);
        if (rc) return rc;
        dv = c->device_view(f, bytes, 0, &staged);
    }
    int rc = c->cuda(launch_get_populations(c->dtype, c->cur(), dv, c->stream), "get_populations launch");
    if (!rc && staged) rc = c->cuda(cudaMemcpyAsync(f, dv, bytes, cudaMemcpyDeviceToHost, c->stream), "populations copy");
    if (!rc && staged) rc = c->sync();
    return rc;
}

extern "C" int lbm_set_populations(lbm_ctx* c, const double* f) {
    if (!c || !f) return c ? c->fail(LBM_EINVAL, "NULL buffer") : LBM_EINVAL;
    const size_t bytes = 9ull * c->nx * c->ny * sizeof(double);
    bool staged = false;
    double* dv = c->device_view(f, bytes, 0, &staged);
    int rc = LBM_OK;
    if (staged) {
        rc = c->ensure_stage(bytes);
        if (rc) return rc;
        dv = c->device_view(f, bytes, 0, &staged);
        rc = c->cuda(cudaMemcpyAsync(dv, f, bytes, cudaMemcpyHostToDevice, c->stream), "populations upload");
    }
    if (!rc) rc = c->cuda(launch_set_populations(c->dtype, c->cur(), dv, c->stream), "set_populations launch");
    if (!rc && staged) rc = c->sync();
    return rc;
}

extern "C" int lbm_stream_function_window(lbm_ctx* c, int i0, int i1, int j0, int j1, double* vmin,
                                          int* imin, int* jmin, double* vmax, int* imax, int* jmax) {
    if (!c) return LBM_EINVAL;
    i0 = i0 < 0 ? 0 : i0;
    j0 = j0 < 0 ? 0 : j0;
    i1 = i1 > c->nx ? c->nx : i1;
    j1 = j1 > c->ny ? c->ny : j1;
    if (i0 >= i1 || j0 >= j1) return c->fail(LBM_EINVAL, "empty window");
    int rc = c->cuda(launch_stream_function(c->dtype, c->cur(), nullptr, i0, i1, j0, j1, c->psi_scratch, c->d_state, c->stream), "stream function launch");
    if (!rc) rc = c->cuda(cudaMemcpyAsync(c->h_state[0].ext, c->d_state->ext, sizeof(c->h_state[0].ext), cudaMemcpyDeviceToHost, c->stream), "extrema copy");
    if (!rc) rc = c->sync();
    if (rc) return rc;
    const double* e = c->h_state[0].ext;
    if (vmin) *vmin = e[0];
    if (imin) *imin = (int)e[1];
    if (jmin) *jmin = (int)e[2];
    if (vmax) *vmax = e[3];
    if (imax) *imax = (int)e[4];
    if (jmax) *jmax = (int)e[5];
    if (!std::isfinite(e[0]) || !std::isfinite(e[3])) return c->fail(LBM_EDIVERGED, "non-finite stream function");
    return LBM_OK;
}

extern "C" int lbm_stream_function(lbm_ctx* c, double* psi, double* psi_min, double* xc, double* yc) {
    NvtxRange r("lbm_stream_function");
    if (!c) return LBM_EINVAL;
    const size_t bytes = (size_t)c->nx * c->ny * sizeof(double);
    double* dv = nullptr;
    bool staged = false;
    int rc = LBM_OK;
    if (psi) {
        dv = c->device_view(psi, bytes, 0, &staged);
        if (staged) {
            if ((rc = c->ensure_stage(bytes))) return rc;
            dv = c->device_view(psi, bytes, 0, &staged);
        }
    }
    rc = c->cuda(launch_stream_function(c->dtype, c->cur(), dv, 0, c->nx, 0, c->ny, c->psi_scratch, c->d_state, c->stream), "stream function launch");
    if (!rc && staged) rc = c->cuda(cudaMemcpyAsync(psi, dv, bytes, cudaMemcpyDeviceToHost, c->stream), "psi copy");
    if (!rc) rc = c->cuda(cudaMemcpyAsync(c->h_state[0].ext, c->d_state->ext, sizeof(c->h_state[0].ext), cudaMemcpyDeviceToHost, c->stream), "extrema copy");
    if (!rc) rc = c->sync();
    if (rc) return rc;
    const double* e = c->h_state[0].ext;
    if (psi_min) *psi_min = e[0];
    if (xc) *xc = e[1] / c->nx;
    if (yc) *yc = e[2] / c->nx;
    if (!std::isfinite(e[0])) return c->fail(LBM_EDIVERGED, "non-finite stream function");
    return LBM_OK;
}

// ------------------------------------------------------------------ probes
extern "C" int lbm_probe(lbm_ctx* c, double x, double y, int every, double* dev_series, long cap) {
    if (!c) return -LBM_EINVAL;
    if (every < 1 || cap < 1 || !dev_series) return -c->fail(LBM_EINVAL, "probe needs every >= 1, cap >= 1 and a buffer");
    if (c->probes.n >= kMaxProbes) return -c->fail(LBM_EINVAL, "too many probes");
    cudaPointerAttributes at{};
    cudaError_t e = cudaPointerGetAttributes(&at, dev_series);
    if (e != cudaSuccess) cudaGetLastError();
    if (!(e == cudaSuccess && (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)))
        return -c->fail(LBM_EINVAL, "probe series must be device memory");
    int px = (int)std::floor(x * c->nx + 0.5), py = (int)std::floor(y * c->nx + 0.5);
    px = px < 0 ? 0 : (px >= c->nx ? c->nx - 1 : px);
    py = py < 0 ? 0 : (py >= c->ny ? c->ny - 1 : py);
    const int q = c->probes.n;
    c->probes.px[q] = px;
    c->probes.py[q] = py;
    c->probes.every[q] = every;
    c->probes.start[q] = c->step;
    c->probes.cap[q] = cap;
    c->probes.series[q] = dev_series;
    c->probes.n = q + 1;
    c->invalidate_graphs();
    return q;
}

extern "C" int lbm_probe_count(lbm_ctx* c, int p, long* n) {
    if (!c || !n || p < 0 || p >= c->probes.n) return c ? c->fail(LBM_EINVAL, "no such probe") : LBM_EINVAL;
    const long long ev = c->probes.every[p];
    *n = (long)(c->step / ev - c->probes.start[p] / ev);
    return LBM_OK;
}

extern "C" int lbm_probe_clear(lbm_ctx* c) {
    if (!c) return LBM_EINVAL;
    int rc = c->sync();
    c->probes = ProbeSet{};
    c->invalidate_graphs();
    return rc;
}

// ------------------------------------------------------------------ checkpoint files
namespace {
struct FileHeader {
    char magic[8];
    uint32_t version;
    int32_t nx, ny, dtype;
    uint32_t flags, pad;
    double tau, U;
    int64_t step;
};
const char kMagic[8] = {'L', 'B', 'M', 'D', '2', 'Q', '9', 0};
}  // namespace

extern "C" int lbm_save(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    const size_t es = storage_bytes(c->dtype);
    const size_t row = (size_t)c->nx * es;
    const size_t pop_bytes = 9ull * c->ny * row;
    const size_t ab = (size_t)arith_bytes(c->dtype);
    const size_t snap_bytes = 2ull * c->ny * c->nx * ab;
    char* host = (char*)malloc(pop_bytes + snap_bytes + sizeof(DevState));
    if (!host) return c->fail(LBM_ENOMEM, "host buffer for checkpoint");
    int rc = c->cuda(cudaMemcpy2DAsync(host, row, c->buf[c->step & 1], (size_t)c->pitch * es, row,
                                       9ull * c->ny, cudaMemcpyDeviceToHost, c->stream), "population copy");
    if (!rc) rc = c->cuda(cudaMemcpy2DAsync(host + pop_bytes, c->nx * ab, c->snap, (size_t)c->pitch * ab,
                                            c->nx * ab, 2ull * c->ny, cudaMemcpyDeviceToHost, c->stream), "snapshot copy");
    if (!rc) rc = c->cuda(cudaMemcpyAsync(host + pop_bytes + snap_bytes, c->d_state, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream), "state copy");
    if (!rc) rc = c->sync();
    if (rc) {
        free(host);
        return rc;
    }
    FileHeader h{};
    memcpy(h.magic, kMagic, 8);
    h.version = 2;
    h.nx = c->nx;
    h.ny = c->ny;
    h.dtype = c->dtype;
    h.flags = c->flags;
    h.tau = c->tau;
    h.U = c->U;
    h.step = c->step;
    FILE* fp = fopen(path, "wb");
    bool ok = fp && fwrite(&h, sizeof h, 1, fp) == 1 &&
              fwrite(host, 1, pop_bytes + snap_bytes + sizeof(DevState), fp) == pop_bytes + snap_bytes + sizeof(DevState);
    if (fp && fclose(fp) != 0) ok = false;
    free(host);
    return ok ? LBM_OK : c->fail(LBM_EIO, fmt("cannot write %s", path));
}

extern "C" int lbm_load(lbm_ctx* c, const char* path) {
    if (!c || !path) return LBM_EINVAL;
    FILE* fp = fopen(path, "rb");
    if (!fp) return c->fail(LBM_EIO, fmt("cannot open %s", path));
    FileHeader h{};
    if (fread(&h, sizeof h, 1, fp) != 1 || memcmp(h.magic, kMagic, 8) != 0 || h.version != 2) {
        fclose(fp);
        return c->fail(LBM_EIO, "not a checkpoint of this library");
    }
    if (h.nx != c->nx || h.ny != c->ny || h.dtype != c->dtype) {
        fclose(fp);
        return c->fail(LBM_EIO, fmt("checkpoint is %d x %d dtype %d, context is %d x %d dtype %d", h.nx, h.ny, h.dtype, c->nx, c->ny, c->dtype));
    }
    const size_t es = storage_bytes(c->dtype);
    const size_t row = (size_t)c->nx * es;
    const size_t pop_bytes = 9ull * c->ny * row;
    const size_t ab = (size_t)arith_bytes(c->dtype);
    const size_t snap_bytes = 2ull * c->ny * c->nx * ab;
    const size_t total = pop_bytes + snap_bytes + sizeof(DevState);
    char* host = (char*)malloc(total);
    if (!host) {
        fclose(fp);
        return c->fail(LBM_ENOMEM, "host buffer for checkpoint");
    }
    const bool ok = fread(host, 1, total, fp) == total;
    fclose(fp);
    if (!ok) {
        free(host);
        return c->fail(LBM_EIO, "truncated checkpoint");
    }
    int rc = c->sync();
    c->tau = h.tau;
    c->U = h.U;
    c->flags = h.flags;
    c->step = h.step;
    for (int q = 0; q < c->probes.n; ++q) c->probes.start[q] = c->step;
    c->invalidate_graphs();
    if (!rc) rc = c->cuda(cudaMemcpy2DAsync(c->buf[c->step & 1], (size_t)c->pitch * es, host, row, row, 9ull * c->ny, cudaMemcpyHostToDevice, c->stream), "population upload");
    if (!rc) rc = c->cuda(cudaMemcpy2DAsync(c->snap, (size_t)c->pitch * ab, host + pop_bytes, c->nx * ab, c->nx * ab, 2ull * c->ny, cudaMemcpyHostToDevice, c->stream), "snapshot upload");
    if (!rc) rc = c->cuda(cudaMemcpyAsync(c->d_state, host + pop_bytes + snap_bytes, sizeof(DevState), cudaMemcpyHostToDevice, c->stream), "state upload");
    if (!rc) {
        // refresh the host mirror of the last checkpoint so lbm_residual works right away
        const DevState* s = (const DevState*)(host + pop_bytes + snap_bytes);
        if (s->valid) c->h_state[(s->at_step / kInterval) & 1] = *s;
    }
    if (!rc) rc = c->sync();
    free(host);
    return rc;
}
