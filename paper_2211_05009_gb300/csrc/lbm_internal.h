// lbm_internal.h -- declarations shared by the translation units of the CUDA library
// (kernel launchers and the per-context state).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>  // header-only; the ranges cost nothing unless a profiler is attached

#include "lbm_device.cuh"

namespace lbm {

// NVTX range over the host side of one library call (named in nsys / ncu timelines).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

struct StepGeometry {
    int grid_x, grid_y, blocks;
};

// Launch shapes of the step kernel (see lbm_step_kernel.cuh); all give identical populations.
constexpr int kStepConfigs = 6;
// Fastest shape per storage type measured on GB300 at 2048 x 2048 (f64, f32, f32s, f16s, bf16s);
// lbm_autotune re-measures on the caller's size.
inline int default_step_config(int dtype) {
    constexpr int k[6] = {1, 4, 0, 2, 2, 2};
    return (dtype >= 0 && dtype < 6) ? k[dtype] : 0;
}

constexpr int kDtypeQ16S = 5;
// LBM_Q16S scale S_j of direction j for lid speed U: the largest code is (2 - 2^-13) S_j, and
// 2 S_j = the power of two at or above K_j w_j max(|U|, 0.01) with K = 2 (rest), 5 (axes),
// 11/2 (diagonals), above the largest deviations met in lid-driven cavities from Re 74 to 8000
// (flat 131 x 13 to 2048^2): |h_j| < 4.5 w_j U (axes), 5.0 w_j U (diagonals), 1.0 w_j U (rest)
// once the mean density is taken out.
double q16_scale(int j, double U);
QCodec q16_codec(double U);

// Geometry of the step launch for a shape (also the number of reduction partials).
StepGeometry step_geometry(int dtype, int cfg, int ny, long long pitch);

// Bytes of the arithmetic type (FP64 for FP64 storage, FP32 otherwise): the Eq. 6 snapshot type.
inline int arith_bytes(int dtype) { return dtype == 0 ? 8 : 4; }

// Row pitch (elements) for a storage type: a multiple of 32 lanes x 16 bytes.
long long row_pitch(int dtype, int nx);
int storage_bytes(int dtype);

cudaError_t launch_step(int dtype, int cfg, const StepArgs& a, bool reduce, cudaStream_t st);
cudaError_t launch_finalize_checkpoint(const double* partials, int nblocks, double nodes,
                                       DevState* st, cudaStream_t s);

struct FieldArgs {
    void* f;  // populations [9][ny][pitch] of the storage type
    int nx, ny;
    long long pitch, plane;
    double U;
    int corner_moving;
    QCodec q;              // LBM_Q16S scales
    const DevState* st;    // LBM_Q16S reference density (rho_ref[0])
};

// f = f^eq(1, u0) with the Sec. 2.2 (i) initial velocity; snapshot = u0.
cudaError_t launch_init(int dtype, const FieldArgs& a, void* snap, cudaStream_t st);
// f = f^eq(rho, u) from dense [ny][nx] FP64 fields; snapshot = u.  neq_tau > 0 adds
// (1 - 1/tau) times the first-order Chapman-Enskog non-equilibrium part (tau = neq_tau).
cudaError_t launch_set_moments(int dtype, const FieldArgs& a, const double* rho, const double* ux,
                               const double* uy, void* snap, double neq_tau, cudaStream_t st);
// Dense [ny][nx] FP64 moments (any output may be null).
cudaError_t launch_moments(int dtype, const FieldArgs& a, double* rho, double* ux, double* uy,
                           cudaStream_t st);
// Dense [9][ny][nx] FP64 populations <-> storage.
cudaError_t launch_get_populations(int dtype, const FieldArgs& a, double* out, cudaStream_t st);
cudaError_t launch_set_populations(int dtype, const FieldArgs& a, const double* in, cudaStream_t st);
// Mass: sum over nodes of (rho - 1) into partials, then N + sum into st->scalar.
cudaError_t launch_mass(int dtype, const FieldArgs& a, double* partials, int max_partials,
                        DevState* state, cudaStream_t st);
// Stream function (u_x = dPsi/dy, trapezoid in y from Psi = 0 at y = 0) with window extrema
// into state->ext; psi (dense [ny][nx]) may be null.  scratch needs psi_scratch_doubles().
size_t psi_scratch_doubles(int nx, int ny);
cudaError_t launch_stream_function(int dtype, const FieldArgs& a, double* psi, int i0, int i1,
                                   int j0, int j1, double* scratch, DevState* state,
                                   cudaStream_t st);

}  // namespace lbm
