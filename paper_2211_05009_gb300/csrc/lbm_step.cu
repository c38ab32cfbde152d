// lbm_step.cu -- dispatch of the fused step kernel over storage types and launch shapes, and
// the fixed-order FP64 reduction that closes each 100-step checkpoint (Eq. 6 residual, mass).
#include <cmath>

#include "lbm_device.cuh"
#include "lbm_internal.h"

namespace lbm {

cudaError_t launch_step_f64(int cfg, const StepArgs& a, bool reduce, cudaStream_t st);
cudaError_t launch_step_f32(int cfg, const StepArgs& a, bool reduce, cudaStream_t st);
cudaError_t launch_step_f32s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st);
cudaError_t launch_step_f16s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st);
cudaError_t launch_step_bf16s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st);
cudaError_t launch_step_q16s(int cfg, const StepArgs& a, bool reduce, cudaStream_t st);

namespace {
struct Shape {
    int R, BY;
};
// must match launch_step_cfg in lbm_step_kernel.cuh
constexpr Shape kShapes[kStepConfigs] = {{2, 2}, {1, 4}, {2, 2}, {4, 1}, {2, 4}, {4, 2}};
}  // namespace

double q16_scale(int j, double U) {
    const double w = j == 0 ? 4.0 / 9.0 : (j < 5 ? 1.0 / 9.0 : 1.0 / 36.0);
    const double K = j == 0 ? 2.0 : (j < 5 ? 5.0 : 5.5);
    const double u = fabs(U) > 0.01 ? fabs(U) : 0.01;
    return 0.5 * exp2(ceil(log2(K * w * u)));  // 2 S_j = the power of two at or above K w u
}

QCodec q16_codec(double U) {
    QCodec q{};
    for (int j = 0; j < 9; ++j) {
        const double S = q16_scale(j, U);
        q.dec[j] = (float)(exp2(124.0) * S);
        q.enc[j] = (float)(exp2(-124.0) / S);
    }
    return q;
}

StepGeometry step_geometry(int dtype, int cfg, int ny, long long pitch) {
    StepGeometry g{};
    const int V = storage_bytes(dtype) == 2 ? 4 : 2;  // as launch_step_cfg
    const Shape s = kShapes[cfg];
    g.grid_x = (int)(pitch / (32 * V));
    g.grid_y = (ny + s.BY * s.R - 1) / (s.BY * s.R);
    g.blocks = g.grid_x * g.grid_y;
    return g;
}

cudaError_t launch_step(int dtype, int cfg, const StepArgs& a, bool reduce, cudaStream_t st) {
    if (cfg < 0 || cfg >= kStepConfigs) return cudaErrorInvalidValue;
    switch (dtype) {
        case 0: return launch_step_f64(cfg, a, reduce, st);
        case 1: return launch_step_f32(cfg, a, reduce, st);
        case 2: return launch_step_f32s(cfg, a, reduce, st);
        case 3: return launch_step_f16s(cfg, a, reduce, st);
        case 4: return launch_step_bf16s(cfg, a, reduce, st);
        case 5: return launch_step_q16s(cfg, a, reduce, st);
        default: return cudaErrorInvalidValue;
    }
}

// Sum the per-block partials in a fixed order and publish the checkpoint (Eq. 6, mass).
__global__ void __launch_bounds__(256) k_finalize_checkpoint(const double* __restrict__ partials,
                                                             int nblocks, double nodes,
                                                             DevState* st) {
    __shared__ double sh[3][256];
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += 256) {
        s0 += partials[3ll * b];
        s1 += partials[3ll * b + 1];
        s2 += partials[3ll * b + 2];
    }
    sh[0][threadIdx.x] = s0;
    sh[1][threadIdx.x] = s1;
    sh[2][threadIdx.x] = s2;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
#pragma unroll
            for (int c = 0; c < 3; ++c) sh[c][threadIdx.x] += sh[c][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        st->num = sh[1][0];
        st->den = sh[2][0];
        st->residual = sqrt(sh[1][0] / sh[2][0]);
        st->mass = nodes + sh[0][0];
        // LBM_Q16S: the checkpoint step stored against rho_ref[1]; the next one stores against
        // the mean density deviation just measured (unused by the other storage types)
        st->rho_ref[0] = st->rho_ref[1];
        if (isfinite(st->mass)) st->rho_ref[1] = st->mass / nodes - 1.0;
        st->base += kInterval;
        st->at_step = st->base;
        st->valid = 1;
    }
}

cudaError_t launch_finalize_checkpoint(const double* partials, int nblocks, double nodes,
                                       DevState* st, cudaStream_t s) {
    k_finalize_checkpoint<<<1, 256, 0, s>>>(partials, nblocks, nodes, st);
    return cudaGetLastError();
}

}  // namespace lbm
