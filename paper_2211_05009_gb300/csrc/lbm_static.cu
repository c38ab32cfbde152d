// lbm_static.cu -- lbm_stream_function_static: the stream-function post-processing of a caller's
// velocity field with no device allocation at all.
//
// Why it exists: some callers cannot call cudaMalloc -- for example a solver embedded in a larger
// application that reserves its whole device-memory budget at start-up and forbids later
// allocations.
// lbm_stream_function needs a context (which owns scratch memory); this variant takes the u_x
// field and the outputs from the caller and keeps its small scratch (column-segment sums and block
// extrema) in a fixed device array that lives as long as the library is loaded.
//
// The arithmetic is that of lbm_stream_function: Psi = 0 on the bottom wall, u_x = dPsi/dy, the
// trapezoid rule in y with dy = 1, FP64 sums; the minimum of Psi and its node.
#include <mutex>

#include "lbm.h"
#include "lbm_device.cuh"

namespace {

constexpr int kCols = 128;  // columns per block
constexpr int kSeg = 32;    // rows per column segment

// Scratch for every call in this process: segment sums [nseg][nx] then 2 doubles per block.
// Its size bounds the grids this entry point accepts (LBM_STATIC_SCRATCH_DOUBLES in lbm.h).
static __device__ __align__(256) double g_psi_scratch[LBM_STATIC_SCRATCH_DOUBLES];

std::mutex g_setup_mutex;
constexpr int kMaxDevices = 64;
double* g_scratch_addr[kMaxDevices] = {};  // device address of g_psi_scratch, per device

__global__ void __launch_bounds__(kCols) k_static_seg(const double* __restrict__ ux, int nx, int ny,
                                                      double* segsum) {
    const int x = blockIdx.x * kCols + threadIdx.x;
    const int seg = blockIdx.y;
    if (x >= nx) return;
    const int y0 = seg * kSeg, y1 = min(ny, y0 + kSeg);
    double s = 0.0;
    for (int y = y0; y < y1; ++y) s += ux[(long long)y * nx + x];
    segsum[(long long)seg * nx + x] = s;
}

__global__ void __launch_bounds__(kCols) k_static_walk(const double* __restrict__ ux, int nx, int ny,
                                                       const double* __restrict__ segsum, double* psi,
                                                       double* part) {
    __shared__ double vmin[kCols];
    __shared__ long long imin[kCols];
    const int x = blockIdx.x * kCols + threadIdx.x;
    const int seg = blockIdx.y;
    double bv = 0.0;
    long long bi = -1;
    if (x < nx) {
        double run = 0.0;
        for (int k = 0; k < seg; ++k) run += segsum[(long long)k * nx + x];
        const double u0 = ux[x];
        const int y0 = seg * kSeg, y1 = min(ny, y0 + kSeg);
        for (int y = y0; y < y1; ++y) {
            const double u = ux[(long long)y * nx + x];
            run += u;
            const double p = y == 0 ? 0.0 : run - 0.5 * u0 - 0.5 * u;
            if (psi) psi[(long long)y * nx + x] = p;
            if (bi < 0 || p < bv) {
                bv = p;
                bi = (long long)y * nx + x;
            }
        }
    }
    vmin[threadIdx.x] = bv;
    imin[threadIdx.x] = bi;
    __syncthreads();
    for (int o = kCols / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            const double v = vmin[threadIdx.x + o];
            const long long i = imin[threadIdx.x + o];
            if (i >= 0 && (imin[threadIdx.x] < 0 || v < vmin[threadIdx.x] ||
                           (v == vmin[threadIdx.x] && i < imin[threadIdx.x]))) {
                vmin[threadIdx.x] = v;
                imin[threadIdx.x] = i;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const long long b = (long long)blockIdx.y * gridDim.x + blockIdx.x;
        part[2 * b] = vmin[0];
        part[2 * b + 1] = (double)imin[0];
    }
}

__global__ void k_static_finalize(const double* part, int nblocks, int nx, double* result) {
    if (threadIdx.x != 0) return;
    double bv = 0.0;
    long long bi = -1;
    for (int b = 0; b < nblocks; ++b) {
        const double v = part[2 * b];
        const long long i = (long long)part[2 * b + 1];
        if (i >= 0 && (bi < 0 || v < bv || (v == bv && i < bi))) {
            bv = v;
            bi = i;
        }
    }
    result[0] = bv;
    result[1] = (double)(bi % nx) / nx;
    result[2] = (double)(bi / nx) / nx;
}

// Device address of the scratch array for the current device, looked up once per device.
cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_psi_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<double*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" int lbm_stream_function_static(const double* ux, int nx, int ny, double* psi,
                                          double* result, void* stream) {
    if (!ux || !result || nx < 1 || ny < 1) return LBM_EINVAL;
    const long long nseg = (ny + kSeg - 1) / kSeg;
    const long long ncb = (nx + kCols - 1) / kCols;
    const long long need = nseg * nx + 2 * nseg * ncb;
    if (need > LBM_STATIC_SCRATCH_DOUBLES) return LBM_ETOOBIG;  // grid too large for the fixed scratch
    if (nseg > 65535) return LBM_ETOOBIG;                        // one grid row per segment (gridDim.y)
    // An error pending from someone else's earlier call: report it, launch nothing, leave it set.
    if (cudaPeekAtLastError() != cudaSuccess) return LBM_ECUDA;
    double* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return LBM_ECUDA;
    }
    double* segsum = scratch;
    double* part = scratch + nseg * nx;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const dim3 grid((unsigned)ncb, (unsigned)nseg);
    // from here on a launch error is this call's own: take it (and clear it) after each launch
    k_static_seg<<<grid, kCols, 0, st>>>(ux, nx, ny, segsum);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    k_static_walk<<<grid, kCols, 0, st>>>(ux, nx, ny, segsum, psi, part);
    if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
    k_static_finalize<<<1, 32, 0, st>>>(part, (int)(nseg * ncb), nx, result);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
