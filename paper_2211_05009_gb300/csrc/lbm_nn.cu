// lbm_nn.cu -- the learned warm start: a 5-level convolutional encoder-decoder (U-Net) that maps
// (Re, Ar, a coarse steady field) to an initial fine rho/u field for the cavity solver, with its
// training (forward, backward, Adam) written as CUDA kernels.  Not part of the paper; it serves
// the time-to-steady-state of the method's runs (Eq. 6 criterion) and is measured by it.
//
// Tensors are FP32 [C][H][W] (one sample).  Every 3x3 convolution (zero padding, stride 1) runs as
// im2col + the BF16 tensor-core GEMM of lbm_nn_gemm.cu with FP32 accumulation:
//   forward        Y[co][p]  = sum_k Wq[co][k] Xc[p][k]           (Xc: im2col of X, pixel-major)
//   data grad      dX[ci][p] = sum_k Wf[ci][k] dZc[p][k]          (Wf: flipped, transposed W;
//                                                                   dZc: im2col of dZ)
//   weight grad    dW[co][k] += sum_p dZ[co][p] XcT[k][p]          (XcT: im2col, k-major)
// Operands are rounded to BF16 where they enter the GEMM (weights, im2col columns, dZ); the FP32
// master weights are updated by Adam.  Activation: leaky ReLU (slope 0.1) after every conv but
// the output head.  Down: 2x2 average pool; up: nearest x2; skips by channel concatenation.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "lbm.h"
#include "lbm_internal.h"
#include "lbm_nn_gemm.cuh"

namespace lbm {
namespace nn {

constexpr float kLeak = 0.1f;

__global__ void k_im2col_pk(const float* __restrict__ x1, int c1, const float* __restrict__ x2, int c2,
                            int H, int W, int Kp, __nv_bfloat16* __restrict__ out) {
    // out[p][k], k = ci*9 + ky*3 + kx over the channels of x1 then x2; zeros past C*9 and outside
    const long long P = (long long)H * W;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * Kp) return;
    const int k = (int)(idx % Kp);
    const long long p = idx / Kp;
    const int C = c1 + c2;
    float v = 0.f;
    if (k < C * 9) {
        const int ci = k / 9, r = k % 9, ky = r / 3, kx = r % 3;
        const int y = (int)(p / W) + ky - 1, x = (int)(p % W) + kx - 1;
        if (y >= 0 && y < H && x >= 0 && x < W)
            v = ci < c1 ? x1[((long long)ci * H + y) * W + x] : x2[((long long)(ci - c1) * H + y) * W + x];
    }
    out[idx] = __float2bfloat16_rn(v);
}

__global__ void k_im2col_kp(const float* __restrict__ x1, int c1, const float* __restrict__ x2, int c2,
                            int H, int W, int Kp, __nv_bfloat16* __restrict__ out) {
    // out[k][p]
    const long long P = (long long)H * W;
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= P * Kp) return;
    const long long p = idx % P;
    const int k = (int)(idx / P);
    const int C = c1 + c2;
    float v = 0.f;
    if (k < C * 9) {
        const int ci = k / 9, r = k % 9, ky = r / 3, kx = r % 3;
        const int y = (int)(p / W) + ky - 1, x = (int)(p % W) + kx - 1;
        if (y >= 0 && y < H && x >= 0 && x < W)
            v = ci < c1 ? x1[((long long)ci * H + y) * W + x] : x2[((long long)(ci - c1) * H + y) * W + x];
    }
    out[idx] = __float2bfloat16_rn(v);
}

__global__ void k_to_bf16(const float* __restrict__ x, long long n, __nv_bfloat16* __restrict__ y) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) y[i] = __float2bfloat16_rn(x[i]);
}

// wq[co][Kp] = w[co][k] (k < ci*9), wf[ci][Kp2] with wf[ci][co*9 + (8 - r)] = w[co][ci*9 + r]
__global__ void k_prep_weights(const float* __restrict__ w, int ci, int co, int Kp, int Kp2,
                               __nv_bfloat16* __restrict__ wq, __nv_bfloat16* __restrict__ wf) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < co * Kp) {
        const int o = idx / Kp, k = idx % Kp;
        wq[idx] = __float2bfloat16_rn(k < ci * 9 ? w[o * ci * 9 + k] : 0.f);
    }
    if (idx < ci * Kp2) {
        const int i = idx / Kp2, k = idx % Kp2;
        float v = 0.f;
        if (k < co * 9) {
            const int o = k / 9, r = 8 - k % 9;
            v = w[(o * ci + i) * 9 + r];
        }
        wf[idx] = __float2bfloat16_rn(v);
    }
}

__global__ void k_bias_act(float* __restrict__ y, const float* __restrict__ b, int C, long long P, int act) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)C * P) return;
    float v = y[i] + b[i / P];
    if (act && v < 0.f) v *= kLeak;
    y[i] = v;
}

// dz = dy * act'(y) (y is the activated output), and db[c] += sum_p dz (one block per channel)
__global__ void k_act_back(const float* __restrict__ y, const float* __restrict__ dy, float* __restrict__ dz,
                           float* __restrict__ db, long long P, int act) {
    __shared__ float sh[256];
    const int c = blockIdx.x;
    float s = 0.f;
    for (long long p = threadIdx.x; p < P; p += blockDim.x) {
        const long long i = (long long)c * P + p;
        float g = dy[i];
        if (act && y[i] <= 0.f) g *= kLeak;
        dz[i] = g;
        s += g;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) db[c] += sh[0];
}

__global__ void k_pool2(const float* __restrict__ x, int C, int H, int W, float* __restrict__ y) {
    const int h = H / 2, w = W / 2;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)C * h * w) return;
    const int xx = (int)(i % w), yy = (int)((i / w) % h), c = (int)(i / ((long long)w * h));
    const float* s = x + ((long long)c * H + 2 * yy) * W + 2 * xx;
    y[i] = 0.25f * ((s[0] + s[1]) + (s[W] + s[W + 1]));
}

__global__ void k_pool2_back(const float* __restrict__ dy, int C, int H, int W, float* __restrict__ dx) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)C * H * W) return;
    const int xx = (int)(i % W), yy = (int)((i / W) % H), c = (int)(i / ((long long)W * H));
    dx[i] += 0.25f * dy[((long long)c * (H / 2) + yy / 2) * (W / 2) + xx / 2];
}

__global__ void k_up2(const float* __restrict__ x, int C, int h, int w, float* __restrict__ y) {
    const int H = 2 * h, W = 2 * w;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)C * H * W) return;
    const int xx = (int)(i % W), yy = (int)((i / W) % H), c = (int)(i / ((long long)W * H));
    y[i] = x[((long long)c * h + yy / 2) * w + xx / 2];
}

__global__ void k_up2_back(const float* __restrict__ dy, int C, int h, int w, float* __restrict__ dx) {
    const int W = 2 * w;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)C * h * w) return;
    const int xx = (int)(i % w), yy = (int)((i / w) % h), c = (int)(i / ((long long)w * h));
    const float* s = dy + ((long long)c * 2 * h + 2 * yy) * W + 2 * xx;
    dx[i] += (s[0] + s[1]) + (s[W] + s[W + 1]);
}

// Number of valid pixels (mask is 0/1) into cnt[0].
// stats[0] = sum mask (the count n); stats[2] = sum mask (base + out - target)_0 / n, the mean
// density-channel error, which the loss ignores (one block, fixed order).
__global__ void k_mask_stats(const float* __restrict__ mask, const float* __restrict__ out, const float* __restrict__ base,
                             const float* __restrict__ tgt, long long P, double* stats) {
    __shared__ double sh[2][256];
    double s = 0.0, e = 0.0;
    for (long long i = threadIdx.x; i < P; i += blockDim.x) {
        s += mask[i];
        e += (double)(mask[i] * (base[i] + out[i] - tgt[i]));
    }
    sh[0][threadIdx.x] = s;
    sh[1][threadIdx.x] = e;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + o];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        stats[0] = sh[0][0];
        stats[2] = sh[0][0] > 0.0 ? sh[1][0] / sh[0][0] : 0.0;
    }
}

// loss = sum mask (e - [c = 0] mean_0)^2 / (3 n), e = base + out - target per channel c: the
// density channel is compared up to a constant (the level of a steady density field only records
// how long the wall scheme's mass loss acted; a uniform offset does not change the flow).
// dout = d loss / d out (the mean's own derivative cancels).  Partial sums per block.
__global__ void k_mse(const float* __restrict__ out, const float* __restrict__ base, const float* __restrict__ tgt,
                      const float* __restrict__ mask, long long P, const double* __restrict__ stats,
                      float* __restrict__ dout, double* __restrict__ part) {
    __shared__ double sh[256];
    const float inv_n = (float)(1.0 / (3.0 * stats[0]));
    const float mean0 = (float)stats[2];
    double s = 0.0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < 3 * P; i += (long long)gridDim.x * blockDim.x) {
        const float m = mask[i % P];
        const float d = m * (base[i] + out[i] - tgt[i] - (i < P ? mean0 : 0.f));
        dout[i] = 2.f * d * inv_n;
        s += (double)d * d;
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int o = 128; o > 0; o >>= 1) {
        if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}

// loss[1] = sum(part) / (3 loss[0])
__global__ void k_sum_parts(const double* part, int n, double* loss) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += part[i];
    loss[1] = s / (3.0 * loss[0]);
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2, float gscale) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i] * gscale;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
}

// ------------------------------------------------------------------ warm-start glue
// in[7][H][W]: bilinear image of the coarse field on the fine grid (rho-1 scaled, u/U), Re/4000,
// Ar/2, wall mask, valid-row mask; rows ny..H-1 are padding (all channels 0).
__global__ void k_warm_input(const double* __restrict__ rc, const double* __restrict__ uxc,
                             const double* __restrict__ uyc, int nxc, int nyc, float re_s, float ar_s,
                             float inv_u, float rho_s, int nx, int ny, int H, float* __restrict__ in) {
    const long long P = (long long)H * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int x = (int)(p % nx), y = (int)(p / nx);
    float v[7] = {0, 0, 0, 0, 0, 0, 0};
    if (y < ny) {
        // node-to-node map of the wall-inclusive grids: fine node i sits at i (nxc-1)/(nx-1)
        const float fx = x * (float)(nxc - 1) / (float)(nx - 1);
        const float fy = y * (float)(nyc - 1) / (float)(ny - 1);
        const int x0 = min((int)fx, nxc - 2), y0 = min((int)fy, nyc - 2);
        const float ax = fx - x0, ay = fy - y0;
        auto bil = [&](const double* f) {
            const double a = f[(long long)y0 * nxc + x0], b = f[(long long)y0 * nxc + x0 + 1];
            const double c = f[(long long)(y0 + 1) * nxc + x0], d = f[(long long)(y0 + 1) * nxc + x0 + 1];
            return (float)((1 - ay) * ((1 - ax) * a + ax * b) + ay * ((1 - ax) * c + ax * d));
        };
        v[0] = (bil(rc) - 1.f) * rho_s;
        v[1] = bil(uxc) * inv_u;
        v[2] = bil(uyc) * inv_u;
        v[3] = re_s;
        v[4] = ar_s;
        v[5] = (x == 0 || x == nx - 1 || y == 0 || y == ny - 1) ? 1.f : 0.f;
        v[6] = 1.f;
    }
    for (int c = 0; c < 7; ++c) in[c * P + p] = v[c];
}

// rho, u fields [ny][nx] from the network output plus its base (input channels 0..2)
__global__ void k_warm_output(const float* __restrict__ in, const float* __restrict__ out, int nx, int ny,
                              int H, float U, float rho_s, double* __restrict__ rho, double* __restrict__ ux,
                              double* __restrict__ uy) {
    const long long P = (long long)H * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= (long long)nx * ny) return;
    rho[p] = 1.0 + (double)(in[p] + out[p]) / rho_s;
    ux[p] = (double)(in[P + p] + out[P + p]) * U;
    uy[p] = (double)(in[2 * P + p] + out[2 * P + p]) * U;
}

// one 3x3 box-filter pass over the three correction channels, rows [0, ny) only, the
// neighbourhood clamped to the valid rows and columns (replicate edges)
__global__ void k_warm_smooth(const float* __restrict__ in, float* __restrict__ out, int ny, int H, int W) {
    const long long P = (long long)H * W;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= 3 * P) return;
    const int c = (int)(p / P), y = (int)((p % P) / W), x = (int)(p % W);
    if (y >= ny) {
        out[p] = in[p];
        return;
    }
    const float* ch = in + (long long)c * P;
    float s = 0.f;
    for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
            const int yy = min(max(y + dy, 0), ny - 1), xx = min(max(x + dx, 0), W - 1);
            s += ch[(long long)yy * W + xx];
        }
    out[p] = s * (1.f / 9.f);
}

// training target: scaled fine fields, zero padding rows
__global__ void k_warm_target(const double* __restrict__ rho, const double* __restrict__ ux, const double* __restrict__ uy,
                              int nx, int ny, int H, double inv_u, float rho_s, float* __restrict__ t) {
    const long long P = (long long)H * nx;
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const bool in = p < (long long)nx * ny;
    t[p] = in ? (float)((rho[p] - 1.0) * rho_s) : 0.f;
    t[P + p] = in ? (float)(ux[p] * inv_u) : 0.f;
    t[2 * P + p] = in ? (float)(uy[p] * inv_u) : 0.f;
}

}  // namespace nn
}  // namespace lbm

using namespace lbm;
using namespace lbm::nn;

namespace {
std::string nfmt(const char* f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}
thread_local std::string g_net_create_error;
inline int pad8(int k) { return (k + 7) / 8 * 8; }
inline unsigned nblk(long long n, int t = 256) { return (unsigned)((n + t - 1) / t); }
}  // namespace

struct ConvSpec {
    int ci, co, act;
    long long woff, boff;  // offsets into the flat parameter vector
    int Kp, Kp2;
    long long wq_off, wf_off;  // offsets into the BF16 weight arrays
};

struct lbm_net {
    int width = 0;
    int ch[5];
    std::vector<ConvSpec> convs;
    long long nparams = 0, nwq = 0, nwf = 0;
    float *params = nullptr, *grads = nullptr, *adam_m = nullptr, *adam_v = nullptr;
    __nv_bfloat16 *wq = nullptr, *wf = nullptr;
    long long adam_t = 0;
    bool weights_dirty = true;
    // activations and gradients for one sample size
    int H = 0, W = 0;
    std::vector<float*> act, gact;  // per tensor
    std::vector<long long> act_size;
    __nv_bfloat16* col = nullptr;  // im2col scratch (backend 3: the channels-last BF16 input)
    long long col_elems = 0;
    __nv_bfloat16* wtap = nullptr;  // backend 3: the current conv's weights, tap-major
    float* dz = nullptr;            // dZ scratch (largest tensor)
    __nv_bfloat16* dzq = nullptr;   // dZ in BF16
    double* parts = nullptr;
    double* d_loss = nullptr;
    double* h_loss = nullptr;
    int* d_err = nullptr;          // set by a tcgen05 GEMM whose bounded wait ran out
    int backend = 3;  // 0: mma.sync GEMM, 1: im2col + tcgen05 GEMM, 2: tcgen05 implicit conv (gather),
                      // 3: tcgen05 implicit conv (channels-last input, TMA boxes); the weight gradient
                      // always takes the explicit k-major im2col
    cudaStream_t stream = nullptr;
    std::string err;

    int fail(int code, const std::string& m) {
        err = m;
        return code;
    }
    int cuda(cudaError_t e, const char* what) {
        if (e == cudaSuccess) return LBM_OK;
        err = nfmt("%s: %s", what, cudaGetErrorString(e));
        return e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
    }
};

namespace {

// Tensor ids of the graph (one sample):
//   0 input(7, L0) | enc: a_l, e_l (l = 0..4), p_l (l = 1..4) | dec: u_l, b_l, d_l (l = 3..0) | out
// Sizes depend on the level.  The table below lists (channels, level) per tensor.
struct TensorSpec {
    int c, level;
};

struct Graph {
    std::vector<TensorSpec> t;
    int input, out;
    int a[5], e[5], p[5], u[4], b[4], d[4];
};

Graph make_graph(const int* ch) {
    Graph g;
    auto add = [&](int c, int lvl) {
        g.t.push_back({c, lvl});
        return (int)g.t.size() - 1;
    };
    g.input = add(7, 0);
    for (int l = 0; l < 5; ++l) {
        g.p[l] = l ? add(ch[l - 1], l) : -1;
        g.a[l] = add(ch[l], l);
        g.e[l] = add(ch[l], l);
    }
    for (int l = 3; l >= 0; --l) {
        g.u[l] = add(ch[l + 1], l);
        g.b[l] = add(ch[l], l);
        g.d[l] = add(ch[l], l);
    }
    g.out = add(3, 0);
    return g;
}

// The 19 convolutions in graph order: enc a_l, e_l (l = 0..4); dec b_l, d_l (l = 3..0); head.
void conv_list(const int* ch, std::vector<std::pair<int, int>>& io) {
    io.clear();
    int prev = 7;
    for (int l = 0; l < 5; ++l) {
        io.push_back({prev, ch[l]});
        io.push_back({ch[l], ch[l]});
        prev = ch[l];
    }
    for (int l = 3; l >= 0; --l) {
        io.push_back({ch[l + 1] + ch[l], ch[l]});
        io.push_back({ch[l], ch[l]});
    }
    io.push_back({ch[0], 3});
}

int ensure_buffers(lbm_net* n, int H, int W) {
    if (n->H == H && n->W == W) return LBM_OK;
    cudaStreamSynchronize(n->stream);
    for (float* p : n->act) cudaFree(p);
    for (float* p : n->gact) cudaFree(p);
    n->act.clear();
    n->gact.clear();
    n->act_size.clear();
    cudaFree(n->col);
    cudaFree(n->wtap);
    cudaFree(n->dz);
    cudaFree(n->dzq);
    n->col = nullptr;
    n->wtap = nullptr;
    n->dz = nullptr;
    n->dzq = nullptr;
    Graph g = make_graph(n->ch);
    long long maxt = 0;
    for (auto& ts : g.t) {
        const long long sz = (long long)ts.c * (H >> ts.level) * (W >> ts.level);
        float *a = nullptr, *ga = nullptr;
        if (cudaMalloc(&a, sz * 4) != cudaSuccess || cudaMalloc(&ga, sz * 4) != cudaSuccess) {
            cudaGetLastError();
            return n->fail(LBM_ENOMEM, "network activation buffers");
        }
        n->act.push_back(a);
        n->gact.push_back(ga);
        n->act_size.push_back(sz);
        maxt = std::max(maxt, sz);
    }
    long long maxcol = 0;
    for (auto& c : n->convs) {
        // find the level of this conv from its output tensor is not tracked: bound by level 0
        maxcol = std::max(maxcol, (long long)std::max(c.Kp, c.Kp2));
    }
    // im2col scratch: largest (pixels at the conv's level) x (Kp or Kp2); bound generously
    long long need = 0;
    {
        std::vector<std::pair<int, int>> io;
        conv_list(n->ch, io);
        const int lv[19] = {0, 0, 1, 1, 2, 2, 3, 3, 4, 4, 3, 3, 2, 2, 1, 1, 0, 0, 0};
        for (int i = 0; i < 19; ++i) {
            const ConvSpec& c = n->convs[i];
            const long long P = (long long)(H >> lv[i]) * (W >> lv[i]);
            need = std::max(need, P * (long long)std::max(c.Kp, c.Kp2));
            need = std::max(need, P * (long long)std::max(conv_cp(c.ci), conv_cp(c.co)));  // channels-last inputs
        }
    }
    long long wtap_elems = 0;
    for (auto& c : n->convs)
        wtap_elems = std::max(wtap_elems, 9ll * std::max((long long)c.co * conv_cp(c.ci), (long long)c.ci * conv_cp(c.co)));
    n->col_elems = need;
    if (cudaMalloc(&n->col, need * 2) != cudaSuccess || cudaMalloc(&n->wtap, wtap_elems * 2) != cudaSuccess ||
        cudaMalloc(&n->dz, maxt * 4) != cudaSuccess || cudaMalloc(&n->dzq, maxt * 2) != cudaSuccess) {
        cudaGetLastError();
        return n->fail(LBM_ENOMEM, "network scratch buffers");
    }
    n->H = H;
    n->W = W;
    return LBM_OK;
}

int prep_weights(lbm_net* n) {
    if (!n->weights_dirty) return LBM_OK;
    for (auto& c : n->convs) {
        const int cnt = std::max(c.co * c.Kp, c.ci * c.Kp2);
        k_prep_weights<<<nblk(cnt), 256, 0, n->stream>>>(n->params + c.woff, c.ci, c.co, c.Kp, c.Kp2, n->wq + c.wq_off,
                                                         n->wf + c.wf_off);
    }
    n->weights_dirty = false;
    return n->cuda(cudaGetLastError(), "weight preparation");
}

// y (tensor) = act(conv(x1 ++ x2) + b)
int conv_fwd(lbm_net* n, const ConvSpec& c, const float* x1, int c1, const float* x2, int c2, int H, int W, float* y) {
    const long long P = (long long)H * W;
    int rc = LBM_OK;
    bool implicit = n->backend == 2 || n->backend == 3;
    if (n->backend == 2) {  // implicit GEMM: the im2col rows are gathered inside the tensor-core kernel
        const cudaError_t e = conv3x3_bf16_umma(x1, c1, x2, c2, H, W, c.Kp, n->wq + c.wq_off, c.co, y, (int)P, kStore,
                                                true, n->d_err, n->stream);
        if (e == cudaErrorInvalidValue) implicit = false;  // shape it does not take: explicit im2col below
        else rc = n->cuda(e, "conv (tcgen05 implicit)");
    } else if (n->backend == 3) {  // implicit GEMM over the channels-last input, A tiles by TMA boxes
        rc = n->cuda(weights_tap_major(n->wq + c.wq_off, c.Kp, c1 + c2, c.co, n->wtap, n->stream), "tap-major weights");
        if (!rc) {
            const cudaError_t e = conv3x3_bf16_tma(x1, c1, x2, c2, H, W, n->wtap, c.co, y, (int)P, kStore, true, n->col,
                                                   n->d_err, n->stream);
            if (e == cudaErrorInvalidValue) implicit = false;  // shape it does not take: explicit im2col below
            else rc = n->cuda(e, "conv (tcgen05, TMA boxes)");
        }
    }
    if (!implicit) {
        k_im2col_pk<<<nblk(P * c.Kp), 256, 0, n->stream>>>(x1, c1, x2, c2, H, W, c.Kp, n->col);
        rc = n->cuda(cudaGetLastError(), "im2col");
    }
    if (!rc && !implicit) {
        if (n->backend != 0)  // pixels on the 128-row side, channels on N, stored transposed
            rc = n->cuda(gemm_bf16_nt_umma((int)P, c.co, c.Kp, n->col, c.Kp, n->wq + c.wq_off, c.Kp, y, (int)P, kStore, true, 1,
                                           n->d_err, n->stream), "conv gemm (tcgen05)");
        else
            rc = n->cuda(gemm_bf16_nt(c.co, (int)P, c.Kp, n->wq + c.wq_off, c.Kp, n->col, c.Kp, y, (int)P, kStore, 1, n->stream),
                         "conv gemm");
    }
    if (!rc) {
        k_bias_act<<<nblk(c.co * P), 256, 0, n->stream>>>(y, n->params + c.boff, c.co, P, c.act);
        rc = n->cuda(cudaGetLastError(), "bias/activation");
    }
    return rc;
}

// given dL/dy (gy) and y: accumulate dW, db; accumulate dL/dx into gx1 (c1 channels), gx2 (c2)
int conv_bwd(lbm_net* n, const ConvSpec& c, const float* x1, int c1, const float* x2, int c2, int H, int W,
             const float* y, const float* gy, float* gx1, float* gx2) {
    const long long P = (long long)H * W;
    k_act_back<<<c.co, 256, 0, n->stream>>>(y, gy, n->dz, n->grads + c.boff, P, c.act);
    k_to_bf16<<<nblk(c.co * P), 256, 0, n->stream>>>(n->dz, c.co * P, n->dzq);
    int rc = n->cuda(cudaGetLastError(), "activation backward");
    // weight gradient: dW[co][k] += sum_p dZ[co][p] XcT[k][p]; accumulate in a scratch of Kp
    // columns is not needed: the GEMM writes only k < ci*9 when N = ci*9 (ldc = ci*9)
    if (!rc) {
        k_im2col_kp<<<nblk(P * c.Kp), 256, 0, n->stream>>>(x1, c1, x2, c2, H, W, c.Kp, n->col);
        rc = n->cuda(cudaGetLastError(), "im2col (k-major)");
    }
    if (!rc) {
        const int split = P >= 16384 ? (int)std::min<long long>(32, P / 4096) : 1;
        if (n->backend != 0)  // rows k of the k-major im2col on the 128-row side, co on N
            rc = n->cuda(gemm_bf16_nt_umma(c.ci * 9, c.co, (int)P, n->col, (int)P, n->dzq, (int)P, n->grads + c.woff, c.ci * 9,
                                           kAtomicAdd, true, split, n->d_err, n->stream), "weight-gradient gemm (tcgen05)");
        else
            rc = n->cuda(gemm_bf16_nt(c.co, c.ci * 9, (int)P, n->dzq, (int)P, n->col, (int)P, n->grads + c.woff, c.ci * 9,
                                      kAtomicAdd, split, n->stream), "weight-gradient gemm");
    }
    // data gradient: dX[ci][p] = sum_k Wf[ci][k] dZc[p][k]
    if (!rc && (gx1 || gx2)) {
        const __nv_bfloat16* wf1 = n->wf + c.wf_off;
        const __nv_bfloat16* wf2 = wf1 + (long long)c1 * c.Kp2;
        bool implicit = n->backend == 2 || n->backend == 3;
        if (n->backend == 3) {  // over dZ (co channels) with the flipped weights, tap-major
            bool first = true;
            for (int part = 0; part < 2 && !rc && implicit; ++part) {
                float* gx = part == 0 ? gx1 : gx2;
                if (!gx) continue;
                const int rows = part == 0 ? c1 : c2;
                rc = n->cuda(weights_tap_major(part == 0 ? wf1 : wf2, c.Kp2, c.co, rows, n->wtap, n->stream),
                             "tap-major weights");
                if (rc) break;
                const cudaError_t e = conv3x3_bf16_tma(n->dz, c.co, nullptr, 0, H, W, n->wtap, rows, gx, (int)P, kAccumulate,
                                                       true, n->col, n->d_err, n->stream);
                if (e == cudaErrorInvalidValue && first) implicit = false;  // explicit im2col below
                else rc = n->cuda(e, "data-gradient conv (tcgen05, TMA boxes)");
                first = false;
            }
        } else if (implicit) {  // implicit GEMM over dZ (co channels) with the flipped weights
            bool first = true;  // a shape the kernel does not take is refused before anything launches
            for (int part = 0; part < 2 && !rc && implicit; ++part) {
                float* gx = part == 0 ? gx1 : gx2;
                if (!gx) continue;
                const cudaError_t e = conv3x3_bf16_umma(n->dz, c.co, nullptr, 0, H, W, c.Kp2, part == 0 ? wf1 : wf2,
                                                        part == 0 ? c1 : c2, gx, (int)P, kAccumulate, true, n->d_err,
                                                        n->stream);
                if (e == cudaErrorInvalidValue && first) implicit = false;  // explicit im2col below
                else rc = n->cuda(e, "data-gradient conv (tcgen05 implicit)");
                first = false;
            }
        }
        if (!implicit) {
            k_im2col_pk<<<nblk(P * c.Kp2), 256, 0, n->stream>>>(n->dz, c.co, nullptr, 0, H, W, c.Kp2, n->col);
            rc = n->cuda(cudaGetLastError(), "im2col of dZ");
        }
        if (!implicit && n->backend != 0) {
            if (!rc && gx1)
                rc = n->cuda(gemm_bf16_nt_umma((int)P, c1, c.Kp2, n->col, c.Kp2, wf1, c.Kp2, gx1, (int)P, kAccumulate, true, 1,
                                               n->d_err, n->stream), "data-gradient gemm (tcgen05)");
            if (!rc && gx2)
                rc = n->cuda(gemm_bf16_nt_umma((int)P, c2, c.Kp2, n->col, c.Kp2, wf2, c.Kp2, gx2, (int)P, kAccumulate, true, 1,
                                               n->d_err, n->stream), "data-gradient gemm (tcgen05)");
        } else if (n->backend == 0) {
            if (!rc && gx1)
                rc = n->cuda(gemm_bf16_nt(c1, (int)P, c.Kp2, wf1, c.Kp2, n->col, c.Kp2, gx1, (int)P, kAccumulate, 1, n->stream),
                             "data-gradient gemm");
            if (!rc && gx2)
                rc = n->cuda(gemm_bf16_nt(c2, (int)P, c.Kp2, wf2, c.Kp2, n->col, c.Kp2, gx2, (int)P, kAccumulate, 1, n->stream),
                             "data-gradient gemm");
        }
    }
    return rc;
}

int forward(lbm_net* n, const float* in, int H, int W) {
    int rc = ensure_buffers(n, H, W);
    if (!rc) rc = prep_weights(n);
    if (rc) return rc;
    Graph g = make_graph(n->ch);
    auto A = [&](int t) { return n->act[t]; };
    rc = n->cuda(cudaMemcpyAsync(A(g.input), in, n->act_size[g.input] * 4, cudaMemcpyDeviceToDevice, n->stream), "input copy");
    int ci = 0;  // conv index
    for (int l = 0; l < 5 && !rc; ++l) {
        const int h = H >> l, w = W >> l;
        const float* src = l ? A(g.p[l]) : A(g.input);
        const int csrc = l ? n->ch[l - 1] : 7;
        if (l) {
            k_pool2<<<nblk(n->act_size[g.p[l]]), 256, 0, n->stream>>>(A(g.e[l - 1]), n->ch[l - 1], h * 2, w * 2, A(g.p[l]));
            rc = n->cuda(cudaGetLastError(), "pool");
        }
        if (!rc) rc = conv_fwd(n, n->convs[ci++], src, csrc, nullptr, 0, h, w, A(g.a[l]));
        if (!rc) rc = conv_fwd(n, n->convs[ci++], A(g.a[l]), n->ch[l], nullptr, 0, h, w, A(g.e[l]));
    }
    for (int l = 3; l >= 0 && !rc; --l) {
        const int h = H >> l, w = W >> l;
        const int below = l == 3 ? g.e[4] : g.d[l + 1];
        k_up2<<<nblk(n->act_size[g.u[l]]), 256, 0, n->stream>>>(A(below), n->ch[l + 1], h / 2, w / 2, A(g.u[l]));
        rc = n->cuda(cudaGetLastError(), "upsample");
        if (!rc) rc = conv_fwd(n, n->convs[ci++], A(g.u[l]), n->ch[l + 1], A(g.e[l]), n->ch[l], h, w, A(g.b[l]));
        if (!rc) rc = conv_fwd(n, n->convs[ci++], A(g.b[l]), n->ch[l], nullptr, 0, h, w, A(g.d[l]));
    }
    if (!rc) rc = conv_fwd(n, n->convs[ci++], A(g.d[0]), n->ch[0], nullptr, 0, H, W, A(g.out));
    return rc;
}

int backward(lbm_net* n, int H, int W, const float* gout) {
    Graph g = make_graph(n->ch);
    auto A = [&](int t) { return n->act[t]; };
    auto G = [&](int t) { return n->gact[t]; };
    int rc = LBM_OK;
    for (size_t t = 0; t < n->gact.size() && !rc; ++t)
        rc = n->cuda(cudaMemsetAsync(n->gact[t], 0, n->act_size[t] * 4, n->stream), "gradient reset");
    if (!rc) rc = n->cuda(cudaMemcpyAsync(G(g.out), gout, n->act_size[g.out] * 4, cudaMemcpyDeviceToDevice, n->stream), "gradient copy");
    int ci = (int)n->convs.size() - 1;
    if (!rc) rc = conv_bwd(n, n->convs[ci--], A(g.d[0]), n->ch[0], nullptr, 0, H, W, A(g.out), G(g.out), G(g.d[0]), nullptr);
    for (int l = 0; l <= 3 && !rc; ++l) {
        const int h = H >> l, w = W >> l;
        rc = conv_bwd(n, n->convs[ci--], A(g.b[l]), n->ch[l], nullptr, 0, h, w, A(g.d[l]), G(g.d[l]), G(g.b[l]), nullptr);
        if (!rc) rc = conv_bwd(n, n->convs[ci--], A(g.u[l]), n->ch[l + 1], A(g.e[l]), n->ch[l], h, w, A(g.b[l]), G(g.b[l]), G(g.u[l]), G(g.e[l]));
        const int below = l == 3 ? g.e[4] : g.d[l + 1];
        if (!rc) {
            k_up2_back<<<nblk((long long)n->ch[l + 1] * (h / 2) * (w / 2)), 256, 0, n->stream>>>(G(g.u[l]), n->ch[l + 1], h / 2, w / 2, G(below));
            rc = n->cuda(cudaGetLastError(), "upsample backward");
        }
    }
    for (int l = 4; l >= 0 && !rc; --l) {
        const int h = H >> l, w = W >> l;
        rc = conv_bwd(n, n->convs[ci--], A(g.a[l]), n->ch[l], nullptr, 0, h, w, A(g.e[l]), G(g.e[l]), G(g.a[l]), nullptr);
        const float* src = l ? A(g.p[l]) : A(g.input);
        const int csrc = l ? n->ch[l - 1] : 7;
        if (!rc) rc = conv_bwd(n, n->convs[ci--], src, csrc, nullptr, 0, h, w, A(g.a[l]), G(g.a[l]), l ? G(g.p[l]) : nullptr, nullptr);
        if (!rc && l) {
            k_pool2_back<<<nblk(n->act_size[g.e[l - 1]]), 256, 0, n->stream>>>(G(g.p[l]), n->ch[l - 1], h * 2, w * 2, G(g.e[l - 1]));
            rc = n->cuda(cudaGetLastError(), "pool backward");
        }
    }
    return rc;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" int lbm_net_create(int width, unsigned long long seed, lbm_net** out) {
    g_net_create_error.clear();
    if (!out) return LBM_EINVAL;
    *out = nullptr;
    if (width < 1 || width > 256) {
        g_net_create_error = "width must be in 1..256";
        return LBM_EINVAL;
    }
    lbm_net* n = new lbm_net();
    n->width = width;
    const int mult[5] = {1, 2, 4, 8, 8};
    for (int l = 0; l < 5; ++l) n->ch[l] = width * mult[l];
    std::vector<std::pair<int, int>> io;
    conv_list(n->ch, io);
    long long off = 0, q = 0, f = 0;
    for (size_t i = 0; i < io.size(); ++i) {
        ConvSpec c{};
        c.ci = io[i].first;
        c.co = io[i].second;
        c.act = i + 1 < io.size();
        c.woff = off;
        off += (long long)c.ci * c.co * 9;
        c.boff = off;
        off += c.co;
        c.Kp = pad8(c.ci * 9);
        c.Kp2 = pad8(c.co * 9);
        c.wq_off = q;
        q += (long long)c.co * c.Kp;
        c.wf_off = f;
        f += (long long)c.ci * c.Kp2;
        n->convs.push_back(c);
    }
    n->nparams = off;
    n->nwq = q;
    n->nwf = f;
    auto fail = [&](const std::string& m) {
        g_net_create_error = m;
        lbm_net_destroy(n);
        return LBM_ENOMEM;
    };
    if (cudaMalloc(&n->params, off * 4) != cudaSuccess || cudaMalloc(&n->grads, off * 4) != cudaSuccess ||
        cudaMalloc(&n->adam_m, off * 4) != cudaSuccess || cudaMalloc(&n->adam_v, off * 4) != cudaSuccess ||
        cudaMalloc(&n->wq, q * 2) != cudaSuccess || cudaMalloc(&n->wf, f * 2) != cudaSuccess ||
        cudaMalloc(&n->parts, 1024 * sizeof(double)) != cudaSuccess || cudaMalloc(&n->d_loss, 3 * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&n->d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&n->h_loss, sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return fail("network parameter allocation");
    }
    // He-uniform initialisation from a seeded host generator; biases zero
    std::vector<float> h(off, 0.f);
    std::mt19937_64 rng(seed);
    for (auto& c : n->convs) {
        const float bound = std::sqrt(6.0f / (c.ci * 9.0f)) * (c.act ? 1.0f : 0.1f);
        std::uniform_real_distribution<float> U(-bound, bound);
        for (long long k = 0; k < (long long)c.ci * c.co * 9; ++k) h[c.woff + k] = U(rng);
    }
    if (cudaMemcpy(n->params, h.data(), off * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(n->grads, 0, off * 4) != cudaSuccess || cudaMemset(n->adam_m, 0, off * 4) != cudaSuccess ||
        cudaMemset(n->adam_v, 0, off * 4) != cudaSuccess || cudaMemset(n->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail("network parameter upload");
    }
    *out = n;
    return LBM_OK;
}

extern "C" void lbm_net_destroy(lbm_net* n) {
    if (!n) return;
    cudaStreamSynchronize(n->stream);
    for (float* p : n->act) cudaFree(p);
    for (float* p : n->gact) cudaFree(p);
    for (void* p : {(void*)n->params, (void*)n->grads, (void*)n->adam_m, (void*)n->adam_v, (void*)n->wq, (void*)n->wf,
                    (void*)n->col, (void*)n->wtap, (void*)n->dz, (void*)n->dzq, (void*)n->parts, (void*)n->d_loss,
                    (void*)n->d_err})
        if (p) cudaFree(p);
    if (n->h_loss) cudaFreeHost(n->h_loss);
    delete n;
}

extern "C" const char* lbm_net_last_error(const lbm_net* n) { return n ? n->err.c_str() : g_net_create_error.c_str(); }

extern "C" int lbm_net_set_stream(lbm_net* n, void* stream) {
    if (!n) return LBM_EINVAL;
    cudaStreamSynchronize(n->stream);
    n->stream = (cudaStream_t)stream;
    return LBM_OK;
}

extern "C" long lbm_net_param_count(const lbm_net* n) { return n ? (long)n->nparams : -1; }

static int copy_params(lbm_net* n, float* dst, const float* src, bool to_net) {
    const size_t bytes = n->nparams * 4;
    int rc = n->cuda(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, n->stream), "parameter copy");
    if (!rc) rc = n->cuda(cudaStreamSynchronize(n->stream), "stream synchronize");
    if (to_net) n->weights_dirty = true;
    return rc;
}

extern "C" int lbm_net_get_params(lbm_net* n, float* p) { return (n && p) ? copy_params(n, p, n->params, false) : LBM_EINVAL; }
extern "C" int lbm_net_set_params(lbm_net* n, const float* p) { return (n && p) ? copy_params(n, n->params, p, true) : LBM_EINVAL; }
extern "C" int lbm_net_get_grads(lbm_net* n, float* g) { return (n && g) ? copy_params(n, g, n->grads, false) : LBM_EINVAL; }

extern "C" int lbm_net_zero_grads(lbm_net* n) {
    if (!n) return LBM_EINVAL;
    return n->cuda(cudaMemsetAsync(n->grads, 0, n->nparams * 4, n->stream), "gradient reset");
}

// A tcgen05 GEMM that gave up waiting leaves 1 in d_err (result incomplete).
static int check_err(lbm_net* n) {
    int h = 0;
    int rc = n->cuda(cudaMemcpy(&h, n->d_err, sizeof(int), cudaMemcpyDeviceToHost), "error word copy");
    if (!rc && h) {
        cudaMemset(n->d_err, 0, sizeof(int));
        return n->fail(LBM_ETIMEOUT, "a tensor-core GEMM wait ran out");
    }
    return rc;
}

extern "C" int lbm_net_set_backend(lbm_net* n, int backend) {
    if (!n || backend < 0 || backend > 3) return LBM_EINVAL;
    n->backend = backend;
    return LBM_OK;
}

static int check_shape(lbm_net* n, int H, int W) {
    // four 2x poolings, and the pixel count of every level a multiple of 8 (GEMM rows of 16 bytes)
    if (H < 16 || W < 16 || (H & 15) || (W & 15) || ((H >> 4) * (W >> 4)) % 8)
        return n->fail(LBM_EINVAL, nfmt("input %d x %d: need multiples of 16 and (H/16)(W/16) %% 8 == 0", H, W));
    return LBM_OK;
}

extern "C" int lbm_net_forward(lbm_net* n, const float* in, int H, int W, float* out) {
    NvtxRange nvtx_range("lbm_net_forward");
    if (!n || !in || !out) return LBM_EINVAL;
    int rc = check_shape(n, H, W);
    if (!rc) rc = forward(n, in, H, W);
    if (!rc) {
        Graph g = make_graph(n->ch);
        rc = n->cuda(cudaMemcpyAsync(out, n->act[g.out], n->act_size[g.out] * 4, cudaMemcpyDeviceToDevice, n->stream), "output copy");
    }
    if (!rc && n->backend != 0) {
        rc = n->cuda(cudaStreamSynchronize(n->stream), "stream synchronize");
        if (!rc) rc = check_err(n);
    }
    return rc;
}

extern "C" int lbm_net_backward(lbm_net* n, const float* in, const float* base, const float* target, const float* mask,
                                int H, int W, double* loss) {
    NvtxRange nvtx_range("lbm_net_backward");
    if (!n || !in || !base || !target || !mask) return LBM_EINVAL;
    int rc = check_shape(n, H, W);
    if (!rc) rc = forward(n, in, H, W);
    if (rc) return rc;
    Graph g = make_graph(n->ch);
    const long long P = (long long)H * W;
    const int nb = 512;
    // loss and dL/d(out) (into the dZ scratch, which backward copies before reusing it)
    k_mask_stats<<<1, 256, 0, n->stream>>>(mask, n->act[g.out], base, target, P, n->d_loss);
    k_mse<<<nb, 256, 0, n->stream>>>(n->act[g.out], base, target, mask, P, n->d_loss, n->dz, n->parts);
    k_sum_parts<<<1, 32, 0, n->stream>>>(n->parts, nb, n->d_loss);
    rc = n->cuda(cudaGetLastError(), "loss");
    if (!rc) rc = backward(n, H, W, n->dz);
    if (!rc) rc = n->cuda(cudaMemcpyAsync(n->h_loss, n->d_loss + 1, sizeof(double), cudaMemcpyDeviceToHost, n->stream), "loss copy");
    if (!rc) rc = n->cuda(cudaStreamSynchronize(n->stream), "stream synchronize");
    if (!rc) rc = check_err(n);
    if (!rc && loss) *loss = *n->h_loss;
    return rc;
}

extern "C" int lbm_net_adam_step(lbm_net* n, float lr, float beta1, float beta2, float eps, float grad_scale) {
    NvtxRange nvtx_range("lbm_net_adam_step");
    if (!n) return LBM_EINVAL;
    n->adam_t += 1;
    const float c1 = 1.f / (1.f - std::pow(beta1, (float)n->adam_t));
    const float c2 = 1.f / (1.f - std::pow(beta2, (float)n->adam_t));
    k_adam<<<nblk(n->nparams), 256, 0, n->stream>>>(n->params, n->grads, n->adam_m, n->adam_v, n->nparams, lr, beta1, beta2,
                                                   eps, c1, c2, grad_scale);
    n->weights_dirty = true;
    return n->cuda(cudaGetLastError(), "adam");
}

extern "C" int lbm_net_save(lbm_net* n, const char* path) {
    if (!n || !path) return LBM_EINVAL;
    std::vector<float> h(n->nparams);
    int rc = copy_params(n, h.data(), n->params, false);
    if (rc) return rc;
    FILE* fp = fopen(path, "wb");
    if (!fp) return n->fail(LBM_EIO, nfmt("cannot write %s", path));
    const int hdr[2] = {0x4c424e54, n->width};
    bool ok = fwrite(hdr, sizeof hdr, 1, fp) == 1 && fwrite(h.data(), 4, h.size(), fp) == h.size();
    ok = (fclose(fp) == 0) && ok;
    return ok ? LBM_OK : n->fail(LBM_EIO, "write failed");
}

extern "C" int lbm_net_load(lbm_net* n, const char* path) {
    if (!n || !path) return LBM_EINVAL;
    FILE* fp = fopen(path, "rb");
    if (!fp) return n->fail(LBM_EIO, nfmt("cannot open %s", path));
    int hdr[2];
    std::vector<float> h(n->nparams);
    bool ok = fread(hdr, sizeof hdr, 1, fp) == 1 && hdr[0] == 0x4c424e54 && hdr[1] == n->width &&
              fread(h.data(), 4, h.size(), fp) == h.size();
    fclose(fp);
    if (!ok) return n->fail(LBM_EIO, "not a network file of this width");
    return copy_params(n, n->params, h.data(), true);
}

extern "C" int lbm_warm_input(const double* rho_c, const double* ux_c, const double* uy_c, int nxc, int nyc, double Re,
                              double Ar, double U, int nx, int ny, int H, float* in, void* stream) {
    if (!rho_c || !ux_c || !uy_c || !in || nxc < 2 || nyc < 2 || nx < 2 || ny < 2 || H < ny || !(U != 0)) return LBM_EINVAL;
    const long long P = (long long)H * nx;
    k_warm_input<<<nblk(P), 256, 0, (cudaStream_t)stream>>>(rho_c, ux_c, uy_c, nxc, nyc, (float)(Re / 4000.0),
                                                            (float)(Ar / 2.0), (float)(1.0 / U), LBM_WARM_RHO_SCALE, nx, ny, H, in);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_warm_output(const float* in, const float* out, int nx, int ny, int H, double U, double* rho,
                               double* ux, double* uy, void* stream) {
    if (!in || !out || !rho || !ux || !uy || H < ny) return LBM_EINVAL;
    k_warm_output<<<nblk((long long)nx * ny), 256, 0, (cudaStream_t)stream>>>(in, out, nx, ny, H, (float)U, LBM_WARM_RHO_SCALE,
                                                                            rho, ux, uy);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_warm_smooth(float* out, int ny, int H, int W, int passes, float* scratch, void* stream) {
    if (!out || !scratch || ny < 1 || H < ny || W < 1 || passes < 0) return LBM_EINVAL;
    const long long n = 3ll * H * W;
    for (int k = 0; k < passes; ++k) {
        const float* src = (k & 1) ? scratch : out;
        float* dst = (k & 1) ? out : scratch;
        k_warm_smooth<<<nblk(n), 256, 0, (cudaStream_t)stream>>>(src, dst, ny, H, W);
    }
    if (passes & 1) cudaMemcpyAsync(out, scratch, n * sizeof(float), cudaMemcpyDeviceToDevice, (cudaStream_t)stream);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_warm_target(const double* rho, const double* ux, const double* uy, int nx, int ny, int H, double U,
                               float* target, void* stream) {
    if (!rho || !ux || !uy || !target || H < ny || nx < 1 || !(U != 0.0)) return LBM_EINVAL;
    k_warm_target<<<nblk((long long)H * nx), 256, 0, (cudaStream_t)stream>>>(rho, ux, uy, nx, ny, H, 1.0 / U,
                                                                           LBM_WARM_RHO_SCALE, target);
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_nn_gemm_bf16(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C, int ldc,
                                int op, int split_k, void* stream) {
    if (!A || !B || !C || op < 0 || op > 2) return LBM_EINVAL;
    const cudaError_t e = gemm_bf16_nt(M, N, K, static_cast<const __nv_bfloat16*>(A), lda,
                                       static_cast<const __nv_bfloat16*>(B), ldb, C, ldc, (GemmOp)op, split_k,
                                       (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return LBM_EINVAL;
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_nn_conv3x3_bf16_tc05(const float* x1, int c1, const float* x2, int c2, int H, int W, int K,
                                        const void* Wt, int N, float* C, int ldc, int op, int trans_c, int* err,
                                        void* stream) {
    if (!x1 || !Wt || !C || !err || op < 0 || op > 2 || H < 1 || W < 1) return LBM_EINVAL;
    const cudaError_t e = conv3x3_bf16_umma(x1, c1, x2, c2, H, W, K, static_cast<const __nv_bfloat16*>(Wt), N, C, ldc,
                                            (GemmOp)op, trans_c != 0, err, (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return LBM_EINVAL;
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_nn_weights_tap_major(const void* Wt, int ldk, int C, int N, void* Wtap, void* stream) {
    if (!Wt || !Wtap || C < 1 || N < 1 || ldk < 9 * C) return LBM_EINVAL;
    const cudaError_t e = weights_tap_major(static_cast<const __nv_bfloat16*>(Wt), ldk, C, N,
                                            static_cast<__nv_bfloat16*>(Wtap), (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return LBM_EINVAL;
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_nn_conv3x3_bf16_tma(const float* x1, int c1, const float* x2, int c2, int H, int W, const void* Wtap,
                                       int N, float* C, int ldc, int op, int trans_c, void* xs, int* err, void* stream) {
    if (!x1 || !Wtap || !C || !xs || !err || op < 0 || op > 2 || H < 1 || W < 1) return LBM_EINVAL;
    const cudaError_t e = conv3x3_bf16_tma(x1, c1, x2, c2, H, W, static_cast<const __nv_bfloat16*>(Wtap), N, C, ldc,
                                           (GemmOp)op, trans_c != 0, static_cast<__nv_bfloat16*>(xs), err,
                                           (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return LBM_EINVAL;
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}

extern "C" int lbm_nn_gemm_bf16_tc05(int M, int N, int K, const void* A, int lda, const void* B, int ldb, float* C,
                                     int ldc, int op, int trans_c, int split_k, int* err, void* stream) {
    if (!A || !B || !C || !err || op < 0 || op > 2) return LBM_EINVAL;
    const cudaError_t e = gemm_bf16_nt_umma(M, N, K, static_cast<const __nv_bfloat16*>(A), lda,
                                            static_cast<const __nv_bfloat16*>(B), ldb, C, ldc, (GemmOp)op, trans_c != 0,
                                            split_k, err, (cudaStream_t)stream);
    if (e == cudaErrorInvalidValue) return LBM_EINVAL;
    return e == cudaSuccess ? LBM_OK : LBM_ECUDA;
}
