// Surrogate network (lb_mlp_*): 3 -> 64 -> 64 -> 3 GELU MLP mapping (T/T_c, kappa, tau_v)
// to (sigma, rho_l, rho_v), trained on the GPU by hand-written kernels:
//   k_mlp_prepare  one CTA: FP64 means / scales of the input features
//                  (ln(1 - T/T_c), ln(1 - kappa), tau_v) and of the transformed targets,
//                  standardised copies (float)
//   k_mlp_grad     forward + backward over tiles of kTile samples; each CTA accumulates
//                  its tiles' gradient in registers and writes one partial vector
//   k_mlp_adam     sums the partials in a fixed order, Adam update of the FP32 master
//                  copy, refreshes the BF16 image used by the next forward pass
//   k_mlp_forward  inference, one thread per sample
//   k_mlp_invert   bisection on kappa for a target sigma, one thread per query
// The weights are read as BF16 and every product is accumulated in FP32 (fmaf, in the
// order of the sums' indices), so the training forward pass and k_mlp_forward give the
// same bits for the same sample.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lb_internal.h"
#include "lb_mlp.h"

namespace {

constexpr int IN = LB_MLP_IN, H = LB_MLP_HIDDEN, OUT = LB_MLP_OUT, NP = LB_MLP_PARAMS;
constexpr int OW1 = 0, OB1 = OW1 + H * IN, OW2 = OB1 + H, OB2 = OW2 + H * H, OW3 = OB2 + H,
              OB3 = OW3 + OUT * H;
static_assert(OB3 + OUT == NP, "parameter layout");

constexpr int kTile = 16;          // samples per tile of k_mlp_grad
constexpr int kThreads = 256;      // k_mlp_grad block
constexpr int kMaxGradCtas = 304;  // 2 x 152 SMs: bounds the partial-gradient buffer
constexpr int kW2Pitch = H + 1;    // padded rows of W2 in shared memory (no bank conflicts)
constexpr int kGraphSteps = 50;
constexpr int kMaxSamples = 1 << 20;
constexpr int kMaxForward = 1 << 22;
constexpr int kBisect = 40;

struct MlpNorm {
    float in_mean[3], in_scale[3], out_mean[3], out_scale[3];
};

struct MlpState {
    int step;          // Adam step count (incremented by the first CTA of k_mlp_grad)
    int n;             // resident samples
    float lr, beta1, beta2, eps;
    float loss;        // loss of the last forward pass of k_mlp_grad (set by k_mlp_adam)
    int pad;
};

__device__ __forceinline__ float gelu(float z) {
    return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f));
}

// d/dz [z Phi(z)] = Phi(z) + z phi(z)
__device__ __forceinline__ float gelu_grad(float z) {
    return 0.5f * (1.0f + erff(z * 0.70710678118654752f))
           + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Weights as float in shared memory; W2 rows padded to kW2Pitch.
struct SmemW {
    float w1[H * IN], b1[H], w2[H * kW2Pitch], b2[H], w3[OUT * H], b3[4];
};

__device__ void load_weights(SmemW &w, const __nv_bfloat16 *__restrict__ wbf) {
    for (int p = threadIdx.x; p < NP; p += blockDim.x) {
        const float v = __bfloat162float(wbf[p]);
        if (p < OB1) w.w1[p] = v;
        else if (p < OW2) w.b1[p - OB1] = v;
        else if (p < OB2) { const int q = p - OW2; w.w2[(q / H) * kW2Pitch + q % H] = v; }
        else if (p < OW3) w.b2[p - OB2] = v;
        else if (p < OB3) w.w3[p - OW3] = v;
        else w.b3[p - OB3] = v;
    }
}

// Input features (ln(1 - T/T_c), ln(1 - kappa), tau_v) in float, as inference computes them.
__device__ __forceinline__ float input_feature(float v, int c) {
    return c == 2 ? v : log1pf(-v);
}

// ---------------------------------------------------------------------------------
// Data preparation: one CTA of 512 threads. Two-pass FP64 mean / variance with a fixed
// reduction tree, the scale rule of the header, then standardised float copies in place.
// ---------------------------------------------------------------------------------
constexpr int kPrepThreads = 512;

__device__ void block_sum6(double (&v)[6], double (*red)[6]) {
    const int t = threadIdx.x;
    for (int c = 0; c < 6; ++c) red[t][c] = v[c];
    __syncthreads();
    for (int s = kPrepThreads / 2; s > 0; s >>= 1) {
        if (t < s)
            for (int c = 0; c < 6; ++c) red[t][c] += red[t + s][c];
        __syncthreads();
    }
    for (int c = 0; c < 6; ++c) v[c] = red[0][c];
    __syncthreads();
}

__global__ void __launch_bounds__(kPrepThreads)
k_mlp_prepare(float *__restrict__ x, float *__restrict__ y, int n, MlpNorm *__restrict__ norm) {
    __shared__ double red[kPrepThreads][6];
    const int t = threadIdx.x;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    auto feature = [&](int i, int c) -> double {
        const double v = (double)x[3 * i + c];
        return c == 2 ? v : log1p(-v);
    };
    auto target = [&](int i, int c) -> double {
        const double v = (double)y[3 * i + c];
        return c == 1 ? v : log(v);
    };
    for (int i = t; i < n; i += kPrepThreads)
        for (int c = 0; c < 3; ++c) {
            acc[c] += feature(i, c);
            acc[3 + c] += target(i, c);
        }
    block_sum6(acc, red);
    double mean[6];
    for (int c = 0; c < 6; ++c) mean[c] = acc[c] / n;
    double sq[6] = {0, 0, 0, 0, 0, 0};
    for (int i = t; i < n; i += kPrepThreads)
        for (int c = 0; c < 3; ++c) {
            const double dx = feature(i, c) - mean[c];
            const double dt = target(i, c) - mean[3 + c];
            sq[c] += dx * dx;
            sq[3 + c] += dt * dt;
        }
    block_sum6(sq, red);
    __shared__ float nm[12];
    if (t == 0) {
        for (int c = 0; c < 6; ++c) {
            const double s = sqrt(sq[c] / n);
            const double scale = (s > 0.0 && s > 1e-9 * fabs(mean[c])) ? s : 1.0;
            const int k = c < 3 ? c : 6 + (c - 3);
            nm[k] = (float)mean[c];
            nm[k + 3] = (float)scale;
        }
        for (int c = 0; c < 3; ++c) {
            norm->in_mean[c] = nm[c];
            norm->in_scale[c] = nm[3 + c];
            norm->out_mean[c] = nm[6 + c];
            norm->out_scale[c] = nm[9 + c];
        }
    }
    __syncthreads();
    for (int i = t; i < n; i += kPrepThreads)
        for (int c = 0; c < 3; ++c) {
            x[3 * i + c] = (input_feature(x[3 * i + c], c) - nm[c]) / nm[3 + c];
            const float yv = y[3 * i + c];
            const float tv = c == 1 ? yv : logf(yv);
            y[3 * i + c] = (tv - nm[6 + c]) / nm[9 + c];
        }
}

// ---------------------------------------------------------------------------------
// Forward + backward. Block of 256 threads, tiles of 16 samples; the CTA walks tiles
// blockIdx.x, blockIdx.x + gridDim.x, ... and keeps the gradient entries it owns in
// registers:
//   gW2: 16 per thread (k = t & 63, j = (t >> 6) + 4q)     gb2: threads 0..63
//   gW3 / gb3: threads 0..191 / 192..194                   gW1 / gb1: 0..191 / 192..255
// Activations of a tile live in shared memory; dz overwrites z in place.
// ---------------------------------------------------------------------------------
__global__ void __launch_bounds__(kThreads)
k_mlp_grad(const __nv_bfloat16 *__restrict__ wbf, const float *__restrict__ xn,
           const float *__restrict__ tn, MlpState *__restrict__ st, int bump_step,
           float *__restrict__ part, float *__restrict__ lpart) {
    __shared__ SmemW w;
    __shared__ float sx[kTile * IN], dout[kTile * OUT];
    __shared__ float z1[kTile * H], a1[kTile * H], z2[kTile * H], a2[kTile * H];
    const int t = threadIdx.x;
    const int n = st->n;
    if (bump_step && blockIdx.x == 0 && t == 0) st->step += 1;
    load_weights(w, wbf);
    const float dscale = 2.0f / (3.0f * (float)n);

    float gw2[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) gw2[q] = 0.f;
    float gb2 = 0.f, g3 = 0.f, g1 = 0.f, lsum = 0.f;

    const int jj = t & 63, sg = t >> 6;   // unit and sample group of the 4-per-thread loops
    for (int base = blockIdx.x * kTile; base < n; base += gridDim.x * kTile) {
        __syncthreads();   // weights loaded / previous tile consumed
        if (t < kTile * IN) {
            const int s = t / IN;
            sx[t] = base + s < n ? xn[(size_t)base * IN + t] : 0.f;
        }
        __syncthreads();
        // layer 1
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = sg + 4 * q;
            float z = w.b1[jj];
#pragma unroll
            for (int i = 0; i < IN; ++i) z = fmaf(w.w1[jj * IN + i], sx[s * IN + i], z);
            z1[s * H + jj] = z;
            a1[s * H + jj] = gelu(z);
        }
        __syncthreads();
        // layer 2
        {
            float acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = w.b2[jj];
#pragma unroll 8
            for (int k = 0; k < H; ++k) {
                const float wv = w.w2[jj * kW2Pitch + k];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(wv, a1[(sg + 4 * q) * H + k], acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                z2[(sg + 4 * q) * H + jj] = acc[q];
                a2[(sg + 4 * q) * H + jj] = gelu(acc[q]);
            }
        }
        __syncthreads();
        // output layer and loss residual
        if (t < kTile * OUT) {
            const int s = t / OUT, c = t % OUT;
            float o = w.b3[c];
            for (int k = 0; k < H; ++k) o = fmaf(w.w3[c * H + k], a2[s * H + k], o);
            const float r = base + s < n ? o - tn[(size_t)base * OUT + t] : 0.f;
            dout[t] = r * dscale;
            sx[t] = r;   // the tile's inputs are re-read below only by gW1: kept in xn
        }
        __syncthreads();
        if (t == 0)
            for (int k = 0; k < kTile * OUT; ++k) lsum = fmaf(sx[k], sx[k], lsum);
        // gW3, gb3; dz2 = (dout W3) * gelu'(z2) in place
        if (t < OUT * H) {
            const int c = t >> 6, k = t & 63;
            for (int s = 0; s < kTile; ++s) g3 = fmaf(dout[s * OUT + c], a2[s * H + k], g3);
        } else if (t < OUT * H + OUT) {
            const int c = t - OUT * H;
            for (int s = 0; s < kTile; ++s) g3 += dout[s * OUT + c];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int s = sg + 4 * q;
            float d = 0.f;
#pragma unroll
            for (int c = 0; c < OUT; ++c) d = fmaf(dout[s * OUT + c], w.w3[c * H + jj], d);
            z2[s * H + jj] = d * gelu_grad(z2[s * H + jj]);
        }
        __syncthreads();
        // gW2, gb2; dz1 = (dz2 W2) * gelu'(z1) in place
        for (int s = 0; s < kTile; ++s) {
            const float av = a1[s * H + jj];
#pragma unroll
            for (int q = 0; q < 16; ++q) gw2[q] = fmaf(z2[s * H + sg + 4 * q], av, gw2[q]);
        }
        if (t < H)
            for (int s = 0; s < kTile; ++s) gb2 += z2[s * H + t];
        {
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
            for (int j = 0; j < H; ++j) {
                const float wv = w.w2[j * kW2Pitch + jj];
#pragma unroll
                for (int q = 0; q < 4; ++q) acc[q] = fmaf(z2[(sg + 4 * q) * H + j], wv, acc[q]);
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int s = sg + 4 * q;
                z1[s * H + jj] = acc[q] * gelu_grad(z1[s * H + jj]);
            }
        }
        __syncthreads();
        // gW1, gb1 (inputs re-read from global memory: sx now holds residuals)
        if (t < H * IN) {
            const int j = t / IN, i = t % IN;
            for (int s = 0; s < kTile; ++s) {
                const float xv = base + s < n ? xn[(size_t)(base + s) * IN + i] : 0.f;
                g1 = fmaf(z1[s * H + j], xv, g1);
            }
        } else {
            const int j = t - H * IN;
            for (int s = 0; s < kTile; ++s) g1 += z1[s * H + j];
        }
    }
    float *out = part + (size_t)blockIdx.x * NP;
#pragma unroll
    for (int q = 0; q < 16; ++q) out[OW2 + (sg + 4 * q) * H + jj] = gw2[q];
    if (t < H) out[OB2 + t] = gb2;
    if (t < OUT * H) out[OW3 + t] = g3;
    else if (t < OUT * H + OUT) out[OB3 + t - OUT * H] = g3;
    if (t < H * IN) out[OW1 + t] = g1;
    else out[OB1 + t - H * IN] = g1;
    if (t == 0) lpart[blockIdx.x] = lsum;
}

// Sum of the partial gradients in CTA order, then Adam on the FP32 master copy.
__global__ void __launch_bounds__(256)
k_mlp_adam(const float *__restrict__ part, const float *__restrict__ lpart, int nparts,
           MlpState *__restrict__ st, float *__restrict__ master, float *__restrict__ m1,
           float *__restrict__ m2, __nv_bfloat16 *__restrict__ wbf, float *__restrict__ grad_out) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        double l = 0.0;
        for (int c = 0; c < nparts; ++c) l += (double)lpart[c];
        st->loss = (float)(l / (3.0 * st->n));
    }
    if (p >= NP) return;
    float g = 0.f;
    for (int c = 0; c < nparts; ++c) g += part[(size_t)c * NP + p];
    if (grad_out) {   // gradient only (no update)
        grad_out[p] = g;
        return;
    }
    const float b1 = st->beta1, b2 = st->beta2;
    const float m = fmaf(b1, m1[p], (1.f - b1) * g);
    const float v = fmaf(b2, m2[p], (1.f - b2) * g * g);
    m1[p] = m;
    m2[p] = v;
    const double tstep = (double)st->step;
    const float c1 = (float)(1.0 - pow((double)b1, tstep));
    const float c2 = (float)(1.0 - pow((double)b2, tstep));
    const float upd = st->lr * (m / c1) / (sqrtf(v / c2) + st->eps);
    const float th = master[p] - upd;
    master[p] = th;
    wbf[p] = __float2bfloat16_rn(th);
}

__global__ void k_mlp_refresh_bf16(const float *__restrict__ master, __nv_bfloat16 *__restrict__ wbf) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p < NP) wbf[p] = __float2bfloat16_rn(master[p]);
}

// One sample through the network (weights in shared memory), standardised output.
__device__ void forward_one(const SmemW &w, const float (&xs)[3], float (&o)[3]) {
    float a[H];
#pragma unroll
    for (int j = 0; j < H; ++j) {
        float z = w.b1[j];
#pragma unroll
        for (int i = 0; i < IN; ++i) z = fmaf(w.w1[j * IN + i], xs[i], z);
        a[j] = gelu(z);
    }
    // the outputs accumulate over j in order, like the output layer of k_mlp_grad
    float acc0 = w.b3[0], acc1 = w.b3[1], acc2 = w.b3[2];
    for (int j = 0; j < H; ++j) {
        float z = w.b2[j];
#pragma unroll
        for (int k = 0; k < H; ++k) z = fmaf(w.w2[j * kW2Pitch + k], a[k], z);
        const float g = gelu(z);
        acc0 = fmaf(w.w3[0 * H + j], g, acc0);
        acc1 = fmaf(w.w3[1 * H + j], g, acc1);
        acc2 = fmaf(w.w3[2 * H + j], g, acc2);
    }
    o[0] = acc0;
    o[1] = acc1;
    o[2] = acc2;
}

__device__ __forceinline__ void standardise(const MlpNorm &nm, const float (&x)[3], float (&xs)[3]) {
#pragma unroll
    for (int i = 0; i < IN; ++i) xs[i] = (input_feature(x[i], i) - nm.in_mean[i]) / nm.in_scale[i];
}

__device__ __forceinline__ float sigma_of(const MlpNorm &nm, float o0) {
    return expf(fmaf(o0, nm.out_scale[0], nm.out_mean[0]));
}

__global__ void __launch_bounds__(128)
k_mlp_forward(const __nv_bfloat16 *__restrict__ wbf, const MlpNorm *__restrict__ norm,
              const float *__restrict__ x, float *__restrict__ y, int n) {
    __shared__ SmemW w;
    __shared__ MlpNorm nm;
    load_weights(w, wbf);
    if (threadIdx.x == 0) nm = *norm;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float xv[3] = {x[3 * i], x[3 * i + 1], x[3 * i + 2]}, xs[3], o[3];
    standardise(nm, xv, xs);
    forward_one(w, xs, o);
    y[3 * i + 0] = sigma_of(nm, o[0]);
    y[3 * i + 1] = fmaf(o[1], nm.out_scale[1], nm.out_mean[1]);
    y[3 * i + 2] = expf(fmaf(o[2], nm.out_scale[2], nm.out_mean[2]));
}

__global__ void __launch_bounds__(128)
k_mlp_invert(const __nv_bfloat16 *__restrict__ wbf, const MlpNorm *__restrict__ norm,
             const float *__restrict__ q, int n, float lo0, float hi0, float *__restrict__ kappa) {
    __shared__ SmemW w;
    __shared__ MlpNorm nm;
    load_weights(w, wbf);
    if (threadIdx.x == 0) nm = *norm;
    __syncthreads();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float tt = q[3 * i], tau = q[3 * i + 1], target = q[3 * i + 2];
    auto sigma = [&](float k) {
        float xv[3] = {tt, k, tau}, xs[3], o[3];
        standardise(nm, xv, xs);
        forward_one(w, xs, o);
        return sigma_of(nm, o[0]);
    };
    // one call site of the network (the bracket check is iterations -2 and -1)
    float lo = lo0, hi = hi0;
    bool ok = true;
    for (int it = -2; it < kBisect && ok; ++it) {
        const float k = it == -2 ? lo : (it == -1 ? hi : 0.5f * (lo + hi));
        const float s = sigma(k);
        if (it == -2) ok = s >= target;
        else if (it == -1) ok = s <= target;
        else if (s > target) lo = k;
        else hi = k;
    }
    if (!ok) {
        kappa[i] = __int_as_float(0x7fc00000);
        return;
    }
    kappa[i] = 0.5f * (lo + hi);
}

}  // namespace

struct lb_mlp {
    cudaStream_t stream = nullptr;
    int max_samples = 0, n = 0, grad_ctas = 0;
    float *master = nullptr, *m1 = nullptr, *m2 = nullptr, *xn = nullptr, *tn = nullptr;
    float *part = nullptr, *lpart = nullptr, *grad = nullptr;
    __nv_bfloat16 *wbf = nullptr;
    MlpNorm *norm = nullptr;
    MlpState *st = nullptr;
    float *io = nullptr;          // staging for forward / invert
    size_t io_floats = 0;
    long long steps = 0;
    bool have_norm = false;
    cudaGraphExec_t graph = nullptr;
    std::string msg;
};

namespace {

lb_status mfail(lb_mlp *m, lb_status s, const std::string &msg) {
    if (m) m->msg = msg;
    return s;
}

#define LB_MCUDA(m, call)                                                              \
    do {                                                                               \
        cudaError_t e_ = (call);                                                       \
        if (e_ != cudaSuccess)                                                         \
            return mfail((m), LB_ECUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

bool finite3(const float *v) {
    return std::isfinite(v[0]) && std::isfinite(v[1]) && std::isfinite(v[2]);
}

cudaError_t launch_grad(lb_mlp *m, int bump, cudaStream_t s) {
    k_mlp_grad<<<m->grad_ctas, kThreads, 0, s>>>(m->wbf, m->xn, m->tn, m->st, bump, m->part,
                                                 m->lpart);
    return cudaGetLastError();
}

cudaError_t launch_adam(lb_mlp *m, float *grad_out, cudaStream_t s) {
    k_mlp_adam<<<(NP + 255) / 256, 256, 0, s>>>(m->part, m->lpart, m->grad_ctas, m->st,
                                                m->master, m->m1, m->m2, m->wbf, grad_out);
    return cudaGetLastError();
}

lb_status ensure_graph(lb_mlp *m) {
    if (m->graph) return LB_OK;
    cudaStream_t cap = nullptr;
    LB_MCUDA(m, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) {
            e = launch_grad(m, 1, cap);
            if (e == cudaSuccess) e = launch_adam(m, nullptr, cap);
        }
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&m->graph, g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess)
        return mfail(m, LB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    return LB_OK;
}

void drop_graph(lb_mlp *m) {
    if (m->graph) cudaGraphExecDestroy(m->graph);
    m->graph = nullptr;
}

lb_status ensure_io(lb_mlp *m, size_t floats) {
    if (floats <= m->io_floats) return LB_OK;
    if (m->io) cudaFree(m->io);
    m->io = nullptr;
    m->io_floats = 0;
    if (cudaMalloc(&m->io, floats * sizeof(float)) != cudaSuccess) {
        cudaGetLastError();
        return mfail(m, LB_ENOMEM, "staging allocation failed");
    }
    m->io_floats = floats;
    return LB_OK;
}

}  // namespace

extern "C" {

lb_status lb_mlp_create(lb_mlp **out, int max_samples, void *stream) {
    if (!out) return LB_EINVAL;
    *out = nullptr;
    if (max_samples < 1 || max_samples > kMaxSamples) return LB_EINVAL;
    lb_mlp *m = new (std::nothrow) lb_mlp();
    if (!m) return LB_ENOMEM;
    m->stream = static_cast<cudaStream_t>(stream);
    m->max_samples = max_samples;
    const size_t ns = (size_t)max_samples;
    bool ok = cudaMalloc(&m->master, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->m1, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->m2, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->grad, NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->wbf, NP * sizeof(__nv_bfloat16)) == cudaSuccess &&
              cudaMalloc(&m->xn, ns * IN * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->tn, ns * OUT * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->part, (size_t)kMaxGradCtas * NP * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->lpart, kMaxGradCtas * sizeof(float)) == cudaSuccess &&
              cudaMalloc(&m->norm, sizeof(MlpNorm)) == cudaSuccess &&
              cudaMalloc(&m->st, sizeof(MlpState)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        lb_mlp_free(m);
        return LB_ENOMEM;
    }
    std::vector<float> zero(NP, 0.f);
    if (lb_mlp_set_params(m, zero.data()) != LB_OK) {
        lb_mlp_free(m);
        return LB_ECUDA;
    }
    MlpNorm nm;
    for (int c = 0; c < 3; ++c) {
        nm.in_mean[c] = nm.out_mean[c] = 0.f;
        nm.in_scale[c] = nm.out_scale[c] = 1.f;
    }
    MlpState st{};
    if (cudaMemcpy(m->norm, &nm, sizeof nm, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(m->st, &st, sizeof st, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaGetLastError();
        lb_mlp_free(m);
        return LB_ECUDA;
    }
    *out = m;
    return LB_OK;
}

lb_status lb_mlp_set_params(lb_mlp *m, const float *params) {
    if (!m || !params) return LB_EINVAL;
    for (int p = 0; p < NP; ++p)
        if (!std::isfinite(params[p])) return mfail(m, LB_EINVAL, "non-finite parameter");
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(m->master, params, NP * sizeof(float), cudaMemcpyHostToDevice));
    LB_MCUDA(m, cudaMemset(m->m1, 0, NP * sizeof(float)));
    LB_MCUDA(m, cudaMemset(m->m2, 0, NP * sizeof(float)));
    LB_MCUDA(m, cudaMemset(m->st, 0, sizeof(int)));   // Adam step count
    k_mlp_refresh_bf16<<<(NP + 255) / 256, 256, 0, m->stream>>>(m->master, m->wbf);
    LB_MCUDA(m, cudaGetLastError());
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    m->steps = 0;
    return LB_OK;
}

lb_status lb_mlp_get_params(lb_mlp *m, float *params) {
    if (!m || !params) return LB_EINVAL;
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(params, m->master, NP * sizeof(float), cudaMemcpyDeviceToHost));
    return LB_OK;
}

lb_status lb_mlp_set_data(lb_mlp *m, const float *x, const float *y, int n) {
    if (!m || !x || !y) return LB_EINVAL;
    if (n < 1 || n > m->max_samples)
        return mfail(m, LB_EINVAL, "sample count outside [1, max_samples]");
    for (int i = 0; i < n; ++i) {
        if (!finite3(x + 3 * i) || !finite3(y + 3 * i))
            return mfail(m, LB_EINVAL, "non-finite sample " + std::to_string(i));
        if (!(y[3 * i] > 0.f && y[3 * i + 1] > 0.f && y[3 * i + 2] > 0.f))
            return mfail(m, LB_EINVAL, "target <= 0 in sample " + std::to_string(i));
        if (!(x[3 * i] < 1.f && x[3 * i + 1] < 1.f))
            return mfail(m, LB_EINVAL, "T/T_c or kappa >= 1 in sample " + std::to_string(i));
    }
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(m->xn, x, (size_t)n * IN * sizeof(float), cudaMemcpyHostToDevice));
    LB_MCUDA(m, cudaMemcpy(m->tn, y, (size_t)n * OUT * sizeof(float), cudaMemcpyHostToDevice));
    k_mlp_prepare<<<1, kPrepThreads, 0, m->stream>>>(m->xn, m->tn, n, m->norm);
    LB_MCUDA(m, cudaGetLastError());
    LB_MCUDA(m, cudaMemcpyAsync(&m->st->n, &n, sizeof(int), cudaMemcpyHostToDevice, m->stream));
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    m->n = n;
    const int tiles = (n + kTile - 1) / kTile;
    const int ctas = tiles < kMaxGradCtas ? tiles : kMaxGradCtas;
    if (ctas != m->grad_ctas) drop_graph(m);
    m->grad_ctas = ctas;
    m->have_norm = true;
    return LB_OK;
}

lb_status lb_mlp_get_norm(lb_mlp *m, lb_mlp_norm *out) {
    if (!m || !out) return LB_EINVAL;
    MlpNorm nm;
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(&nm, m->norm, sizeof nm, cudaMemcpyDeviceToHost));
    static_assert(sizeof(MlpNorm) == sizeof(lb_mlp_norm), "norm layout");
    std::memcpy(out, &nm, sizeof nm);
    return LB_OK;
}

lb_status lb_mlp_set_norm(lb_mlp *m, const lb_mlp_norm *norm) {
    if (!m || !norm) return LB_EINVAL;
    for (int c = 0; c < 3; ++c)
        if (!(std::isfinite(norm->in_mean[c]) && std::isfinite(norm->out_mean[c]) &&
              norm->in_scale[c] > 0.f && std::isfinite(norm->in_scale[c]) &&
              norm->out_scale[c] > 0.f && std::isfinite(norm->out_scale[c])))
            return mfail(m, LB_EINVAL, "scales must be positive and finite");
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(m->norm, norm, sizeof(MlpNorm), cudaMemcpyHostToDevice));
    return LB_OK;
}

lb_status lb_mlp_loss_grad(lb_mlp *m, float *loss, float *grad) {
    if (!m) return LB_EINVAL;
    if (m->n < 1) return mfail(m, LB_EINVAL, "no training data");
    LB_MCUDA(m, launch_grad(m, 0, m->stream));
    LB_MCUDA(m, launch_adam(m, m->grad, m->stream));
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    if (grad) LB_MCUDA(m, cudaMemcpy(grad, m->grad, NP * sizeof(float), cudaMemcpyDeviceToHost));
    if (loss)
        LB_MCUDA(m, cudaMemcpy(loss, &m->st->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return LB_OK;
}

lb_status lb_mlp_train(lb_mlp *m, int steps, float lr, float beta1, float beta2, float eps,
                       float *loss) {
    const lbm::NvtxRange nvtx_range("lb_mlp_train");
    if (!m || steps < 0) return LB_EINVAL;
    if (m->n < 1) return mfail(m, LB_EINVAL, "no training data");
    if (!(lr > 0.f && std::isfinite(lr) && beta1 >= 0.f && beta1 < 1.f && beta2 >= 0.f &&
          beta2 < 1.f && eps > 0.f && std::isfinite(eps)))
        return mfail(m, LB_EINVAL, "bad Adam hyper-parameters");
    const float hp[4] = {lr, beta1, beta2, eps};
    LB_MCUDA(m, cudaMemcpyAsync(&m->st->lr, hp, sizeof hp, cudaMemcpyHostToDevice, m->stream));
    // the host array must stay valid until the copy ran
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    int left = steps;
    while (left >= kGraphSteps) {
        lb_status s = ensure_graph(m);
        if (s != LB_OK) return s;
        LB_MCUDA(m, cudaGraphLaunch(m->graph, m->stream));
        left -= kGraphSteps;
    }
    for (; left > 0; --left) {
        LB_MCUDA(m, launch_grad(m, 1, m->stream));
        LB_MCUDA(m, launch_adam(m, nullptr, m->stream));
    }
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    m->steps += steps;
    if (loss)
        LB_MCUDA(m, cudaMemcpy(loss, &m->st->loss, sizeof(float), cudaMemcpyDeviceToHost));
    return LB_OK;
}

long long lb_mlp_steps_done(const lb_mlp *m) { return m ? m->steps : -1; }

lb_status lb_mlp_forward(lb_mlp *m, const float *x, float *y, int n) {
    if (!m || n < 0 || n > kMaxForward || (n > 0 && (!x || !y))) return LB_EINVAL;
    if (n == 0) return LB_OK;
    for (int i = 0; i < n; ++i)
        if (!(finite3(x + 3 * i) && x[3 * i] < 1.f && x[3 * i + 1] < 1.f))
            return mfail(m, LB_EINVAL, "need finite inputs with T/T_c < 1 and kappa < 1");
    lb_status s = ensure_io(m, (size_t)n * 6);
    if (s != LB_OK) return s;
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(m->io, x, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice));
    k_mlp_forward<<<(n + 127) / 128, 128, 0, m->stream>>>(m->wbf, m->norm, m->io,
                                                          m->io + (size_t)n * 3, n);
    LB_MCUDA(m, cudaGetLastError());
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(y, m->io + (size_t)n * 3, (size_t)n * 3 * sizeof(float),
                           cudaMemcpyDeviceToHost));
    return LB_OK;
}

lb_status lb_mlp_invert_kappa(lb_mlp *m, const float *q, int n, float kappa_lo,
                              float kappa_hi, float *kappa) {
    if (!m || n < 0 || n > kMaxSamples || (n > 0 && (!q || !kappa))) return LB_EINVAL;
    if (!(std::isfinite(kappa_lo) && kappa_lo < kappa_hi && kappa_hi < 1.f))
        return mfail(m, LB_EINVAL, "need kappa_lo < kappa_hi < 1");
    if (n == 0) return LB_OK;
    for (int i = 0; i < n; ++i)
        if (!(finite3(q + 3 * i) && q[3 * i] < 1.f))
            return mfail(m, LB_EINVAL, "need finite queries with T/T_c < 1");
    lb_status s = ensure_io(m, (size_t)n * 4);
    if (s != LB_OK) return s;
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(m->io, q, (size_t)n * 3 * sizeof(float), cudaMemcpyHostToDevice));
    k_mlp_invert<<<(n + 127) / 128, 128, 0, m->stream>>>(m->wbf, m->norm, m->io, n, kappa_lo,
                                                         kappa_hi, m->io + (size_t)n * 3);
    LB_MCUDA(m, cudaGetLastError());
    LB_MCUDA(m, cudaStreamSynchronize(m->stream));
    LB_MCUDA(m, cudaMemcpy(kappa, m->io + (size_t)n * 3, (size_t)n * sizeof(float),
                           cudaMemcpyDeviceToHost));
    return LB_OK;
}

const char *lb_mlp_last_error(const lb_mlp *m) { return m ? m->msg.c_str() : "null network"; }

void lb_mlp_free(lb_mlp *m) {
    if (!m) return;
    cudaStreamSynchronize(m->stream);
    drop_graph(m);
    float *fl[] = {m->master, m->m1, m->m2, m->xn, m->tn, m->part, m->lpart, m->grad, m->io};
    for (float *p : fl)
        if (p) cudaFree(p);
    if (m->wbf) cudaFree(m->wbf);
    if (m->norm) cudaFree(m->norm);
    if (m->st) cudaFree(m->st);
    delete m;
}

}  // extern "C"
