// lb_reduce_noalloc: the diagnostics reduction of lb_reduce (mass, momentum, max |v|)
// for callers that cannot allocate device memory, for example a plugin that must stay
// inside a device-memory budget handed to it by its host application, or a loop that must
// not call cudaMalloc/cudaFree because those may synchronise the whole device. It
// allocates nothing: its scratch is the file-scope array below, which every GPU that
// loads this library holds until the process exits.
//
// Differences from lb_reduce (which stores a psi field and allocates its partial sums on
// first use): psi at a site's eight neighbours is recomputed from their populations, so
// the only scratch is the per-block partial sums, the final four values and an error
// word. The block split and per-thread order are those of lb_reduce, and the per-site
// arithmetic is the same, so the two usually agree to the last bit.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <type_traits>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace {

using lbm::DevConsts;

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = 1024;
constexpr long long NA_MAX_SITES = 1LL << 24;   // each block then sums at most 16384 sites
constexpr int NA_OUT = 4 * NA_MAX_BLOCKS;        // [NA_OUT, NA_OUT + 4): final results
constexpr int NA_ERR = NA_OUT + 4;               // error bits (as an integer word)
constexpr int NA_DOUBLES = NA_ERR + 4;

// The scratch: 4104 doubles (32.8 KB) per GPU, shared by every call.
static __device__ __align__(256) double lb_noalloc_scratch[NA_DOUBLES];

template <typename T>
constexpr int GHOST = lbm::ghost_of_prec(std::is_same<T, float>::value ? LB_FP32 : LB_FP64);

__device__ __forceinline__ int na_opp(int a) {
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5);
}
__device__ __forceinline__ int na_ex(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__device__ __forceinline__ int na_ey(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}

// population a of site (x, y) at the current time, pulled from the stored state
template <typename T, bool WALLS>
__device__ __forceinline__ T na_pull(const T *__restrict__ g, int a, int x, int y, int nx, int ny,
                                     int pitch, long long plane) {
    int sy = y - na_ey(a);
    if (WALLS && (sy < 0 || sy >= ny))
        return g[lbm::plane_of(na_opp(a)) * plane + (long long)y * pitch + x + GHOST<T>];
    if (!WALLS) sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
    int sx = x - na_ex(a);
    sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
    return g[lbm::plane_of(a) * plane + (long long)sy * pitch + sx + GHOST<T>];
}

template <typename T, bool WALLS>
__device__ __forceinline__ void na_pops(const T *__restrict__ g, int x, int y, int nx, int ny,
                                        int pitch, long long plane, T (&v)[9]) {
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = na_pull<T, WALLS>(g, a, x, y, nx, ny, pitch, plane);
}

template <typename T>
__device__ __forceinline__ T na_sum9(const T (&v)[9]) {
    using lbm::radd;
    return radd(v[0], radd(radd(radd(v[1], v[3]), radd(v[2], v[4])),
                           radd(radd(v[5], v[7]), radd(v[6], v[8]))));
}

template <typename T, int EOS, bool WALLS>
__device__ __forceinline__ T na_psi(const T *__restrict__ g, const DevConsts<T> &P, int x, int y,
                                    int nx, int ny, int pitch, long long plane, bool &bad) {
    T v[9];
    na_pops<T, WALLS>(g, x, y, nx, ny, pitch, plane, v);
    return lbm::eos_psi<T, EOS>(na_sum9(v), P, bad);
}

// Block b sums sites [b*chunk, (b+1)*chunk) in the same order as lb_reduce and writes its
// four partials to scratch[4b .. 4b+3]; a psi-domain violation sets scratch[NA_ERR].
template <typename T, int EOS, bool WALLS>
__global__ void __launch_bounds__(NA_THREADS)
k_na_partials(const T *__restrict__ g, const DevConsts<T> P, int nx, int ny, int pitch,
              long long plane, long long chunk, double *__restrict__ scratch) {
    __shared__ double s[4][NA_THREADS];
    const long long n = (long long)nx * ny;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    double m = 0, px = 0, py = 0, vmax = 0;
    bool bad = false;
    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0);
    for (long long i = beg + threadIdx.x; i < end; i += NA_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        T v[9];
        na_pops<T, WALLS>(g, x, y, nx, ny, pitch, plane, v);
        const T r = na_sum9(v);
        const T jx = (v[1] - v[3]) + (v[5] - v[7]) - (v[6] - v[8]);
        const T jy = (v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]);
        const int xp = (x + 1 == nx) ? 0 : x + 1, xm = (x == 0) ? nx - 1 : x - 1;
        int yp, ym;
        if (WALLS) {
            yp = (y + 1 == ny) ? y : y + 1;
            ym = (y == 0) ? 0 : y - 1;
        } else {
            yp = (y + 1 == ny) ? 0 : y + 1;
            ym = (y == 0) ? ny - 1 : y - 1;
        }
        auto ps = [&](int xx, int yy) {
            return na_psi<T, EOS, WALLS>(g, P, xx, yy, nx, ny, pitch, plane, bad);
        };
        const T pc = ps(x, y);
        const T p_xp = ps(xp, y), p_xm = ps(xm, y), p_yp = ps(x, yp), p_ym = ps(x, ym);
        const T p_pp = ps(xp, yp), p_mm = ps(xm, ym), p_mp = ps(xm, yp), p_pm = ps(xp, ym);
        const T sx = (p_xp - p_xm) * third + ((p_pp - p_mm) - (p_mp - p_pm)) * twelfth;
        const T sy = (p_yp - p_ym) * third + ((p_pp - p_mm) + (p_mp - p_pm)) * twelfth;
        const T Fx = -P.G * pc * sx, Fy = -P.G * pc * sy;
        const T rinv = T(1) / r;
        const T vx = (jx + T(0.5) * Fx) * rinv;
        const T vy = (jy + T(0.5) * Fy) * rinv;
        const double dr = r, dvx = vx, dvy = vy;
        m += dr;
        px += dr * dvx;
        py += dr * dvy;
        const double sp = sqrt(dvx * dvx + dvy * dvy);
        vmax = (sp > vmax || sp != sp) ? sp : vmax;
    }
    if (bad) atomicOr(reinterpret_cast<unsigned long long *>(scratch + NA_ERR), 1ull);
    s[0][threadIdx.x] = m;
    s[1][threadIdx.x] = px;
    s[2][threadIdx.x] = py;
    s[3][threadIdx.x] = vmax;
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
            const double o = s[3][threadIdx.x + w], c = s[3][threadIdx.x];
            s[3][threadIdx.x] = (o > c || o != o) ? o : c;
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) scratch[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void __launch_bounds__(NA_THREADS)
k_na_final(double *__restrict__ scratch, int nblocks) {
    __shared__ double s[4][NA_THREADS];
    double m = 0, px = 0, py = 0, vmax = 0;
    for (int b = threadIdx.x; b < nblocks; b += NA_THREADS) {
        m += scratch[b * 4 + 0];
        px += scratch[b * 4 + 1];
        py += scratch[b * 4 + 2];
        const double o = scratch[b * 4 + 3];
        vmax = (o > vmax || o != o) ? o : vmax;
    }
    s[0][threadIdx.x] = m;
    s[1][threadIdx.x] = px;
    s[2][threadIdx.x] = py;
    s[3][threadIdx.x] = vmax;
    __syncthreads();
    for (int w = NA_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
            const double o = s[3][threadIdx.x + w], c = s[3][threadIdx.x];
            s[3][threadIdx.x] = (o > c || o != o) ? o : c;
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) scratch[NA_OUT + threadIdx.x] = s[threadIdx.x][0];
}

template <typename T, int EOS, bool WALLS>
void na_launch(const lbm::CtxView &v, double *scratch, int nb, long long chunk) {
    k_na_partials<T, EOS, WALLS><<<nb, NA_THREADS, 0, v.stream>>>(
        static_cast<const T *>(v.g), lbm::to_dev<T>(v.consts), v.geom.nx, v.geom.ny, v.geom.pitch,
        v.geom.plane, chunk, scratch);
}

template <typename T>
void na_launch_eos(const lbm::CtxView &v, double *scratch, int nb, long long chunk) {
    const bool w = v.geom.walls != 0;
    switch (v.consts.eos_kind) {
        case LB_EOS_CS:
            w ? na_launch<T, LB_EOS_CS, true>(v, scratch, nb, chunk)
              : na_launch<T, LB_EOS_CS, false>(v, scratch, nb, chunk);
            break;
        case LB_EOS_EXP:
            w ? na_launch<T, LB_EOS_EXP, true>(v, scratch, nb, chunk)
              : na_launch<T, LB_EOS_EXP, false>(v, scratch, nb, chunk);
            break;
        default:
            w ? na_launch<T, LB_EOS_PIECEWISE, true>(v, scratch, nb, chunk)
              : na_launch<T, LB_EOS_PIECEWISE, false>(v, scratch, nb, chunk);
            break;
    }
}

// Device address of lb_noalloc_scratch, looked up once per device (the host-side name
// of the array is only a stand-in and must never be handed to a kernel).
constexpr int NA_MAX_DEVICES = 64;
std::mutex na_mutex;
double *na_addr[NA_MAX_DEVICES] = {};

cudaError_t scratch_address(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(na_mutex);
    if (!na_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, lb_noalloc_scratch);   // the current device is `dev`
        if (e != cudaSuccess) return e;
        na_addr[dev] = static_cast<double *>(p);
    }
    *out = na_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" lb_status lb_reduce_noalloc(lb_ctx *ctx, double out[4]) {
    lbm::CtxView v;
    if (!ctx || !out) return LB_EINVAL;
    if (lbm::ctx_view(ctx, &v) != LB_OK) return LB_EINVAL;
    if (v.sticky != LB_OK) return v.sticky;
    if (v.prec == LB_BF16 || v.geom.walls == LB_BC_OPEN)
        return lbm::ctx_fail(ctx, LB_EINVAL,
                             "lb_reduce_noalloc: LB_BF16 and LB_BC_OPEN contexts use lb_reduce",
                             false);
    const long long n = (long long)v.geom.nx * v.geom.ny;
    if (n > NA_MAX_SITES) {
        char msg[160];
        std::snprintf(msg, sizeof msg,
                      "lb_reduce_noalloc: the lattice has %lld sites; this entry point handles at "
                      "most %lld (use lb_reduce)", n, NA_MAX_SITES);
        return lbm::ctx_fail(ctx, LB_EINVAL, msg, false);
    }
    double *scratch = nullptr;
    cudaError_t e = scratch_address(&scratch);
    if (e != cudaSuccess)
        return lbm::ctx_fail(ctx, LB_ECUDA, cudaGetErrorString(e), false);
    // same block split as lb_reduce
    long long nbl = (n + NA_THREADS * 4 - 1) / (NA_THREADS * 4);
    const int nb = (int)(nbl < 1 ? 1 : (nbl > NA_MAX_BLOCKS ? NA_MAX_BLOCKS : nbl));
    const long long chunk = (n + nb - 1) / nb;
    // the error word must start at zero; partials and results are fully rewritten
    e = cudaMemsetAsync(scratch + NA_ERR, 0, sizeof(double), v.stream);
    if (e == cudaSuccess) {
        if (v.prec == LB_FP32) na_launch_eos<float>(v, scratch, nb, chunk);
        else na_launch_eos<double>(v, scratch, nb, chunk);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        k_na_final<<<1, NA_THREADS, 0, v.stream>>>(scratch, nb);
        e = cudaGetLastError();
    }
    double res[5];
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(res, scratch + NA_OUT, 5 * sizeof(double), cudaMemcpyDeviceToHost,
                            v.stream);
    if (e != cudaSuccess) return lbm::ctx_fail(ctx, LB_ECUDA, cudaGetErrorString(e), false);
    // wait, then take the context's own error word as lb_reduce does: a bounded wait that
    // gave up (LB_ETIMEOUT) or a psi-domain violation in a step queued before this call
    // (LB_EDOMAIN) poisons the context and is returned instead of the sums
    const lb_status s = lbm::ctx_sync_check(ctx);
    if (s != LB_OK) return s;
    unsigned long long flags;
    static_assert(sizeof(flags) == sizeof(double), "error word layout");
    std::memcpy(&flags, &res[4], sizeof flags);
    if (flags & 1ull)
        return lbm::ctx_fail(ctx, LB_EDOMAIN,
                             "psi^2 < 0 or rho <= 0 at some site (EOS domain left)", true);
    for (int i = 0; i < 4; ++i) {
        if (!std::isfinite(res[i]))
            return lbm::ctx_fail(ctx, LB_ENONFINITE,
                                 "lb_reduce_noalloc: non-finite mass, momentum or |v|", true);
        out[i] = res[i];
    }
    return LB_OK;
}
