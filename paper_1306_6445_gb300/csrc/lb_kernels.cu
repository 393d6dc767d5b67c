// Kernels of the D2Q9 MRT pseudopotential update with the surface-tension source term
// (Li & Luo, arXiv 1306.6445, Sec. II and IV) for sm_103a.
//
// Storage: populations f_a(x, t) AFTER streaming (pre-collision), as 9 planes of ny rows
// of `pitch` elements, x fastest. One step reads each population once and writes each
// once (push streaming into the second buffer).
//
// Fused step kernel (one launch per time step). Each CTA owns a strip of TX columns and
// marches upward over `rows` rows. The potential psi is recomputed from the populations
// (rho = sum f, then the EOS) and kept for four consecutive rows in a shared-memory ring
// with one halo column on each side, so F (Eq. 7) and Q (Eq. 19) see all eight
// neighbours without a psi array in global memory. A thread prefetches the populations
// two rows ahead into registers; the only extra global reads are the strip's two halo
// columns and the rows just below and above its range (these hit L2).
#include <cuda_runtime.h>

#include <algorithm>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbm {

namespace {

template <typename T, bool WALLS>
__device__ __forceinline__ int psi_row_index(int y, int ny) {
    if (WALLS) return y < 0 ? 0 : (y >= ny ? ny - 1 : y);   // wall rows copy the fluid row
    return y < 0 ? y + ny : (y >= ny ? y - ny : y);          // periodic
}

template <typename T>
__device__ __forceinline__ void load9(T (&v)[9], const T *__restrict__ base, long long plane) {
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = __ldg(base + a * plane);
}

template <typename T>
__device__ __forceinline__ T sum9(const T (&v)[9]) {
    return v[0] + ((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
}

template <typename T, int EOS, bool WALLS, int TX>
__global__ void __launch_bounds__(TX)
k_fused_step(const T *__restrict__ fin, T *__restrict__ fout, const DevConsts<T> P,
             const int nx, const int ny, const int pitch, const long long plane,
             const int rows, int *__restrict__ err) {
    __shared__ T psi_s[4][TX + 2];

    const int tx = threadIdx.x;
    const int x0 = blockIdx.x * TX;
    const int width = min(TX, nx - x0);
    const bool active = tx < width;
    const int x = x0 + (active ? tx : 0);
    const int yb = blockIdx.y * rows;
    const int ye = min(yb + rows, ny);
    const int xl = (x0 == 0) ? nx - 1 : x0 - 1;
    const int xr = (x0 + width >= nx) ? 0 : x0 + width;
    bool bad = false;

    // psi of row y (y may be yb-1 .. ye) into ring slot y & 3: own column from `own`,
    // halo columns by thread 0 (left) and thread TX-1 (right).
    auto psi_row = [&](int y, const T (&own)[9]) {
        const int slot = y & 3;
        const int ry = psi_row_index<T, WALLS>(y, ny);
        if (active) psi_s[slot][tx + 1] = eos_psi<T, EOS>(sum9(own), P, bad);
        if (tx == 0) {
            T h[9];
            load9(h, fin + (long long)ry * pitch + xl, plane);
            psi_s[slot][0] = eos_psi<T, EOS>(sum9(h), P, bad);
        }
        if (tx == TX - 1) {
            T h[9];
            load9(h, fin + (long long)ry * pitch + xr, plane);
            psi_s[slot][width + 1] = eos_psi<T, EOS>(sum9(h), P, bad);
        }
    };

    T fc[9], fn[9];
    {
        T fm[9];
        if (active) load9(fm, fin + (long long)psi_row_index<T, WALLS>(yb - 1, ny) * pitch + x, plane);
        psi_row(yb - 1, fm);
    }
    if (active) load9(fc, fin + (long long)yb * pitch + x, plane);
    psi_row(yb, fc);
    if (active) load9(fn, fin + (long long)psi_row_index<T, WALLS>(yb + 1, ny) * pitch + x, plane);
    psi_row(yb + 1, fn);

    const int xp = (x + 1 == nx) ? 0 : x + 1;
    const int xm = (x == 0) ? nx - 1 : x - 1;

    for (int y = yb; y < ye; ++y) {
        __syncthreads();  // psi rows y-1, y, y+1 are complete
        const bool more = (y + 1 < ye);
        T fnn[9];
        if (more && active)
            load9(fnn, fin + (long long)psi_row_index<T, WALLS>(y + 2, ny) * pitch + x, plane);

        if (active) {
            const int sm = (y - 1) & 3, s0 = y & 3, sp = (y + 1) & 3;
            const int c = tx + 1;
            T pn[9];
            pn[0] = psi_s[s0][c];
            pn[1] = psi_s[s0][c + 1];
            pn[2] = psi_s[sp][c];
            pn[3] = psi_s[s0][c - 1];
            pn[4] = psi_s[sm][c];
            pn[5] = psi_s[sp][c + 1];
            pn[6] = psi_s[sp][c - 1];
            pn[7] = psi_s[sm][c - 1];
            pn[8] = psi_s[sm][c + 1];
            collide_site<T>(fc, pn, P);

            // push streaming (Eq. 4): f*_a(x) -> f_a(x + e_a); half-way bounce-back at walls
            const bool top = WALLS && (y + 1 == ny);
            const bool bottom = WALLS && (y == 0);
            const int yu = (y + 1 == ny) ? 0 : y + 1;
            const int yd = (y == 0) ? ny - 1 : y - 1;
            T *row0 = fout + (long long)y * pitch;
            T *rowu = fout + (long long)yu * pitch;
            T *rowd = fout + (long long)yd * pitch;
            row0[0 * plane + x] = fc[0];
            row0[1 * plane + xp] = fc[1];
            row0[3 * plane + xm] = fc[3];
            if (top) {
                row0[4 * plane + x] = fc[2];
                row0[7 * plane + x] = fc[5];
                row0[8 * plane + x] = fc[6];
            } else {
                rowu[2 * plane + x] = fc[2];
                rowu[5 * plane + xp] = fc[5];
                rowu[6 * plane + xm] = fc[6];
            }
            if (bottom) {
                row0[2 * plane + x] = fc[4];
                row0[5 * plane + x] = fc[7];
                row0[6 * plane + x] = fc[8];
            } else {
                rowd[4 * plane + x] = fc[4];
                rowd[7 * plane + xm] = fc[7];
                rowd[8 * plane + xp] = fc[8];
            }
        }
        if (more) {
            psi_row(y + 2, fnn);
#pragma unroll
            for (int a = 0; a < 9; ++a) {
                fc[a] = fn[a];
                fn[a] = fnn[a];
            }
        }
    }
    if (bad) atomicOr(err, ERR_DOMAIN);
}

// f = M^-1 m_eq(rho, u) (Eq. 3) at every site, computed in double.
template <typename T, int EOS>
__global__ void k_init_feq(const double *__restrict__ rho, const double *__restrict__ ux,
                           const double *__restrict__ uy, T *__restrict__ f, const DevConsts<T> P,
                           int nx, int ny, int pitch, long long plane, int *__restrict__ err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    const double r = rho[i], vx = ux[i], vy = uy[i];
    bool bad = false;
    (void)eos_psi<T, EOS>(T(r), P, bad);
    if (bad) atomicOr(err, ERR_DOMAIN);
    const double v2 = vx * vx + vy * vy;
    double m[9] = {r, r * (-2.0 + 3.0 * v2), r * (1.0 - 3.0 * v2), r * vx, -r * vx,
                   r * vy, -r * vy, r * (vx * vx - vy * vy), r * vx * vy};
    const double a0 = m[0] / 9.0;
    const double ba = a0 - m[1] / 36.0 - m[2] / 18.0;
    const double bd = a0 + m[1] / 18.0 + m[2] / 36.0;
    double o[9];
    o[0] = a0 - m[1] / 9.0 + m[2] / 9.0;
    o[1] = ba + m[3] / 6.0 - m[4] / 6.0 + m[7] / 4.0;
    o[3] = ba - m[3] / 6.0 + m[4] / 6.0 + m[7] / 4.0;
    o[2] = ba + m[5] / 6.0 - m[6] / 6.0 - m[7] / 4.0;
    o[4] = ba - m[5] / 6.0 + m[6] / 6.0 - m[7] / 4.0;
    o[5] = bd + m[3] / 6.0 + m[4] / 12.0 + m[5] / 6.0 + m[6] / 12.0 + m[8] / 4.0;
    o[6] = bd - m[3] / 6.0 - m[4] / 12.0 + m[5] / 6.0 + m[6] / 12.0 - m[8] / 4.0;
    o[7] = bd - m[3] / 6.0 - m[4] / 12.0 - m[5] / 6.0 - m[6] / 12.0 + m[8] / 4.0;
    o[8] = bd + m[3] / 6.0 + m[4] / 12.0 - m[5] / 6.0 - m[6] / 12.0 - m[8] / 4.0;
    T *p = f + (long long)y * pitch + x;
#pragma unroll
    for (int a = 0; a < 9; ++a) p[a * plane] = T(o[a]);
}

// psi(rho(x)) in double for the diagnostics.
template <typename T, int EOS>
__global__ void k_psi_field(const T *__restrict__ f, double *__restrict__ psi,
                            const DevConsts<double> P, int nx, int ny, int pitch, long long plane,
                            int *__restrict__ err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    const T *p = f + (long long)y * pitch + x;
    double r = 0.0;
    double v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = double(p[a * plane]);
    r = v[0] + ((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
    bool bad = false;
    psi[i] = eos_psi<double, EOS>(r, P, bad);
    if (bad) atomicOr(err, ERR_DOMAIN);
}

// rho and v = (sum e f + F/2)/rho (Eq. 6) of one site, in double, from f and the psi field.
template <typename T, bool WALLS>
__device__ __forceinline__ void site_macro(const T *__restrict__ f, const double *__restrict__ psi,
                                           double G, int nx, int ny, int pitch, long long plane,
                                           int x, int y, double &rho, double &vx, double &vy) {
    const T *p = f + (long long)y * pitch + x;
    double v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = double(p[a * plane]);
    rho = v[0] + ((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
    const double jx = (v[1] - v[3]) + (v[5] - v[7]) - (v[6] - v[8]);
    const double jy = (v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]);
    const int xp = (x + 1 == nx) ? 0 : x + 1, xm = (x == 0) ? nx - 1 : x - 1;
    int yp, ym;
    if (WALLS) {
        yp = (y + 1 == ny) ? y : y + 1;
        ym = (y == 0) ? 0 : y - 1;
    } else {
        yp = (y + 1 == ny) ? 0 : y + 1;
        ym = (y == 0) ? ny - 1 : y - 1;
    }
    auto ps = [&](int xx, int yy) { return psi[(long long)yy * nx + xx]; };
    const double pc = ps(x, y);
    const double sx = (ps(xp, y) - ps(xm, y)) / 3.0 +
                      ((ps(xp, yp) - ps(xm, ym)) - (ps(xm, yp) - ps(xp, ym))) / 12.0;
    const double sy = (ps(x, yp) - ps(x, ym)) / 3.0 +
                      ((ps(xp, yp) - ps(xm, ym)) + (ps(xm, yp) - ps(xp, ym))) / 12.0;
    const double Fx = -G * pc * sx, Fy = -G * pc * sy;
    vx = (jx + 0.5 * Fx) / rho;
    vy = (jy + 0.5 * Fy) / rho;
}

template <typename T, bool WALLS>
__global__ void k_macro_fields(const T *__restrict__ f, const double *__restrict__ psi, double G,
                               int nx, int ny, int pitch, long long plane,
                               double *__restrict__ rho, double *__restrict__ ux,
                               double *__restrict__ uy) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    if (!ux && !uy) {  // density only: psi is not needed
        const T *p = f + (long long)y * pitch + x;
        double v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = double(p[a * plane]);
        rho[i] = v[0] + ((v[1] + v[3]) + (v[2] + v[4])) + ((v[5] + v[7]) + (v[6] + v[8]));
        return;
    }
    double r, vx, vy;
    site_macro<T, WALLS>(f, psi, G, nx, ny, pitch, plane, x, y, r, vx, vy);
    if (rho) rho[i] = r;
    if (ux) ux[i] = vx;
    if (uy) uy[i] = vy;
}

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

// Block b reduces the contiguous site range [b*chunk, (b+1)*chunk) with a fixed
// per-thread order and a fixed shared-memory tree: the result does not depend on timing.
template <typename T, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS)
k_macro_reduce(const T *__restrict__ f, const double *__restrict__ psi, double G, int nx, int ny,
               int pitch, long long plane, long long chunk, double *__restrict__ partials) {
    __shared__ double s[4][RED_THREADS];
    const long long n = (long long)nx * ny;
    const long long beg = blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    double m = 0, px = 0, py = 0, vmax = 0;
    for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        double r, vx, vy;
        site_macro<T, WALLS>(f, psi, G, nx, ny, pitch, plane, x, y, r, vx, vy);
        m += r;
        px += r * vx;
        py += r * vy;
        const double sp = sqrt(vx * vx + vy * vy);
        vmax = (sp > vmax || sp != sp) ? sp : vmax;  // NaN propagates
    }
    s[0][threadIdx.x] = m;
    s[1][threadIdx.x] = px;
    s[2][threadIdx.x] = py;
    s[3][threadIdx.x] = vmax;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
            const double o = s[3][threadIdx.x + w];
            const double c = s[3][threadIdx.x];
            s[3][threadIdx.x] = (o > c || o != o) ? o : c;
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

__global__ void __launch_bounds__(RED_THREADS)
k_reduce_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
    __shared__ double s[4][RED_THREADS];
    double m = 0, px = 0, py = 0, vmax = 0;
    for (int b = threadIdx.x; b < nblocks; b += RED_THREADS) {
        m += partials[b * 4 + 0];
        px += partials[b * 4 + 1];
        py += partials[b * 4 + 2];
        const double o = partials[b * 4 + 3];
        vmax = (o > vmax || o != o) ? o : vmax;
    }
    s[0][threadIdx.x] = m;
    s[1][threadIdx.x] = px;
    s[2][threadIdx.x] = py;
    s[3][threadIdx.x] = vmax;
    __syncthreads();
    for (int w = RED_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s[0][threadIdx.x] += s[0][threadIdx.x + w];
            s[1][threadIdx.x] += s[1][threadIdx.x + w];
            s[2][threadIdx.x] += s[2][threadIdx.x + w];
            const double o = s[3][threadIdx.x + w];
            const double c = s[3][threadIdx.x];
            s[3][threadIdx.x] = (o > c || o != o) ? o : c;
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

// ---- dispatch helpers ------------------------------------------------------------------

template <typename T, int TX>
cudaError_t step_dispatch(const Consts &c, const Geom &g, const StepLaunch &l, const void *fin,
                          void *fout, int *err, cudaStream_t st) {
    const DevConsts<T> P = to_dev<T>(c);
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + l.rows - 1) / l.rows);
    const T *in = static_cast<const T *>(fin);
    T *out = static_cast<T *>(fout);
#define LB_STEP_CASE(EOSK, W)                                                              \
    k_fused_step<T, EOSK, W, TX><<<grid, TX, 0, st>>>(in, out, P, g.nx, g.ny, g.pitch,      \
                                                       g.plane, l.rows, err)
    const bool w = g.walls != 0;
    switch (c.eos_kind) {
        case LB_EOS_CS:
            if (w) LB_STEP_CASE(LB_EOS_CS, true); else LB_STEP_CASE(LB_EOS_CS, false);
            break;
        case LB_EOS_EXP:
            if (w) LB_STEP_CASE(LB_EOS_EXP, true); else LB_STEP_CASE(LB_EOS_EXP, false);
            break;
        default:
            if (w) LB_STEP_CASE(LB_EOS_PIECEWISE, true); else LB_STEP_CASE(LB_EOS_PIECEWISE, false);
            break;
    }
#undef LB_STEP_CASE
    return cudaGetLastError();
}

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

StepLaunch default_step_launch(const Geom &g, int num_sms) {
    StepLaunch l;
    l.tx = 128;
    const long long strips = (g.nx + l.tx - 1) / l.tx;
    const long long target = (long long)std::max(num_sms, 1) * 8;
    long long rows = (g.ny * strips + target - 1) / target;
    rows = std::max<long long>(rows, 4);
    rows = std::min<long long>(rows, g.ny);
    l.rows = (int)rows;
    return l;
}

cudaError_t launch_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l,
                        const void *fin, void *fout, int *err, cudaStream_t st) {
    if (l.tx != 128) return cudaErrorInvalidValue;
    if (prec == LB_FP32) return step_dispatch<float, 128>(c, g, l, fin, fout, err, st);
    return step_dispatch<double, 128>(c, g, l, fin, fout, err, st);
}

cudaError_t launch_init_feq(int prec, const Consts &c, const Geom &g, const double *rho,
                            const double *ux, const double *uy, void *f, int *err,
                            cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const unsigned nb = blocks_for(n, 256);
#define LB_INIT(T, EOSK)                                                                   \
    k_init_feq<T, EOSK><<<nb, 256, 0, st>>>(rho, ux, uy, static_cast<T *>(f), to_dev<T>(c), \
                                            g.nx, g.ny, g.pitch, g.plane, err)
    if (prec == LB_FP32) {
        if (c.eos_kind == LB_EOS_CS) LB_INIT(float, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_INIT(float, LB_EOS_EXP);
        else LB_INIT(float, LB_EOS_PIECEWISE);
    } else {
        if (c.eos_kind == LB_EOS_CS) LB_INIT(double, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_INIT(double, LB_EOS_EXP);
        else LB_INIT(double, LB_EOS_PIECEWISE);
    }
#undef LB_INIT
    return cudaGetLastError();
}

cudaError_t launch_psi_field(int prec, const Consts &c, const Geom &g, const void *f,
                             double *psi, int *err, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const unsigned nb = blocks_for(n, 256);
    const DevConsts<double> P = to_dev<double>(c);
#define LB_PSI(T, EOSK)                                                                    \
    k_psi_field<T, EOSK><<<nb, 256, 0, st>>>(static_cast<const T *>(f), psi, P, g.nx, g.ny, \
                                             g.pitch, g.plane, err)
    if (prec == LB_FP32) {
        if (c.eos_kind == LB_EOS_CS) LB_PSI(float, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_PSI(float, LB_EOS_EXP);
        else LB_PSI(float, LB_EOS_PIECEWISE);
    } else {
        if (c.eos_kind == LB_EOS_CS) LB_PSI(double, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_PSI(double, LB_EOS_EXP);
        else LB_PSI(double, LB_EOS_PIECEWISE);
    }
#undef LB_PSI
    return cudaGetLastError();
}

cudaError_t launch_macro_fields(int prec, const Consts &c, const Geom &g, const void *f,
                                const double *psi, double *rho, double *ux, double *uy,
                                cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const unsigned nb = blocks_for(n, 256);
#define LB_MAC(T, W)                                                                       \
    k_macro_fields<T, W><<<nb, 256, 0, st>>>(static_cast<const T *>(f), psi, c.G, g.nx, g.ny, \
                                             g.pitch, g.plane, rho, ux, uy)
    if (prec == LB_FP32) {
        if (g.walls) LB_MAC(float, true); else LB_MAC(float, false);
    } else {
        if (g.walls) LB_MAC(double, true); else LB_MAC(double, false);
    }
#undef LB_MAC
    return cudaGetLastError();
}

int reduce_blocks(long long n_sites) {
    long long nb = (n_sites + RED_THREADS * 4 - 1) / (RED_THREADS * 4);
    return (int)std::max<long long>(1, std::min<long long>(nb, RED_MAX_BLOCKS));
}

cudaError_t launch_macro_reduce(int prec, const Consts &c, const Geom &g, const void *f,
                                const double *psi, double *partials, double *out4,
                                cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const int nb = reduce_blocks(n);
    const long long chunk = (n + nb - 1) / nb;
#define LB_RED(T, W)                                                                         \
    k_macro_reduce<T, W><<<nb, RED_THREADS, 0, st>>>(static_cast<const T *>(f), psi, c.G, g.nx, \
                                                     g.ny, g.pitch, g.plane, chunk, partials)
    if (prec == LB_FP32) {
        if (g.walls) LB_RED(float, true); else LB_RED(float, false);
    } else {
        if (g.walls) LB_RED(double, true); else LB_RED(double, false);
    }
#undef LB_RED
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, RED_THREADS, 0, st>>>(partials, nb, out4);
    return cudaGetLastError();
}

}  // namespace lbm
