// Auxiliary kernels of the library (permutations between the stored and the natural
// population layout, equilibrium initialisation, diagnostics and reductions) and the
// public launch functions; the step kernels live in the per-precision units.
#include "lb_step.cuh"

namespace lbm {

namespace {

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// launch X(T, BC) for the geometry's boundary kind
#define BC3(X, T)                       \
    do {                                \
        if (g.walls == 2) X(T, 2);      \
        else if (g.walls == 1) X(T, 1); \
        else X(T, 0);                   \
    } while (0)

// ---------------------------------------------------------------- permutations

// Element of population b at (x, y) in f: the padded layout (pitch, ghost offset), or,
// PACKED, the host layout [b][y][x] without padding.
template <typename T, bool PACKED>
__device__ __forceinline__ long long f_index(int b, int x, int y, int nx, int ny, int pitch,
                                             long long plane) {
    if (PACKED) return ((long long)b * ny + y) * nx + x;
    return b * plane + (long long)y * pitch + x + GH<T>;
}

// g_b(y) = f_b(y + e_b) where y + e_b is inside the lattice, else f_opp(b)(y) at a wall
// (inverse of the pull with bounce-back); a population leaving through an open boundary
// (BC 2) is not pulled back by any site and keeps f_b(y). g uses the padded layout and its
// ghost columns are written (periodic images, or copies of the edge columns); f is padded
// or packed (PACKED).
template <typename T, int BC, bool PACKED>
__global__ void k_unstream(const T *__restrict__ f, T *__restrict__ g, int nx, int ny, int pitch,
                           long long plane) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        int ty = y + EYv(b), tx = x + EXv(b);
        T v;
        if ((BC != 0 && ty < 0) || (BC == 1 && ty >= ny)) {
            v = f[f_index<T, PACKED>(opp(b), x, y, nx, ny, pitch, plane)];
        } else if (BC == 2 && (ty >= ny || tx < 0 || tx >= nx)) {
            v = f[f_index<T, PACKED>(b, x, y, nx, ny, pitch, plane)];
        } else {
            if (BC == 0) ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
            tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
            v = f[f_index<T, PACKED>(b, tx, ty, nx, ny, pitch, plane)];
        }
        T *rowg = g + plane_of(b) * plane + (long long)y * pitch;
        rowg[x + GH<T>] = v;
        if (BC == 2) {
            if (x == 0) rowg[GH<T> - 1] = rowg[GH<T> - 2] = v;
            if (x == nx - 1) rowg[nx + GH<T>] = rowg[nx + GH<T> + 1] = v;
        } else {
            if (x < 2) rowg[nx + GH<T> + x] = v;
            if (x >= nx - 2) rowg[x - nx + GH<T>] = v;
        }
    }
}

// f_a(x) = pull of g (the populations of the current time), into the padded layout (no
// ghosts) or, PACKED, the host layout.
template <typename T, int BC, bool PACKED>
__global__ void k_stream(const T *__restrict__ g, T *__restrict__ f, int nx, int ny, int pitch,
                         long long plane) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
#pragma unroll
    for (int a = 0; a < 9; ++a)
        f[f_index<T, PACKED>(a, x, y, nx, ny, pitch, plane)] =
            pull_global<T, BC>(g, a, x, y, nx, ny, pitch, plane);
}

// f = M^-1 m_eq(rho, u) (Eq. 3) at every site, computed in double, in the padded layout.
template <typename T, int EOS>
__global__ void k_init_feq(const double *__restrict__ rho, const double *__restrict__ ux,
                           const double *__restrict__ uy, T *__restrict__ f,
                           const DevConsts<Arith<T>> P,
                           int nx, int ny, int pitch, long long plane, int *__restrict__ err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    const double r = rho[i], vx = ux[i], vy = uy[i];
    bool bad = false;
    (void)eos_psi<Arith<T>, EOS>(Arith<T>(r), P, bad);
    if (bad) atomicOr(err, ERR_DOMAIN);
    const double v2 = vx * vx + vy * vy;
    const double m[9] = {r, r * (-2.0 + 3.0 * v2), r * (1.0 - 3.0 * v2), r * vx, -r * vx,
                         r * vy, -r * vy, r * (vx * vx - vy * vy), r * vx * vy};
    const double i9 = 1.0 / 9.0, i18 = 1.0 / 18.0, i36 = 1.0 / 36.0, i6 = 1.0 / 6.0,
                 i12 = 1.0 / 12.0;
    const double a0 = m[0] * i9;
    const double ba = a0 - m[1] * i36 - m[2] * i18;
    const double bd = a0 + m[1] * i18 + m[2] * i36;
    double o[9];
    o[0] = a0 - m[1] * i9 + m[2] * i9;
    o[1] = ba + m[3] * i6 - m[4] * i6 + m[7] * 0.25;
    o[3] = ba - m[3] * i6 + m[4] * i6 + m[7] * 0.25;
    o[2] = ba + m[5] * i6 - m[6] * i6 - m[7] * 0.25;
    o[4] = ba - m[5] * i6 + m[6] * i6 - m[7] * 0.25;
    o[5] = bd + m[3] * i6 + m[4] * i12 + m[5] * i6 + m[6] * i12 + m[8] * 0.25;
    o[6] = bd - m[3] * i6 - m[4] * i12 + m[5] * i6 + m[6] * i12 - m[8] * 0.25;
    o[7] = bd - m[3] * i6 - m[4] * i12 - m[5] * i6 - m[6] * i12 + m[8] * 0.25;
    o[8] = bd + m[3] * i6 + m[4] * i12 - m[5] * i6 - m[6] * i12 - m[8] * 0.25;
    T *p = f + (long long)y * pitch + x + GH<T>;
#pragma unroll
    for (int a = 0; a < 9; ++a) p[a * plane] = pop_enc<T>(Arith<T>(o[a]), a, P);
}

// ---------------------------------------------------------------- diagnostics

// psi(rho(x)) in the arithmetic type, into a packed nx*ny array.
template <typename T, int EOS, int BC>
__global__ void k_psi_field(const T *__restrict__ g, Arith<T> *__restrict__ psi,
                            const DevConsts<Arith<T>> P, int nx, int ny, int pitch,
                            long long plane, int *__restrict__ err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    Arith<T> v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = pull_val<T, BC>(g, a, x, y, nx, ny, pitch, plane, P);
    bool bad = false;
    psi[i] = eos_psi<Arith<T>, EOS>(sum9(v), P, bad);
    if (bad) atomicOr(err, ERR_DOMAIN);
}

// rho and v = (sum e f + F/2)/rho (Eq. 6) of one site, from g and the psi field.
template <typename T, int BC, typename A = Arith<T>>
__device__ __forceinline__ void site_macro(const T *__restrict__ g, const A *__restrict__ psi,
                                           const DevConsts<A> &P, int nx, int ny, int pitch,
                                           long long plane, int x, int y, A &rho, A &vx, A &vy) {
    const A G = P.G;
    A v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = pull_val<T, BC>(g, a, x, y, nx, ny, pitch, plane, P);
    rho = sum9(v);
    const A jx = (v[1] - v[3]) + (v[5] - v[7]) - (v[6] - v[8]);
    const A jy = (v[2] - v[4]) + (v[5] - v[7]) + (v[6] - v[8]);
    int xp = (x + 1 == nx) ? 0 : x + 1, xm = (x == 0) ? nx - 1 : x - 1;
    if (BC == 2) {   // open sides: psi beyond the lattice is that of the edge column
        xp = (x + 1 == nx) ? x : x + 1;
        xm = (x == 0) ? 0 : x - 1;
    }
    int yp, ym;
    if (BC != 0) {
        yp = (y + 1 == ny) ? y : y + 1;
        ym = (y == 0) ? 0 : y - 1;
    } else {
        yp = (y + 1 == ny) ? 0 : y + 1;
        ym = (y == 0) ? ny - 1 : y - 1;
    }
    auto ps = [&](int xx, int yy) { return psi[(long long)yy * nx + xx]; };
    const A third = A(1.0 / 3.0), twelfth = A(1.0 / 12.0);
    const A pc = ps(x, y);
    const A sx = (ps(xp, y) - ps(xm, y)) * third +
                 ((ps(xp, yp) - ps(xm, ym)) - (ps(xm, yp) - ps(xp, ym))) * twelfth;
    const A sy = (ps(x, yp) - ps(x, ym)) * third +
                 ((ps(xp, yp) - ps(xm, ym)) + (ps(xm, yp) - ps(xp, ym))) * twelfth;
    const A Fx = -G * pc * sx, Fy = -G * pc * sy;
    const A rinv = A(1) / rho;
    vx = (jx + A(0.5) * Fx) * rinv;
    vy = (jy + A(0.5) * Fy) * rinv;
}

template <typename T, int BC>
__global__ void k_macro_fields(const T *__restrict__ g, const Arith<T> *__restrict__ psi,
                               const DevConsts<Arith<T>> P, int nx, int ny, int pitch,
                               long long plane, double *__restrict__ rho,
                               double *__restrict__ ux, double *__restrict__ uy) {
    using A = Arith<T>;
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    if (!ux && !uy) {  // density only: psi is not needed
        A v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = pull_val<T, BC>(g, a, x, y, nx, ny, pitch, plane, P);
        rho[i] = double(sum9(v));
        return;
    }
    A r, vx, vy;
    site_macro<T, BC>(g, psi, P, nx, ny, pitch, plane, x, y, r, vx, vy);
    if (rho) rho[i] = double(r);
    if (ux) ux[i] = double(vx);
    if (uy) uy[i] = double(vy);
}


// Block b reduces the contiguous site range [b*chunk, (b+1)*chunk) in FP64 with a fixed
// per-thread order and a fixed shared-memory tree: the result does not depend on timing.
template <typename T, int BC>
__global__ void __launch_bounds__(RED_THREADS)
k_macro_reduce(const T *__restrict__ g, const Arith<T> *__restrict__ psi,
               const DevConsts<Arith<T>> P, int nx, int ny, int pitch, long long plane,
               long long chunk, double *__restrict__ partials) {
    __shared__ double s[4][RED_THREADS];
    const long long n = (long long)nx * ny;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    double m = 0, px = 0, py = 0, vmax = 0;
    for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        Arith<T> r, vx, vy;
        site_macro<T, BC>(g, psi, P, nx, ny, pitch, plane, x, y, r, vx, vy);
        const double dr = r, dvx = vx, dvy = vy;
        m += dr;
        px += dr * dvx;
        py += dr * dvy;
        const double sp = sqrt(dvx * dvx + dvy * dvy);
        vmax = (sp > vmax || sp != sp) ? sp : vmax;  // NaN propagates
    }
    s[0][threadIdx.x] = m;
    s[1][threadIdx.x] = px;
    s[2][threadIdx.x] = py;
    s[3][threadIdx.x] = vmax;
    __syncthreads();
    for (int wdt = RED_THREADS / 2; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
            s[0][threadIdx.x] += s[0][threadIdx.x + wdt];
            s[1][threadIdx.x] += s[1][threadIdx.x + wdt];
            s[2][threadIdx.x] += s[2][threadIdx.x + wdt];
            const double o = s[3][threadIdx.x + wdt];
            const double c = s[3][threadIdx.x];
            s[3][threadIdx.x] = (o > c || o != o) ? o : c;
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) partials[blockIdx.x * 4 + threadIdx.x] = s[threadIdx.x][0];
}

// Laplace-law sums of a droplet (Sec. V.A): block b sums the site range [b*chunk,
// (b+1)*chunk) with a fixed per-thread order and a fixed tree. q[0] mass, q[1] / q[2] sum
// of rho / count over r < r_in, q[3] / q[4] over r > r_out, q[5] / q[6] sum of the bulk
// pressure p = rho/3 + (G/2) psi^2 inside / outside, q[7] sites with a non-finite rho or p
// or psi off its real branch; r is the distance from (cx, cy).
template <typename T, int EOS, int BC>
__global__ void __launch_bounds__(RED_THREADS)
k_droplet_sums(const T *__restrict__ g, const DevConsts<Arith<T>> P, int nx, int ny, int pitch,
               long long plane, long long chunk, double cx, double cy, double r_in,
               double r_out, double *__restrict__ partials) {
    using A = Arith<T>;
    __shared__ double s[8][RED_THREADS];
    const long long n = (long long)nx * ny;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        A v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = pull_val<T, BC>(g, a, x, y, nx, ny, pitch, plane, P);
        const A rho = sum9(v);
        bool bad = false;
        const A psi = eos_psi<A, EOS>(rho, P, bad);
        const double dr = double(rho);
        const double pr = dr / 3.0 + 0.5 * double(P.G) * double(psi) * double(psi);
        q[0] += dr;
        const double r = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
        if (r < r_in) { q[1] += dr; q[2] += 1; q[5] += pr; }
        if (r > r_out) { q[3] += dr; q[4] += 1; q[6] += pr; }
        if (bad || !(dr == dr) || !(pr == pr)) q[7] += 1;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k][threadIdx.x] = q[k];
    __syncthreads();
    for (int wdt = RED_THREADS / 2; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + wdt];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) partials[blockIdx.x * 8 + threadIdx.x] = s[threadIdx.x][0];
}

// Sum of nblocks partial 8-vectors in a fixed order.
__global__ void __launch_bounds__(RED_THREADS)
k_sum8_final(const double *__restrict__ partials, int nblocks, double *__restrict__ out) {
    __shared__ double s[8][RED_THREADS];
    double q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += RED_THREADS) {
#pragma unroll
        for (int k = 0; k < 8; ++k) q[k] += partials[b * 8 + k];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) s[k][threadIdx.x] = q[k];
    __syncthreads();
    for (int wdt = RED_THREADS / 2; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
#pragma unroll
            for (int k = 0; k < 8; ++k) s[k][threadIdx.x] += s[k][threadIdx.x + wdt];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) out[threadIdx.x] = s[threadIdx.x][0];
}

// Interface height per column (Sec. V.B), pass 1: thread (x, segment) scans the rows of
// its segment upward and records the first row whose density is below rho_mid in
// first[x] (atomicMin: the minimum does not depend on the order of the updates).
template <typename T, int BC>
__global__ void k_interface_first(const T *__restrict__ g, const DevConsts<Arith<T>> P, int nx,
                                  int ny, int pitch, long long plane, double rho_mid, int seg,
                                  int *__restrict__ first) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int y0 = blockIdx.y * seg, y1 = min(ny, y0 + seg);
    for (int y = y0; y < y1; ++y) {
        Arith<T> v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = pull_val<T, BC>(g, a, x, y, nx, ny, pitch, plane, P);
        if (double(sum9(v)) < rho_mid) {
            atomicMin(&first[x], y);
            return;
        }
    }
}

// pass 2: linear interpolation between the last liquid row y-1 and the first vapour row y,
// (y - 1) + (rho(y-1) - rho_mid) / (rho(y-1) - rho(y)); NaN where row 0 is already below
// rho_mid or no row is
template <typename T, int BC>
__global__ void k_interface_height(const T *__restrict__ g, const DevConsts<Arith<T>> P, int nx,
                                   int ny, int pitch, long long plane, double rho_mid,
                                   const int *__restrict__ first, double *__restrict__ h) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= nx) return;
    const int y = first[x];
    if (y <= 0 || y >= ny) {
        h[x] = __longlong_as_double(0x7ff8000000000000ll);   // quiet NaN
        return;
    }
    auto rho_at = [&](int yy) {
        Arith<T> v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = pull_val<T, BC>(g, a, x, yy, nx, ny, pitch, plane, P);
        return double(sum9(v));
    };
    const double r0 = rho_at(y - 1), r1 = rho_at(y);
    h[x] = double(y - 1) + (r0 - rho_mid) / (r0 - r1);
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
    for (int wdt = RED_THREADS / 2; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
            s[0][threadIdx.x] += s[0][threadIdx.x + wdt];
            s[1][threadIdx.x] += s[1][threadIdx.x + wdt];
            s[2][threadIdx.x] += s[2][threadIdx.x + wdt];
            const double o = s[3][threadIdx.x + wdt];
            const double c = s[3][threadIdx.x];
            s[3][threadIdx.x] = (o > c || o != o) ? o : c;
        }
        __syncthreads();
    }
    if (threadIdx.x < 4) out[threadIdx.x] = s[threadIdx.x][0];
}

}  // namespace


// the variants of LB_STEP_VARIANTS (lb_step.cuh): strip width and planes per TMA box (9:
// whole stored rows, 3: one plane group of the stage ring)
int step_variant_count() { return 7; }

int step_variant_tx(int variant) {
    static const int tx[] = {128, 128, 240, 64, 128, 128, 240};
    return (variant >= 0 && variant < 7) ? tx[variant] : 0;
}

int step_variant_kind(int variant) { return variant >= 4 ? 1 : 0; }

int step_variant_planes(int variant) { return step_variant_kind(variant) ? 3 : 9; }

// the launch a new context or batch starts with: the stage ring, 128-column strips, S = 3
int default_step_variant() { return 4; }

StepLaunch make_step_launch(int prec, int eos_kind, const Geom &g, int num_sms, int variant,
                            int rows_override) {
    StepLaunch l;
    l.variant = variant;
    l.tx = step_variant_tx(variant);
    const bool st = step_variant_kind(variant) == 1;
    const int per_sm =
        prec == LB_FP32 ? (st ? occupancy_f32_k1 : occupancy_f32_k0)(variant, eos_kind, g.walls)
        : prec == LB_BF16 ? (st ? occupancy_bf16_k1 : occupancy_bf16_k0)(variant, eos_kind, g.walls)
                          : (st ? occupancy_f64_k1 : occupancy_f64_k0)(variant, eos_kind, g.walls);
    l.ctas_per_sm = std::max(per_sm, 1);
    if (rows_override > 0) {
        l.rows = std::min(rows_override, g.ny);
        return l;
    }
    // about three waves of resident CTAs (measured on GB300 at 2048^2: 2.7 waves of
    // 10-row CTAs beat two waves of 14 rows and one wave of 28, the staggered CTA phases
    // overlapping the ring fill of some with the compute of others), at least 8 rows
    const long long strips = (g.nx + l.tx - 1) / l.tx;
    const long long slots = (long long)std::max(num_sms, 1) * l.ctas_per_sm;
    long long blocks_y = std::max<long long>(1, 3 * slots / strips);
    long long rows = (g.ny + blocks_y - 1) / blocks_y;
    rows = std::max<long long>(rows, 8);
    l.rows = (int)std::min<long long>(rows, g.ny);
    return l;
}

// the step unit of the storage type and the variant's ring kind
static cudaError_t launch_step_unit(int prec, const Consts &c, const Geom &g, const StepLaunch &l,
                                    int order, const void *tmap, void *gout, int *err,
                                    cudaStream_t st, bool configure) {
    const bool k1 = step_variant_kind(l.variant) == 1;
    auto f = prec == LB_FP32 ? (k1 ? step_f32_k1 : step_f32_k0)
           : prec == LB_BF16 ? (k1 ? step_bf16_k1 : step_bf16_k0)
                             : (k1 ? step_f64_k1 : step_f64_k0);
    return f(c, g, l, order, tmap, gout, err, st, configure);
}

cudaError_t configure_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l) {
    static const CUtensorMap dummy{};
    return launch_step_unit(prec, c, g, l, 0, &dummy, nullptr, nullptr, nullptr, true);
}

cudaError_t launch_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l, int order,
                        const void *tensor_map_in, void *gout, int *err, cudaStream_t st) {
    return launch_step_unit(prec, c, g, l, order, tensor_map_in, gout, err, st, false);
}

cudaError_t launch_unstream(int prec, const Geom &g, const void *f, void *gbuf, bool packed,
                            cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_UNS(T, W)                                                                           \
    do {                                                                                       \
        if (packed)                                                                            \
            k_unstream<T, W, true><<<nb, 256, 0, st>>>(static_cast<const T *>(f),              \
                                                       static_cast<T *>(gbuf), g.nx, g.ny,     \
                                                       g.pitch, g.plane);                      \
        else                                                                                   \
            k_unstream<T, W, false><<<nb, 256, 0, st>>>(static_cast<const T *>(f),             \
                                                        static_cast<T *>(gbuf), g.nx, g.ny,    \
                                                        g.pitch, g.plane);                     \
    } while (0)
    if (prec == LB_FP32) {
        BC3(LB_UNS, float);
    } else if (prec == LB_BF16) {
        BC3(LB_UNS, __nv_bfloat16);
    } else {
        BC3(LB_UNS, double);
    }
#undef LB_UNS
    return cudaGetLastError();
}

cudaError_t launch_stream(int prec, const Geom &g, const void *gbuf, void *f, bool packed,
                          cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_STR(T, W)                                                                           \
    do {                                                                                       \
        if (packed)                                                                            \
            k_stream<T, W, true><<<nb, 256, 0, st>>>(static_cast<const T *>(gbuf),             \
                                                     static_cast<T *>(f), g.nx, g.ny, g.pitch, \
                                                     g.plane);                                 \
        else                                                                                   \
            k_stream<T, W, false><<<nb, 256, 0, st>>>(static_cast<const T *>(gbuf),            \
                                                      static_cast<T *>(f), g.nx, g.ny,         \
                                                      g.pitch, g.plane);                       \
    } while (0)
    if (prec == LB_FP32) {
        BC3(LB_STR, float);
    } else if (prec == LB_BF16) {
        BC3(LB_STR, __nv_bfloat16);
    } else {
        BC3(LB_STR, double);
    }
#undef LB_STR
    return cudaGetLastError();
}

cudaError_t launch_init_feq(int prec, const Consts &c_in, const Geom &g, const double *rho,
                            const double *ux, const double *uy, void *f, int *err,
                            cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
    const Consts &c = c_in;   // the initial state is rounded to nearest (pop_enc default)

#define LB_INIT(T, EOSK)                                                                   \
    k_init_feq<T, EOSK><<<nb, 256, 0, st>>>(rho, ux, uy, static_cast<T *>(f),               \
                                            to_dev<Arith<T>>(c),                             \
                                            g.nx, g.ny, g.pitch, g.plane, err)
    if (prec == LB_FP32) {
        if (c.eos_kind == LB_EOS_CS) LB_INIT(float, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_INIT(float, LB_EOS_EXP);
        else LB_INIT(float, LB_EOS_PIECEWISE);
    } else if (prec == LB_BF16) {
        if (c.eos_kind == LB_EOS_CS) LB_INIT(__nv_bfloat16, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_INIT(__nv_bfloat16, LB_EOS_EXP);
        else LB_INIT(__nv_bfloat16, LB_EOS_PIECEWISE);
    } else {
        if (c.eos_kind == LB_EOS_CS) LB_INIT(double, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_INIT(double, LB_EOS_EXP);
        else LB_INIT(double, LB_EOS_PIECEWISE);
    }
#undef LB_INIT
    return cudaGetLastError();
}

cudaError_t launch_psi_field(int prec, const Consts &c, const Geom &g, const void *gbuf,
                             void *psi, int *err, cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_PSI(T, EOSK, W)                                                                   \
    k_psi_field<T, EOSK, W><<<nb, 256, 0, st>>>(static_cast<const T *>(gbuf),                \
                                                static_cast<Arith<T> *>(psi),                \
                                                to_dev<Arith<T>>(c), g.nx, g.ny, g.pitch,    \
                                                g.plane, err)
#define LB_PSI_W(T, EOSK)                                              \
    do {                                                               \
        if (g.walls == 2) LB_PSI(T, EOSK, 2);                          \
        else if (g.walls == 1) LB_PSI(T, EOSK, 1);                     \
        else LB_PSI(T, EOSK, 0);                                       \
    } while (0)
    if (prec == LB_FP32) {
        if (c.eos_kind == LB_EOS_CS) LB_PSI_W(float, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_PSI_W(float, LB_EOS_EXP);
        else LB_PSI_W(float, LB_EOS_PIECEWISE);
    } else if (prec == LB_BF16) {
        if (c.eos_kind == LB_EOS_CS) LB_PSI_W(__nv_bfloat16, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_PSI_W(__nv_bfloat16, LB_EOS_EXP);
        else LB_PSI_W(__nv_bfloat16, LB_EOS_PIECEWISE);
    } else {
        if (c.eos_kind == LB_EOS_CS) LB_PSI_W(double, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_PSI_W(double, LB_EOS_EXP);
        else LB_PSI_W(double, LB_EOS_PIECEWISE);
    }
#undef LB_PSI_W
#undef LB_PSI
    return cudaGetLastError();
}

cudaError_t launch_macro_fields(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                const void *psi, double *rho, double *ux, double *uy,
                                cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_MAC(T, W)                                                                          \
    k_macro_fields<T, W><<<nb, 256, 0, st>>>(static_cast<const T *>(gbuf),                    \
                                             static_cast<const Arith<T> *>(psi),              \
                                             to_dev<Arith<T>>(c), g.nx, g.ny, g.pitch,        \
                                             g.plane, rho, ux, uy)
    if (prec == LB_FP32) {
        BC3(LB_MAC, float);
    } else if (prec == LB_BF16) {
        BC3(LB_MAC, __nv_bfloat16);
    } else {
        BC3(LB_MAC, double);
    }
#undef LB_MAC
    return cudaGetLastError();
}

int reduce_blocks(long long n_sites) {
    long long nb = (n_sites + RED_THREADS * 4 - 1) / (RED_THREADS * 4);
    return (int)std::max<long long>(1, std::min<long long>(nb, RED_MAX_BLOCKS));
}

cudaError_t launch_macro_reduce(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                const void *psi, double *partials, double *out4,
                                cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const int nb = reduce_blocks(n);
    const long long chunk = (n + nb - 1) / nb;
#define LB_RED(T, W)                                                                           \
    k_macro_reduce<T, W><<<nb, RED_THREADS, 0, st>>>(static_cast<const T *>(gbuf),              \
                                                     static_cast<const Arith<T> *>(psi),       \
                                                     to_dev<Arith<T>>(c), g.nx, g.ny, g.pitch, \
                                                     g.plane, chunk, partials)
    if (prec == LB_FP32) {
        BC3(LB_RED, float);
    } else if (prec == LB_BF16) {
        BC3(LB_RED, __nv_bfloat16);
    } else {
        BC3(LB_RED, double);
    }
#undef LB_RED
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, RED_THREADS, 0, st>>>(partials, nb, out4);
    return cudaGetLastError();
}

cudaError_t launch_droplet_sums(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                double cx, double cy, double r_in, double r_out,
                                double *partials, double *out8, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const int nb = reduce_blocks(n);
    const long long chunk = (n + nb - 1) / nb;
#define LB_DS(T, EOSK, W)                                                                     \
    k_droplet_sums<T, EOSK, W><<<nb, RED_THREADS, 0, st>>>(static_cast<const T *>(gbuf),       \
                                                           to_dev<Arith<T>>(c), g.nx, g.ny,    \
                                                           g.pitch, g.plane, chunk, cx, cy,    \
                                                           r_in, r_out, partials)
#define LB_DS_W(T, EOSK)                                              \
    do {                                                              \
        if (g.walls == 2) LB_DS(T, EOSK, 2);                          \
        else if (g.walls == 1) LB_DS(T, EOSK, 1);                     \
        else LB_DS(T, EOSK, 0);                                       \
    } while (0)
#define LB_DS_E(T)                                                    \
    do {                                                              \
        if (c.eos_kind == LB_EOS_CS) LB_DS_W(T, LB_EOS_CS);           \
        else if (c.eos_kind == LB_EOS_EXP) LB_DS_W(T, LB_EOS_EXP);    \
        else LB_DS_W(T, LB_EOS_PIECEWISE);                            \
    } while (0)
    if (prec == LB_FP32) LB_DS_E(float);
    else if (prec == LB_BF16) LB_DS_E(__nv_bfloat16);
    else LB_DS_E(double);
#undef LB_DS_E
#undef LB_DS_W
#undef LB_DS
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sum8_final<<<1, RED_THREADS, 0, st>>>(partials, nb, out8);
    return cudaGetLastError();
}

cudaError_t launch_interface_height(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                    double rho_mid, int *first, double *h, cudaStream_t st) {
    constexpr int SEG = 64, TPB = 128;
    // 0x7f7f7f7f: larger than any row index ("no vapour row")
    cudaError_t e = cudaMemsetAsync(first, 0x7f, sizeof(int) * (size_t)g.nx, st);
    if (e != cudaSuccess) return e;
    const dim3 grid1((g.nx + TPB - 1) / TPB, (g.ny + SEG - 1) / SEG);
    const unsigned grid2 = (g.nx + TPB - 1) / TPB;
#define LB_IH(T, W)                                                                           \
    do {                                                                                      \
        k_interface_first<T, W><<<grid1, TPB, 0, st>>>(static_cast<const T *>(gbuf),          \
                                                       to_dev<Arith<T>>(c), g.nx, g.ny,       \
                                                       g.pitch, g.plane, rho_mid, SEG, first); \
        k_interface_height<T, W><<<grid2, TPB, 0, st>>>(static_cast<const T *>(gbuf),         \
                                                        to_dev<Arith<T>>(c), g.nx, g.ny,      \
                                                        g.pitch, g.plane, rho_mid, first, h); \
    } while (0)
    if (prec == LB_FP32) {
        BC3(LB_IH, float);
    } else if (prec == LB_BF16) {
        BC3(LB_IH, __nv_bfloat16);
    } else {
        BC3(LB_IH, double);
    }
#undef LB_IH
    return cudaGetLastError();
}

}  // namespace lbm

namespace lbm {

// the batched-step unit of the storage type and the variant's ring kind
static cudaError_t batch_unit(int prec, int variant, int eos_kind, bool configure, int *occ,
                              int grid, const void *maps, const void *lats, const BatchItem *items,
                              int n_items, int phase, int *errs, cudaStream_t st) {
    const bool k1 = step_variant_kind(variant) == 1;
    auto f = prec == LB_FP32 ? (k1 ? batch_f32_k1 : batch_f32_k0)
                             : (k1 ? batch_f64_k1 : batch_f64_k0);
    return f(variant, eos_kind, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
}

cudaError_t configure_batch(int prec, int eos_kind, int variant, int *ctas_per_sm) {
    return batch_unit(prec, variant, eos_kind, true, ctas_per_sm, 0, nullptr, nullptr, nullptr, 0,
                      0, nullptr, nullptr);
}

cudaError_t launch_batch_step(int prec, int eos_kind, int variant, int grid, const void *maps,
                              const void *lats, const BatchItem *items, int n_items, int phase,
                              int *errs, cudaStream_t st) {
    return batch_unit(prec, variant, eos_kind, false, nullptr, grid, maps, lats, items, n_items,
                      phase, errs, st);
}

}  // namespace lbm
