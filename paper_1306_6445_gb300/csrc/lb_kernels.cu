// Kernels of the D2Q9 MRT pseudopotential update with the surface-tension source term
// (Li & Luo, arXiv 1306.6445, Sec. II and IV) for sm_103a.
//
// State layout
// ------------
// The device buffer holds g with f_a(x, t) = g_a(x - e_a) (the populations of time t are
// obtained by PULLING from g; where x - e_a lies in a wall, f_a(x) = g_opp(a)(x), half-way
// bounce-back). A time step reads g, pulls f, collides and writes the post-collision f*
// at the site itself: that f* is the g of the next step (Eq. 4 is the pull). So every step
// reads each population once and writes it once, with aligned, site-local stores.
//
// Each population plane has ny rows of `pitch` elements. Column x of the lattice lives at
// element x + GH of its row (GH = 4); elements 2, 3 and nx+4, nx+5 are ghost copies of
// columns nx-2, nx-1 and 0, 1 (periodic images), rewritten by every kernel that writes g.
//
// Hot kernel (k_pull_collide): a CTA owns a strip of TX columns (two per thread) and
// marches up `rows` rows. Rows of g (9 planes x (TX + 8) columns, i.e. the strip plus a
// 4-column apron on each side) arrive through a ring of S shared-memory stages fed by
// 3-D TMA loads (cp.async.bulk.tensor) completing on per-stage mbarriers. From the ring a
// thread pulls f for its two sites, forms rho and psi (psi is never stored in HBM; a
// four-row psi ring with one halo column on each side lives in shared memory), then
// collides (Eqs. 3-8, 17-19) in packed two-lane arithmetic and stores f* as one 8-byte
// (FP32) or 16-byte (FP64) store per population.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbm {

namespace {

constexpr int GH = 4;  // ghost columns before column 0 of each row

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for the phase with the given parity; give up after ~1 s (returns false).
__device__ __noinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y,
                                            int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap *map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// ---------------------------------------------------------------- lattice helpers
__device__ __forceinline__ int opp(int a) {
    // 0 -> 0, 1 <-> 3, 2 <-> 4, 5 <-> 7, 6 <-> 8
    return a == 0 ? 0 : (a <= 4 ? ((a + 1) & 3) + 1 : ((a - 3) & 3) + 5);
}

__host__ __device__ constexpr int EXv(int a) {
    return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0);
}
__host__ __device__ constexpr int EYv(int a) {
    return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0);
}

// rho = sum_a f_a, always in this association (the packed pair sum below matches it)
template <typename T>
__device__ __forceinline__ T sum9(const T (&v)[9]) {
    return radd(v[0], radd(radd(radd(v[1], v[3]), radd(v[2], v[4])),
                           radd(radd(v[5], v[7]), radd(v[6], v[8]))));
}

// f_a(x, y) pulled from g in global memory (periodic x; periodic y or walls).
template <typename T, bool WALLS>
__device__ __forceinline__ T pull_global(const T *__restrict__ g, int a, int x, int y, int nx,
                                         int ny, int pitch, long long plane) {
    const int ex = EXv(a), ey = EYv(a);
    int sy = y - ey;
    if (WALLS && (sy < 0 || sy >= ny)) return g[opp(a) * plane + (long long)y * pitch + x + GH];
    if (!WALLS) sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
    int sx = x - ex;
    sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
    return g[a * plane + (long long)sy * pitch + sx + GH];
}

// ---------------------------------------------------------------- the hot kernel

template <typename T>
struct Ring {
    // pointers to the three ring rows holding g rows Y-1, Y, Y+1 (each [9][BW])
    const T *m, *z, *p;
};

// f of two adjacent sites (ring column c and c+1) pulled from the ring rows.
template <typename T, bool WALLS, int BW>
__device__ __forceinline__ void pull_pair(V2<T> (&f)[9], const Ring<T> &r, int c, bool bottom,
                                          bool top) {
    auto at = [&](const T *row, int a, int col) { return row[a * BW + col]; };
    f[0] = V2<T>(at(r.z, 0, c), at(r.z, 0, c + 1));
    f[1] = V2<T>(at(r.z, 1, c - 1), at(r.z, 1, c));
    f[3] = V2<T>(at(r.z, 3, c + 1), at(r.z, 3, c + 2));
    if (WALLS && bottom) {  // sources below row 0 are wall links: bounce back
        f[2] = V2<T>(at(r.z, 4, c), at(r.z, 4, c + 1));
        f[5] = V2<T>(at(r.z, 7, c), at(r.z, 7, c + 1));
        f[6] = V2<T>(at(r.z, 8, c), at(r.z, 8, c + 1));
    } else {
        f[2] = V2<T>(at(r.m, 2, c), at(r.m, 2, c + 1));
        f[5] = V2<T>(at(r.m, 5, c - 1), at(r.m, 5, c));
        f[6] = V2<T>(at(r.m, 6, c + 1), at(r.m, 6, c + 2));
    }
    if (WALLS && top) {
        f[4] = V2<T>(at(r.z, 2, c), at(r.z, 2, c + 1));
        f[7] = V2<T>(at(r.z, 5, c), at(r.z, 5, c + 1));
        f[8] = V2<T>(at(r.z, 6, c), at(r.z, 6, c + 1));
    } else {
        f[4] = V2<T>(at(r.p, 4, c), at(r.p, 4, c + 1));
        f[7] = V2<T>(at(r.p, 7, c + 1), at(r.p, 7, c + 2));
        f[8] = V2<T>(at(r.p, 8, c - 1), at(r.p, 8, c));
    }
}

// density of one site at ring column c
template <typename T, bool WALLS, int BW>
__device__ __forceinline__ T pull_rho(const Ring<T> &r, int c, bool bottom, bool top) {
    auto at = [&](const T *row, int a, int col) { return row[a * BW + col]; };
    T v[9];
    v[0] = at(r.z, 0, c);
    v[1] = at(r.z, 1, c - 1);
    v[3] = at(r.z, 3, c + 1);
    if (WALLS && bottom) {
        v[2] = at(r.z, 4, c); v[5] = at(r.z, 7, c); v[6] = at(r.z, 8, c);
    } else {
        v[2] = at(r.m, 2, c); v[5] = at(r.m, 5, c - 1); v[6] = at(r.m, 6, c + 1);
    }
    if (WALLS && top) {
        v[4] = at(r.z, 2, c); v[7] = at(r.z, 5, c); v[8] = at(r.z, 6, c);
    } else {
        v[4] = at(r.p, 4, c); v[7] = at(r.p, 7, c + 1); v[8] = at(r.p, 8, c - 1);
    }
    return sum9(v);
}

template <typename T>
__device__ __forceinline__ V2<T> rho_pair(const V2<T> (&f)[9]) {
    return f[0] + (((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8])));
}

template <typename T>
__device__ __forceinline__ void store_pair(T *p, V2<T> v, bool both);
template <>
__device__ __forceinline__ void store_pair<float>(float *p, V2<float> v, bool both) {
    if (both) *reinterpret_cast<float2 *>(p) = v.v;
    else p[0] = v.v.x;
}
template <>
__device__ __forceinline__ void store_pair<double>(double *p, V2<double> v, bool both) {
    if (both) *reinterpret_cast<double2 *>(p) = make_double2(v.x, v.y);
    else p[0] = v.x;
}

// shared-memory layout of k_pull_collide: S ring stages (each rounded up to 128 bytes),
// the four-row psi ring, then S mbarriers
template <typename T, int TX, int S>
__host__ __device__ constexpr size_t step_bar_offset() {
    return (size_t)S * (((9u * (TX + 8) * sizeof(T)) + 127u) / 128u * 128u) +
           (((size_t)4 * (TX + 4) * sizeof(T) + 15u) / 16u * 16u);
}
template <typename T, int TX, int S>
__host__ __device__ constexpr size_t step_smem_bytes() {
    return step_bar_offset<T, TX, S>() + (size_t)S * 8 + 128;   // + room to align the base
}

template <typename T, int EOS, bool WALLS, int TX, int S>
__global__ void __launch_bounds__(TX / 2)
k_pull_collide(const __grid_constant__ CUtensorMap tin, T *__restrict__ gout,
               const DevConsts<T> P, const int nx, const int ny, const int pitch,
               const long long plane, const int rows, int *__restrict__ err) {
    static_assert(S >= 5, "the ring must hold rows y..y+2 while row y+2 is requested a step ahead");
    static_assert(TX % 4 == 0 && TX + 8 <= 256, "TMA box: 16-byte aligned start, at most 256 columns");
    constexpr int NT = TX / 2;
    constexpr int BW = TX + 8;      // ring row: columns x0-4 .. x0+TX+3 -> ring col = x - x0 + 4
    constexpr int RW = TX + 4;      // psi row: columns x0-2 .. x0+TX+1 -> psi col = x - x0 + 2
    constexpr uint32_t STAGE_BYTES = 9u * BW * sizeof(T);
    constexpr int STAGE_ELEMS = (int)(((STAGE_BYTES + 127u) / 128u) * 128u / sizeof(T));
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // the TMA destinations are placed on 128-byte boundaries of the shared window
    unsigned char *smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    T *ring = reinterpret_cast<T *>(smem_raw);                 // S stages, 128-byte aligned
    T *psis = ring + S * STAGE_ELEMS;                           // [4][RW]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + step_bar_offset<T, TX, S>());

    const int t = threadIdx.x;
    const int x0 = blockIdx.x * TX;
    const int w = min(TX, nx - x0);
    const int c0 = 2 * t;                 // first of the thread's two columns, relative to x0
    const bool act = c0 < w;
    const bool both = c0 + 1 < w;
    const int yb = blockIdx.y * rows;
    const int ye = min(yb + rows, ny);
    const int base = yb - 2;              // first ring row
    const int last = ye + 1;              // last ring row needed
    bool bad = false;

    auto slot = [&](int r) { return (r - base) % S; };
    auto parity = [&](int r) { return (uint32_t)(((r - base) / S) & 1); };
    auto rowp = [&](int r) -> const T * { return ring + slot(r) * STAGE_ELEMS; };
    auto issue = [&](int r) {
        // periodic: wrap the row; walls: rows outside the lattice are zero-filled by the
        // TMA unit and never read (bounce-back replaces those links)
        const int gy = WALLS ? r : ((r % ny) + ny) % ny;
        if (r == P.stall_row) return;   // test hook: the wait for this row must time out
        uint64_t *b = &bar[slot(r)];
        mbar_arrive_expect_tx(b, STAGE_BYTES);
        tma_load_3d(ring + slot(r) * STAGE_ELEMS, &tin, x0, gy, 0, b);
    };

    int next_issue = base;   // next ring row to request (thread 0's view)
    if (t == 0) {
        prefetch_tensormap(&tin);
        for (int s = 0; s < S; ++s) mbar_init(&bar[s], 1);
        fence_mbar_init();
    }
    __syncthreads();
    if (t == 0) {
        for (; next_issue <= min(base + S - 1, last); ++next_issue) issue(next_issue);
    }

    // psi of lattice row Y into psi-ring slot Y & 3 (walls: rows -1 and ny copy rows 0, ny-1)
    auto psi_row = [&](int Y, V2<T> *keep) {
        const int Ye = WALLS ? min(max(Y, 0), ny - 1) : Y;
        const Ring<T> r{rowp(Ye - 1), rowp(Ye), rowp(Ye + 1)};
        const bool bottom = WALLS && Ye == 0, top = WALLS && Ye == ny - 1;
        T *ps = psis + (Y & 3) * RW;
        if (act) {
            V2<T> f[9];
            pull_pair<T, WALLS, BW>(f, r, c0 + 4, bottom, top);
            const V2<T> rho = rho_pair(f);
            const T p0 = eos_psi<T, EOS>(rho.lo(), P, bad);
            const T p1 = both ? eos_psi<T, EOS>(rho.hi(), P, bad) : T(0);
            ps[c0 + 2] = p0;
            if (both) ps[c0 + 3] = p1;   // a lone last site leaves the halo slot to thread NT-1
            if (keep) {
#pragma unroll
                for (int a = 0; a < 9; ++a) keep[a] = f[a];
            }
        }
        if (t == 0) ps[1] = eos_psi<T, EOS>(pull_rho<T, WALLS, BW>(r, 3, bottom, top), P, bad);
        if (t == NT - 1) ps[w + 2] = eos_psi<T, EOS>(pull_rho<T, WALLS, BW>(r, w + 4, bottom, top), P, bad);
    };

    // prologue: rows base .. base+3 are needed for psi(yb-1), psi(yb) and f(yb)
    bool tmo = false;
    for (int r = base; r <= base + 3; ++r) tmo |= !mbar_wait_bounded(&bar[slot(r)], parity(r));
    V2<T> fc[9], fn[9];
    if (!tmo) {
        psi_row(yb - 1, nullptr);
        psi_row(yb, fc);
    }
    int waited = base + 3;

    for (int y = yb; y < ye; ++y) {
        if (!tmo && y + 2 > waited) {
            tmo |= !mbar_wait_bounded(&bar[slot(y + 2)], parity(y + 2));
            waited = y + 2;
        }
        if (!tmo) psi_row(y + 1, (y + 1 < ye) ? fn : nullptr);
        if (__syncthreads_or(tmo)) {
            // a bounded wait gave up: report, let the copies in flight land, leave
            if (t == 0) {
                atomicOr(err, ERR_TIMEOUT);
                for (int r = waited + 1; r < next_issue; ++r)
                    (void)mbar_wait_bounded(&bar[slot(r)], parity(r));
            }
            __syncthreads();
            return;
        }
        // the slot of ring row y-2 is free from here on
        if (t == 0 && next_issue <= last && next_issue <= y - 2 + S) issue(next_issue++);

        if (act) {
            const T *pm = psis + ((y - 1) & 3) * RW;
            const T *p0 = psis + (y & 3) * RW;
            const T *pp = psis + ((y + 1) & 3) * RW;
            const int c = c0 + 2;
            V2<T> pn[9];
            pn[0] = V2<T>(p0[c], p0[c + 1]);
            pn[1] = V2<T>(p0[c + 1], p0[c + 2]);
            pn[2] = V2<T>(pp[c], pp[c + 1]);
            pn[3] = V2<T>(p0[c - 1], p0[c]);
            pn[4] = V2<T>(pm[c], pm[c + 1]);
            pn[5] = V2<T>(pp[c + 1], pp[c + 2]);
            pn[6] = V2<T>(pp[c - 1], pp[c]);
            pn[7] = V2<T>(pm[c - 1], pm[c]);
            pn[8] = V2<T>(pm[c + 1], pm[c + 2]);
            collide_pair<T>(fc, pn, P);

            const int x = x0 + c0;
            T *o = gout + (long long)y * pitch + x + GH;
#pragma unroll
            for (int a = 0; a < 9; ++a) store_pair<T>(o + a * plane, fc[a], both);
            // ghost images of columns 0, 1 (right of nx-1) and nx-2, nx-1 (left of 0)
            if (x < 2 || x + 1 >= nx - 2) {
                T *rowb = gout + (long long)y * pitch;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const T v0 = fc[a].lo(), v1 = fc[a].hi();
                    if (x < 2) rowb[a * plane + nx + GH + x] = v0;
                    if (both && x + 1 < 2) rowb[a * plane + nx + GH + x + 1] = v1;
                    if (x >= nx - 2) rowb[a * plane + x - nx + GH] = v0;
                    if (both && x + 1 >= nx - 2) rowb[a * plane + x + 1 - nx + GH] = v1;
                }
            }
        }
#pragma unroll
        for (int a = 0; a < 9; ++a) fc[a] = fn[a];
    }
    if (bad) atomicOr(err, ERR_DOMAIN);
}

// ---------------------------------------------------------------- permutations

// g_b(y) = f_b(y + e_b) where y + e_b is inside the lattice, else f_opp(b)(y) (inverse of
// the pull with bounce-back). f and g use the padded layout; ghosts of g are written.
template <typename T, bool WALLS>
__global__ void k_unstream(const T *__restrict__ f, T *__restrict__ g, int nx, int ny, int pitch,
                           long long plane) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
#pragma unroll
    for (int b = 0; b < 9; ++b) {
        int ty = y + EYv(b);
        T v;
        if (WALLS && (ty < 0 || ty >= ny)) {
            v = f[opp(b) * plane + (long long)y * pitch + x + GH];
        } else {
            if (!WALLS) ty = ty < 0 ? ty + ny : (ty >= ny ? ty - ny : ty);
            int tx = x + EXv(b);
            tx = tx < 0 ? tx + nx : (tx >= nx ? tx - nx : tx);
            v = f[b * plane + (long long)ty * pitch + tx + GH];
        }
        T *rowg = g + b * plane + (long long)y * pitch;
        rowg[x + GH] = v;
        if (x < 2) rowg[nx + GH + x] = v;
        if (x >= nx - 2) rowg[x - nx + GH] = v;
    }
}

// f_a(x) = pull of g (the populations of the current time), padded layout, no ghosts.
template <typename T, bool WALLS>
__global__ void k_stream(const T *__restrict__ g, T *__restrict__ f, int nx, int ny, int pitch,
                         long long plane) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
#pragma unroll
    for (int a = 0; a < 9; ++a)
        f[a * plane + (long long)y * pitch + x + GH] =
            pull_global<T, WALLS>(g, a, x, y, nx, ny, pitch, plane);
}

// f = M^-1 m_eq(rho, u) (Eq. 3) at every site, computed in double, in the padded layout.
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
    T *p = f + (long long)y * pitch + x + GH;
#pragma unroll
    for (int a = 0; a < 9; ++a) p[a * plane] = T(o[a]);
}

// ---------------------------------------------------------------- diagnostics

// psi(rho(x)) in the storage type, into a packed nx*ny array.
template <typename T, int EOS, bool WALLS>
__global__ void k_psi_field(const T *__restrict__ g, T *__restrict__ psi, const DevConsts<T> P,
                            int nx, int ny, int pitch, long long plane, int *__restrict__ err) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    T v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = pull_global<T, WALLS>(g, a, x, y, nx, ny, pitch, plane);
    bool bad = false;
    psi[i] = eos_psi<T, EOS>(sum9(v), P, bad);
    if (bad) atomicOr(err, ERR_DOMAIN);
}

// rho and v = (sum e f + F/2)/rho (Eq. 6) of one site, from g and the psi field.
template <typename T, bool WALLS>
__device__ __forceinline__ void site_macro(const T *__restrict__ g, const T *__restrict__ psi,
                                           T G, int nx, int ny, int pitch, long long plane,
                                           int x, int y, T &rho, T &vx, T &vy) {
    T v[9];
#pragma unroll
    for (int a = 0; a < 9; ++a) v[a] = pull_global<T, WALLS>(g, a, x, y, nx, ny, pitch, plane);
    rho = sum9(v);
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
    auto ps = [&](int xx, int yy) { return psi[(long long)yy * nx + xx]; };
    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0);
    const T pc = ps(x, y);
    const T sx = (ps(xp, y) - ps(xm, y)) * third +
                 ((ps(xp, yp) - ps(xm, ym)) - (ps(xm, yp) - ps(xp, ym))) * twelfth;
    const T sy = (ps(x, yp) - ps(x, ym)) * third +
                 ((ps(xp, yp) - ps(xm, ym)) + (ps(xm, yp) - ps(xp, ym))) * twelfth;
    const T Fx = -G * pc * sx, Fy = -G * pc * sy;
    const T rinv = T(1) / rho;
    vx = (jx + T(0.5) * Fx) * rinv;
    vy = (jy + T(0.5) * Fy) * rinv;
}

template <typename T, bool WALLS>
__global__ void k_macro_fields(const T *__restrict__ g, const T *__restrict__ psi, T G, int nx,
                               int ny, int pitch, long long plane, double *__restrict__ rho,
                               double *__restrict__ ux, double *__restrict__ uy) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (long long)nx * ny) return;
    const int y = (int)(i / nx), x = (int)(i % nx);
    if (!ux && !uy) {  // density only: psi is not needed
        T v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a) v[a] = pull_global<T, WALLS>(g, a, x, y, nx, ny, pitch, plane);
        rho[i] = double(sum9(v));
        return;
    }
    T r, vx, vy;
    site_macro<T, WALLS>(g, psi, G, nx, ny, pitch, plane, x, y, r, vx, vy);
    if (rho) rho[i] = double(r);
    if (ux) ux[i] = double(vx);
    if (uy) uy[i] = double(vy);
}

constexpr int RED_THREADS = 256;
constexpr int RED_MAX_BLOCKS = 1024;

// Block b reduces the contiguous site range [b*chunk, (b+1)*chunk) in FP64 with a fixed
// per-thread order and a fixed shared-memory tree: the result does not depend on timing.
template <typename T, bool WALLS>
__global__ void __launch_bounds__(RED_THREADS)
k_macro_reduce(const T *__restrict__ g, const T *__restrict__ psi, T G, int nx, int ny,
               int pitch, long long plane, long long chunk, double *__restrict__ partials) {
    __shared__ double s[4][RED_THREADS];
    const long long n = (long long)nx * ny;
    const long long beg = (long long)blockIdx.x * chunk;
    const long long end = min(n, beg + chunk);
    double m = 0, px = 0, py = 0, vmax = 0;
    for (long long i = beg + threadIdx.x; i < end; i += RED_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        T r, vx, vy;
        site_macro<T, WALLS>(g, psi, G, nx, ny, pitch, plane, x, y, r, vx, vy);
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

// ---------------------------------------------------------------- dispatch

inline unsigned blocks_for(long long n, int t) { return (unsigned)((n + t - 1) / t); }


template <typename T, int EOS, bool WALLS, int TX, int S>
cudaError_t step_variant(const Consts &c, const Geom &g, int rows, const CUtensorMap &tin,
                         void *out, int *err, cudaStream_t st, bool configure) {
    auto kern = k_pull_collide<T, EOS, WALLS, TX, S>;
    constexpr size_t smem = step_smem_bytes<T, TX, S>();
    if (configure) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    dim3 grid((g.nx + TX - 1) / TX, (g.ny + rows - 1) / rows);
    kern<<<grid, TX / 2, smem, st>>>(tin, static_cast<T *>(out), to_dev<T>(c), g.nx, g.ny,
                                     g.pitch, g.plane, rows, err);
    return cudaGetLastError();
}

template <typename T, int TX, int S>
cudaError_t step_eos(const Consts &c, const Geom &g, int rows, const CUtensorMap &tin, void *out,
                     int *err, cudaStream_t st, bool configure) {
    const bool w = g.walls != 0;
    switch (c.eos_kind) {
        case LB_EOS_CS:
            return w ? step_variant<T, LB_EOS_CS, true, TX, S>(c, g, rows, tin, out, err, st, configure)
                     : step_variant<T, LB_EOS_CS, false, TX, S>(c, g, rows, tin, out, err, st, configure);
        case LB_EOS_EXP:
            return w ? step_variant<T, LB_EOS_EXP, true, TX, S>(c, g, rows, tin, out, err, st, configure)
                     : step_variant<T, LB_EOS_EXP, false, TX, S>(c, g, rows, tin, out, err, st, configure);
        default:
            return w ? step_variant<T, LB_EOS_PIECEWISE, true, TX, S>(c, g, rows, tin, out, err, st, configure)
                     : step_variant<T, LB_EOS_PIECEWISE, false, TX, S>(c, g, rows, tin, out, err, st, configure);
    }
}

template <typename T>
cudaError_t step_dispatch(const Consts &c, const Geom &g, const StepLaunch &l,
                          const CUtensorMap &tin, void *out, int *err, cudaStream_t st,
                          bool configure) {
    switch (l.variant) {
        case 0: return step_eos<T, 128, 6>(c, g, l.rows, tin, out, err, st, configure);
        case 1: return step_eos<T, 128, 5>(c, g, l.rows, tin, out, err, st, configure);
        case 2: return step_eos<T, 240, 6>(c, g, l.rows, tin, out, err, st, configure);
        case 3: return step_eos<T, 128, 8>(c, g, l.rows, tin, out, err, st, configure);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int EOS, bool WALLS, int TX, int S>
int occupancy_variant() {
    int n = 0;
    constexpr size_t smem = step_smem_bytes<T, TX, S>();
    auto kern = k_pull_collide<T, EOS, WALLS, TX, S>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX / 2, smem) != cudaSuccess) return 0;
    return n;
}

template <typename T, int TX, int S>
int occupancy_eos(int eos, bool w) {
    switch (eos) {
        case LB_EOS_CS:
            return w ? occupancy_variant<T, LB_EOS_CS, true, TX, S>() : occupancy_variant<T, LB_EOS_CS, false, TX, S>();
        case LB_EOS_EXP:
            return w ? occupancy_variant<T, LB_EOS_EXP, true, TX, S>() : occupancy_variant<T, LB_EOS_EXP, false, TX, S>();
        default:
            return w ? occupancy_variant<T, LB_EOS_PIECEWISE, true, TX, S>() : occupancy_variant<T, LB_EOS_PIECEWISE, false, TX, S>();
    }
}

template <typename T>
int occupancy(int variant, int eos, bool w) {
    switch (variant) {
        case 0: return occupancy_eos<T, 128, 6>(eos, w);
        case 1: return occupancy_eos<T, 128, 5>(eos, w);
        case 2: return occupancy_eos<T, 240, 6>(eos, w);
        case 3: return occupancy_eos<T, 128, 8>(eos, w);
        default: return 0;
    }
}

}  // namespace

int step_variant_count() { return 4; }

int step_variant_tx(int variant) {
    static const int tx[] = {128, 128, 240, 128};
    return (variant >= 0 && variant < 4) ? tx[variant] : 0;
}

StepLaunch make_step_launch(int prec, int eos_kind, const Geom &g, int num_sms, int variant,
                            int rows_override) {
    StepLaunch l;
    l.variant = variant;
    l.tx = step_variant_tx(variant);
    const int per_sm = prec == LB_FP32 ? occupancy<float>(variant, eos_kind, g.walls != 0)
                                       : occupancy<double>(variant, eos_kind, g.walls != 0);
    l.ctas_per_sm = std::max(per_sm, 1);
    if (rows_override > 0) {
        l.rows = std::min(rows_override, g.ny);
        return l;
    }
    // about two waves of resident CTAs (measured on GB300 at 2048^2: two waves of 16-row
    // CTAs beat one wave of 44-row CTAs, the staggered CTA phases overlapping the ring
    // fill of some with the compute of others), never below 8 rows per CTA
    const long long strips = (g.nx + l.tx - 1) / l.tx;
    const long long slots = (long long)std::max(num_sms, 1) * l.ctas_per_sm;
    long long blocks_y = std::max<long long>(1, 2 * slots / strips);
    long long rows = (g.ny + blocks_y - 1) / blocks_y;
    rows = std::max<long long>(rows, 8);
    l.rows = (int)std::min<long long>(rows, g.ny);
    return l;
}

cudaError_t configure_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l) {
    static const CUtensorMap dummy{};
    if (prec == LB_FP32) return step_dispatch<float>(c, g, l, dummy, nullptr, nullptr, nullptr, true);
    return step_dispatch<double>(c, g, l, dummy, nullptr, nullptr, nullptr, true);
}

cudaError_t launch_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l,
                        const void *tensor_map_in, void *gout, int *err, cudaStream_t st) {
    const CUtensorMap &tin = *static_cast<const CUtensorMap *>(tensor_map_in);
    if (prec == LB_FP32) return step_dispatch<float>(c, g, l, tin, gout, err, st, false);
    return step_dispatch<double>(c, g, l, tin, gout, err, st, false);
}

cudaError_t launch_unstream(int prec, const Geom &g, const void *f, void *gbuf, cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_UNS(T, W)                                                                          \
    k_unstream<T, W><<<nb, 256, 0, st>>>(static_cast<const T *>(f), static_cast<T *>(gbuf), g.nx, \
                                         g.ny, g.pitch, g.plane)
    if (prec == LB_FP32) {
        if (g.walls) LB_UNS(float, true); else LB_UNS(float, false);
    } else {
        if (g.walls) LB_UNS(double, true); else LB_UNS(double, false);
    }
#undef LB_UNS
    return cudaGetLastError();
}

cudaError_t launch_stream(int prec, const Geom &g, const void *gbuf, void *f, cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_STR(T, W)                                                                         \
    k_stream<T, W><<<nb, 256, 0, st>>>(static_cast<const T *>(gbuf), static_cast<T *>(f), g.nx, \
                                       g.ny, g.pitch, g.plane)
    if (prec == LB_FP32) {
        if (g.walls) LB_STR(float, true); else LB_STR(float, false);
    } else {
        if (g.walls) LB_STR(double, true); else LB_STR(double, false);
    }
#undef LB_STR
    return cudaGetLastError();
}

cudaError_t launch_init_feq(int prec, const Consts &c, const Geom &g, const double *rho,
                            const double *ux, const double *uy, void *f, int *err,
                            cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
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

cudaError_t launch_psi_field(int prec, const Consts &c, const Geom &g, const void *gbuf,
                             void *psi, int *err, cudaStream_t st) {
    const unsigned nb = blocks_for((long long)g.nx * g.ny, 256);
#define LB_PSI(T, EOSK, W)                                                                   \
    k_psi_field<T, EOSK, W><<<nb, 256, 0, st>>>(static_cast<const T *>(gbuf),                \
                                                static_cast<T *>(psi), to_dev<T>(c), g.nx,   \
                                                g.ny, g.pitch, g.plane, err)
#define LB_PSI_W(T, EOSK) \
    do { if (g.walls) LB_PSI(T, EOSK, true); else LB_PSI(T, EOSK, false); } while (0)
    if (prec == LB_FP32) {
        if (c.eos_kind == LB_EOS_CS) LB_PSI_W(float, LB_EOS_CS);
        else if (c.eos_kind == LB_EOS_EXP) LB_PSI_W(float, LB_EOS_EXP);
        else LB_PSI_W(float, LB_EOS_PIECEWISE);
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
                                             static_cast<const T *>(psi), T(c.G), g.nx, g.ny,  \
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

cudaError_t launch_macro_reduce(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                const void *psi, double *partials, double *out4,
                                cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny;
    const int nb = reduce_blocks(n);
    const long long chunk = (n + nb - 1) / nb;
#define LB_RED(T, W)                                                                           \
    k_macro_reduce<T, W><<<nb, RED_THREADS, 0, st>>>(static_cast<const T *>(gbuf),              \
                                                     static_cast<const T *>(psi), T(c.G), g.nx, \
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
