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

__device__ __forceinline__ void mbar_inval(uint64_t *bar) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
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

// Slow path of mbar_wait_bounded: poll until the phase completes or ~1 s has passed.
__device__ __noinline__ bool mbar_wait_slow(uint64_t *bar, uint32_t parity) {
    const uint64_t t0 = global_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_ns() - t0 > 1000000000ull) return false;
    }
}

// Wait for the phase with the given parity; give up after ~1 s (returns false). The first
// try is inline: in the steady state the row has landed and no call is made.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity) {
    return mbar_try_wait(bar, parity) || mbar_wait_slow(bar, parity);
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

template <typename T>
__device__ __forceinline__ V2<T> rho_pair(const V2<T> (&f)[9]) {
    return f[0] + (((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8])));
}

// rows of the psi ring for G row groups: at least 3G + 1 (see march), a power of two
template <int G>
__host__ __device__ constexpr int psi_ring_rows() { return G == 1 ? 4 : 8; }

// shared-memory layout of k_pull_collide: S ring stages (each rounded up to 128 bytes),
// the psi ring, then S mbarriers
template <typename T, int TX, int S, int G>
__host__ __device__ constexpr size_t step_bar_offset() {
    return (size_t)S * (((9u * (TX + 8) * sizeof(T)) + 127u) / 128u * 128u) +
           (((size_t)psi_ring_rows<G>() * (TX + 4) * sizeof(T) + 15u) / 16u * 16u);
}
template <typename T, int TX, int S, int G>
__host__ __device__ constexpr size_t step_smem_bytes() {
    return step_bar_offset<T, TX, S, G>() + (size_t)S * 8 + 128;   // + room to align the base
}

template <typename T>
struct Vec2Of;
template <>
struct Vec2Of<float> { using type = float2; };
template <>
struct Vec2Of<double> { using type = double2; };

// an aligned pair of adjacent elements from shared memory
template <typename T>
__device__ __forceinline__ V2<T> lds_pair(const T *p) {
    const typename Vec2Of<T>::type v = *reinterpret_cast<const typename Vec2Of<T>::type *>(p);
    return V2<T>(v.x, v.y);
}

// f of two sites at ring columns cA, cB (adjacent c, c+1 for a thread's own pair; the two
// strip-halo columns for the halo pair) pulled from the ring rows r.m, r.z, r.p (lattice
// rows Y-1, Y, Y+1); bounce-back at the walls. ADJ: cB == cA + 1 with cA even, so the
// unshifted populations come in one aligned 2-element load.
template <typename T, bool WALLS, int BW, bool ADJ>
__device__ __forceinline__ void pull2(V2<T> (&f)[9], const Ring<T> &r, int cA, int cB,
                                      bool bottom, bool top) {
    auto at = [&](const T *row, int a, int col) { return row[a * BW + col]; };
    auto two = [&](const T *row, int a, int dc) -> V2<T> {
        if (ADJ && dc == 0) return lds_pair<T>(row + a * BW + cA);
        return V2<T>(at(row, a, cA + dc), at(row, a, cB + dc));
    };
    f[0] = two(r.z, 0, 0);
    f[1] = two(r.z, 1, -1);
    f[3] = two(r.z, 3, 1);
    if (WALLS && bottom) {   // links from below row 0 are wall links: bounce back
        f[2] = two(r.z, 4, 0);
        f[5] = two(r.z, 7, 0);
        f[6] = two(r.z, 8, 0);
    } else {
        f[2] = two(r.m, 2, 0);
        f[5] = two(r.m, 5, -1);
        f[6] = two(r.m, 6, 1);
    }
    if (WALLS && top) {
        f[4] = two(r.z, 2, 0);
        f[7] = two(r.z, 5, 0);
        f[8] = two(r.z, 6, 0);
    } else {
        f[4] = two(r.p, 4, 0);
        f[7] = two(r.p, 7, 1);
        f[8] = two(r.p, 8, -1);
    }
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

__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void grid_dependents_launch() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// One time step for one strip of a lattice: columns x0 .. x0+w-1 (w <= TX, x0 a multiple of
// 4) and rows yb .. yb+n-1, visited from `start` in direction dir. In the single-lattice
// kernel dir = +1 for even row blocks and -1 for odd (reversed on odd time steps, see
// k_pull_collide), so that neighbouring row blocks
// reach their shared apron rows at the same time and the second read hits L2.
//
// The CTA holds G row groups of TX/2 threads. Iteration k collides the G rows
// y_k + g dir (y_k = start + G k dir), group g taking row y_k + g dir, with psi of the rows
// around it; before that, group g pulls row y_k + (G + g) dir (the row it collides next
// iteration, kept in registers) and forms its psi. Lattice row start + (j-2) dir is the
// j-th row requested into the ring (slot j mod S): iteration k reads ring rows
// G k + G + 1 .. G k + 2G + 2; after its barrier rows up to G k + 2G are dead and their
// slots receive rows up to G k + 2G + S, i.e. (S - 2) / G iterations ahead of use.
// Psi of row Y sits in psi-ring row Y mod psi_ring_rows<G>(); a row is written one
// iteration before the last collision that reads it, and the rows read and written in
// two consecutive iterations span 3G + 1 rows. With walls, psi of rows -1 and ny is
// that of rows 0 and ny-1 (the collision reads those rows instead).
//
// The caller has initialised the S ring mbarriers (fresh, phase 0) and waited for the
// previous grid. Returns 0, or ERR_TIMEOUT after a bounded wait gave up (then every copy
// still in flight has landed, or its own bounded wait gave up too).
template <typename T, int EOS, bool WALLS, int TX, int S, int G>
__device__ __forceinline__ int march(const CUtensorMap *tmap, T *__restrict__ gout,
                                     const DevConsts<T> &P, const int nx, const int ny,
                                     const int pitch, const unsigned plane, const int x0,
                                     const int w, const int yb, const int n, const int dir,
                                     unsigned char *smem_raw, bool &bad) {
    static_assert(G == 1 || G == 2, "one or two row groups");
    static_assert(S >= G + 4, "ring rows of one iteration plus one row in flight");
    static_assert(TX % 4 == 0 && TX + 8 <= 256, "TMA box: 16-byte aligned start, at most 256 columns");
    constexpr int NT = TX / 2;      // threads per row group
    constexpr int BW = TX + 8;      // ring row: columns x0-4 .. x0+TX+3 -> ring col = x - x0 + 4
    constexpr int RW = TX + 4;      // psi row: columns x0-2 .. x0+TX+1 -> psi col = x - x0 + 2
    constexpr int PR = psi_ring_rows<G>();
    constexpr uint32_t STAGE_BYTES = 9u * BW * sizeof(T);
    constexpr int STAGE_ELEMS = (int)(((STAGE_BYTES + 127u) / 128u) * 128u / sizeof(T));
    T *ring = reinterpret_cast<T *>(smem_raw);                 // S stages, 128-byte aligned
    T *psis = ring + S * STAGE_ELEMS;                           // [PR][RW]
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + step_bar_offset<T, TX, S, G>());

    const int grp = G == 1 ? 0 : (int)threadIdx.x / NT;      // row group
    const int t = (int)threadIdx.x - grp * NT;                // thread within the group
    const bool lead = threadIdx.x == 0;                       // requests the ring rows
    const int c0 = 2 * t;                 // first of the thread's two columns, relative to x0
    const bool act = c0 < w;
    const bool both = c0 + 1 < w;
    const int start = dir > 0 ? yb : yb + n - 1;
    const int K = (n + G - 1) / G;        // iterations
    const int nj = G * K + G + 3;         // ring rows j = 0 .. nj-1

    // the lead thread requests ring rows in order
    int ji = 0, si = 0;
    auto issue_upto = [&](int jmax) {
        for (; ji <= jmax && ji < nj; ++ji) {
            const int r = start + (ji - 2) * dir;
            const uint32_t sl = (uint32_t)si;
            si = (si + 1 == S) ? 0 : si + 1;
            if (r == P.stall_row) continue;   // test hook: the wait for this row must time out
            // periodic: wrap the row; walls: rows outside the lattice are zero-filled by the
            // TMA unit and never read (bounce-back replaces those links)
            const int gy = WALLS ? r : ((r % ny) + ny) % ny;
            mbar_arrive_expect_tx(&bar[sl], STAGE_BYTES);
            tma_load_3d(ring + sl * STAGE_ELEMS, tmap, x0, gy, 0, &bar[sl]);
        }
    };

    if (lead) issue_upto(S - 1);

    auto stage = [&](int j) -> const T * { return ring + (j % S) * STAGE_ELEMS; };
    auto wait_row = [&](int j) -> bool {
        return mbar_wait_bounded(&bar[j % S], (uint32_t)((j / S) & 1));
    };

    // psi of lattice row Y (ring rows j-1, j, j+1 hold lattice rows Y - dir, Y, Y + dir)
    // into psi-ring row Y, keeping the pulled populations of the thread's two sites in
    // `keep`. With walls, rows outside the lattice are skipped (see above).
    auto psi_row = [&](int Y, int j, V2<T> (&keep)[9]) {
        if (WALLS && (Y < 0 || Y >= ny)) return;
        T *ps = psis + (Y & (PR - 1)) * RW;
        const Ring<T> r = dir > 0 ? Ring<T>{stage(j - 1), stage(j), stage(j + 1)}
                                  : Ring<T>{stage(j + 1), stage(j), stage(j - 1)};
        const bool bottom = WALLS && Y == 0, top = WALLS && Y == ny - 1;
        if (act) {
            pull2<T, WALLS, BW, true>(keep, r, c0 + 4, c0 + 5, bottom, top);
            const V2<T> psi = eos_psi2<T, EOS>(rho_pair(keep), P, both, bad);
            if (both) {
                store_pair<T>(ps + c0 + 2, psi, true);
            } else {
                ps[c0 + 2] = psi.lo();
            }
        }
        if (t == NT - 1) {   // the two halo columns x0-1 and x0+w as one packed pair
            V2<T> h[9];
            pull2<T, WALLS, BW, false>(h, r, 3, w + 4, bottom, top);
            const V2<T> psi = eos_psi2<T, EOS>(rho_pair(h), P, true, bad);
            ps[1] = psi.lo();
            ps[w + 2] = psi.hi();
        }
    };
    // psi-ring row holding psi of lattice row Y (walls: rows -1 and ny read rows 0, ny-1)
    auto psi_at = [&](int Y) -> const T * {
        if (WALLS) Y = Y < 0 ? 0 : (Y >= ny ? ny - 1 : Y);
        return psis + (Y & (PR - 1)) * RW;
    };

    // prologue: psi of rows start - dir .. start + (G-1) dir from ring rows 0 .. G+2;
    // group g keeps the populations of row start + g dir (its first collision row).
    // Group 0 also forms psi(start - dir), after psi(start), in the same threads.
    bool tmo = false;
    int jw = 0;                                  // first ring row not yet seen complete
#pragma unroll 1
    for (int j = 0; j <= G + 2; ++j) {
        tmo |= !wait_row(j);
        if (!tmo) jw = j + 1;
    }
    V2<T> fA[9], fB[9];
    if (!tmo) {
        psi_row(start + grp * dir, grp + 2, fA);
        if (grp == 0) psi_row(start - dir, 1, fB);
    }
    // ring rows 0 .. G are dead now: refill their slots at once
    tmo = __syncthreads_or(tmo);
    if (!tmo && lead) issue_upto(S + G);

    auto body = [&](int k, V2<T> (&fc)[9], V2<T> (&fn)[9]) -> bool {
        const int y = start + G * k * dir;
#pragma unroll
        for (int i = 0; i < G; ++i) {
            const int j = G * k + G + 3 + i;
            if (!tmo) tmo = !wait_row(j);
            if (!tmo) jw = j + 1;
        }
        if (!tmo) psi_row(y + (G + grp) * dir, G * k + G + 2 + grp, fn);
        if (__syncthreads_or(tmo)) return false;
        if (lead) issue_upto(G * k + 2 * G + S);   // refill the slots of the dead rows

        const int yr = y + grp * dir;            // this group's collision row
        if (act && G * k + grp < n) {
            const T *pm = psi_at(yr - 1);
            const T *p0 = psi_at(yr);
            const T *pp = psi_at(yr + 1);
            const int c = c0 + 2;
            const V2<T> m0 = lds_pair<T>(pm + c), z0 = lds_pair<T>(p0 + c), q0 = lds_pair<T>(pp + c);
            const T mL = pm[c - 1], mR = pm[c + 2], zL = p0[c - 1], zR = p0[c + 2];
            const T qL = pp[c - 1], qR = pp[c + 2];
            V2<T> pn[9];
            pn[0] = z0;
            pn[1] = V2<T>(z0.hi(), zR);
            pn[2] = q0;
            pn[3] = V2<T>(zL, z0.lo());
            pn[4] = m0;
            pn[5] = V2<T>(q0.hi(), qR);
            pn[6] = V2<T>(qL, q0.lo());
            pn[7] = V2<T>(mL, m0.lo());
            pn[8] = V2<T>(m0.hi(), mR);
            collide_pair<T>(fc, pn, P);

            const int x = x0 + c0;
            const unsigned idx = (unsigned)yr * (unsigned)pitch + (unsigned)(x + GH);
#pragma unroll
            for (int a = 0; a < 9; ++a) store_pair<T>(gout + (idx + a * plane), fc[a], both);
            // ghost images of columns 0, 1 (right of nx-1) and nx-2, nx-1 (left of 0)
            if (x < 2 || x + 1 >= nx - 2) {
                const unsigned rowi = (unsigned)yr * (unsigned)pitch;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const T v0 = fc[a].lo(), v1 = fc[a].hi();
                    T *rb = gout + (rowi + a * plane);
                    if (x < 2) rb[nx + GH + x] = v0;
                    if (both && x + 1 < 2) rb[nx + GH + x + 1] = v1;
                    if (x >= nx - 2) rb[x - nx + GH] = v0;
                    if (both && x + 1 >= nx - 2) rb[x + 1 - nx + GH] = v1;
                }
            }
        }
        return true;
    };

    int k = 0;
    bool ok = !tmo;                              // the same in every thread (barrier above)
    if (ok) {
        for (; k + 1 < K; k += 2) {
            if (!body(k, fA, fB) || !body(k + 1, fB, fA)) { ok = false; break; }
        }
        if (ok && k < K) ok = body(k, fA, fB);
    }
    if (!ok) {
        // a bounded wait gave up: let every requested copy land (each wait bounded; the
        // test hook's row was never requested), then leave
        if (lead)
            for (int j = jw; j < ji; ++j)
                if (start + (j - 2) * dir != P.stall_row) (void)wait_row(j);
        __syncthreads();
        return ERR_TIMEOUT;
    }
    return 0;
}

__device__ __forceinline__ unsigned char *align_smem128(unsigned char *p) {
    return p + ((128u - (smem_u32(p) & 127u)) & 127u);
}

template <int S>
__device__ __forceinline__ void init_ring_barriers(uint64_t *bar, bool reuse) {
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            if (reuse) mbar_inval(&bar[s]);
            mbar_init(&bar[s], 1);
        }
        fence_mbar_init();
    }
    __syncthreads();
}

// Single lattice: CTA (bx, by) owns strip bx and row block by of one lattice.
template <typename T, int EOS, bool WALLS, int TX, int S, int G>
__global__ void __launch_bounds__(G * TX / 2)
k_pull_collide(const __grid_constant__ CUtensorMap tin, T *__restrict__ gout,
               const DevConsts<T> P, const int nx, const int ny, const int pitch,
               const unsigned plane, const int rows, const int order, int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char *smem_raw = align_smem128(smem_dyn);
    if (threadIdx.x == 0) prefetch_tensormap(&tin);
    init_ring_barriers<S>(reinterpret_cast<uint64_t *>(smem_raw + step_bar_offset<T, TX, S, G>()),
                          false);
    // everything below reads the previous step's output or writes this step's: wait for
    // the previous grid to complete (programmatic dependent launch), then let the next one
    // start its own set-up
    grid_dependency_wait();
    grid_dependents_launch();
    // order 1 walks the blocks (and the rows inside each block) in reverse: the rows the
    // previous step wrote last, still in L2, are read first
    const int bx = order ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int by = order ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    const int x0 = bx * TX;
    const int yb = by * rows;
    bool bad = false;
    const int st = march<T, EOS, WALLS, TX, S, G>(&tin, gout, P, nx, ny, pitch, plane, x0,
                                               min(TX, nx - x0), yb, min(yb + rows, ny) - yb,
                                               ((by & 1) ^ order) ? -1 : 1, smem_raw, bad);
    if (threadIdx.x == 0 && st) atomicOr(err, st);
    if (bad) atomicOr(err, ERR_DOMAIN);
}

// Many lattices (periodic) in one launch: a persistent grid walks a fixed list of work
// items (lattice, strip, row block), item i going to CTA i mod gridDim.x. Per-lattice
// constants, buffers and TMA descriptors come from device tables; `phase` says which of a
// lattice's two buffers holds the current state. Errors are recorded per lattice.
template <typename T, int EOS, int TX, int S, int G>
__global__ void __launch_bounds__(G * TX / 2)
k_batch_step(const CUtensorMap *__restrict__ maps, const BatchLattice<T> *__restrict__ lats,
             const BatchItem *__restrict__ items, const int n_items, const int phase,
             int *__restrict__ errs) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char *smem_raw = align_smem128(smem_dyn);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + step_bar_offset<T, TX, S, G>());
    init_ring_barriers<S>(bar, false);
    grid_dependency_wait();
    grid_dependents_launch();
    for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
        const BatchItem it = items[i];
        const BatchLattice<T> &L = lats[it.lat];
        const DevConsts<T> P = L.P;
        const CUtensorMap *map = maps + 2 * it.lat + phase;
        if (threadIdx.x == 0) prefetch_tensormap(map);
        bool bad = false;
        const int st = march<T, EOS, false, TX, S, G>(map, L.g[phase ^ 1], P, L.nx, L.ny, L.pitch,
                                                   L.plane, it.x0, it.w, it.yb, it.n, it.dir,
                                                   smem_raw, bad);
        if (bad) atomicOr(&errs[it.lat], ERR_DOMAIN);
        if (st) {
            if (threadIdx.x == 0) atomicOr(&errs[it.lat], st);
            return;   // the ring is in an unknown state: this CTA stops
        }
        __syncthreads();                 // every thread is done with the ring of this item
        init_ring_barriers<S>(bar, true);
    }
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


template <typename T, int EOS, bool WALLS, int TX, int S, int G>
cudaError_t step_variant(const Consts &c, const Geom &g, int rows, int order,
                         const CUtensorMap &tin, void *out, int *err, cudaStream_t st,
                         bool configure) {
    auto kern = k_pull_collide<T, EOS, WALLS, TX, S, G>;
    constexpr size_t smem = step_smem_bytes<T, TX, S, G>();
    if (configure) {
        return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((g.nx + TX - 1) / TX, (g.ny + rows - 1) / rows);
    cfg.blockDim = dim3(G * TX / 2);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    // programmatic dependent launch: this grid's CTAs may start their set-up while the
    // previous step drains; they wait (griddepcontrol.wait) before touching global memory
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tin, static_cast<T *>(out), to_dev<T>(c), g.nx, g.ny,
                              g.pitch, (unsigned)g.plane, rows, order, err);
}

template <typename T, int TX, int S, int G>
cudaError_t step_eos(const Consts &c, const Geom &g, int rows, int order, const CUtensorMap &tin,
                     void *out, int *err, cudaStream_t st, bool configure) {
    const bool w = g.walls != 0;
    switch (c.eos_kind) {
        case LB_EOS_CS:
            return w ? step_variant<T, LB_EOS_CS, true, TX, S, G>(c, g, rows, order, tin, out, err, st, configure)
                     : step_variant<T, LB_EOS_CS, false, TX, S, G>(c, g, rows, order, tin, out, err, st, configure);
        case LB_EOS_EXP:
            return w ? step_variant<T, LB_EOS_EXP, true, TX, S, G>(c, g, rows, order, tin, out, err, st, configure)
                     : step_variant<T, LB_EOS_EXP, false, TX, S, G>(c, g, rows, order, tin, out, err, st, configure);
        default:
            return w ? step_variant<T, LB_EOS_PIECEWISE, true, TX, S, G>(c, g, rows, order, tin, out, err, st, configure)
                     : step_variant<T, LB_EOS_PIECEWISE, false, TX, S, G>(c, g, rows, order, tin, out, err, st, configure);
    }
}

template <typename T>
cudaError_t step_dispatch(const Consts &c, const Geom &g, const StepLaunch &l, int order,
                          const CUtensorMap &tin, void *out, int *err, cudaStream_t st,
                          bool configure) {
    switch (l.variant) {
        case 0: return step_eos<T, 128, 5, 1>(c, g, l.rows, order, tin, out, err, st, configure);
        case 1: return step_eos<T, 128, 6, 1>(c, g, l.rows, order, tin, out, err, st, configure);
        case 2: return step_eos<T, 240, 5, 1>(c, g, l.rows, order, tin, out, err, st, configure);
        case 3: return step_eos<T, 64, 6, 1>(c, g, l.rows, order, tin, out, err, st, configure);
        case 4: return step_eos<T, 128, 6, 2>(c, g, l.rows, order, tin, out, err, st, configure);
        case 5: return step_eos<T, 128, 8, 2>(c, g, l.rows, order, tin, out, err, st, configure);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int EOS, bool WALLS, int TX, int S, int G>
int occupancy_variant() {
    int n = 0;
    constexpr size_t smem = step_smem_bytes<T, TX, S, G>();
    auto kern = k_pull_collide<T, EOS, WALLS, TX, S, G>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, G * TX / 2, smem) != cudaSuccess)
        return 0;
    return n;
}

template <typename T, int TX, int S, int G>
int occupancy_eos(int eos, bool w) {
    switch (eos) {
        case LB_EOS_CS:
            return w ? occupancy_variant<T, LB_EOS_CS, true, TX, S, G>() : occupancy_variant<T, LB_EOS_CS, false, TX, S, G>();
        case LB_EOS_EXP:
            return w ? occupancy_variant<T, LB_EOS_EXP, true, TX, S, G>() : occupancy_variant<T, LB_EOS_EXP, false, TX, S, G>();
        default:
            return w ? occupancy_variant<T, LB_EOS_PIECEWISE, true, TX, S, G>() : occupancy_variant<T, LB_EOS_PIECEWISE, false, TX, S, G>();
    }
}

template <typename T>
int occupancy(int variant, int eos, bool w) {
    switch (variant) {
        case 0: return occupancy_eos<T, 128, 5, 1>(eos, w);
        case 1: return occupancy_eos<T, 128, 6, 1>(eos, w);
        case 2: return occupancy_eos<T, 240, 5, 1>(eos, w);
        case 3: return occupancy_eos<T, 64, 6, 1>(eos, w);
        case 4: return occupancy_eos<T, 128, 6, 2>(eos, w);
        case 5: return occupancy_eos<T, 128, 8, 2>(eos, w);
        default: return 0;
    }
}

// Per-lattice Laplace sums for the batched sweep: one CTA per lattice, fixed per-thread
// order and fixed tree (deterministic). Inside: r < R/2; outside: r > R + 0.3 min(nx,ny)/2,
// around the lattice centre ((nx-1)/2, (ny-1)/2); p = rho/3 + (G/2) psi^2.
template <typename T, int EOS>
__global__ void __launch_bounds__(RED_THREADS)
k_batch_measure(const BatchLattice<T> *__restrict__ lats, int phase,
                const double *__restrict__ radius, double *__restrict__ out) {
    __shared__ double s[8][RED_THREADS];
    const BatchLattice<T> &L = lats[blockIdx.x];
    const DevConsts<T> P = L.P;
    const int nx = L.nx, ny = L.ny;
    const T *g = L.g[phase];
    const double R = radius[blockIdx.x];
    const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1);
    const double r_in = 0.5 * R, r_out = R + 0.3 * 0.5 * min(nx, ny);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long n = (long long)nx * ny;
    for (long long i = threadIdx.x; i < n; i += RED_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        T v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a)
            v[a] = pull_global<T, false>(g, a, x, y, nx, ny, L.pitch, (long long)L.plane);
        const T rho = sum9(v);
        bool bad = false;
        const T psi = eos_psi<T, EOS>(rho, P, bad);
        const double dr = double(rho);
        const double p = dr / 3.0 + 0.5 * double(P.G) * double(psi) * double(psi);
        acc[0] += dr;
        const double r = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
        if (r < r_in) { acc[1] += dr; acc[2] += 1; acc[5] += p; }
        if (r > r_out) { acc[3] += dr; acc[4] += 1; acc[6] += p; }
        if (bad || !(dr == dr) || !(p == p)) acc[7] += 1;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int wdt = RED_THREADS / 2; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
#pragma unroll
            for (int q = 0; q < 8; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + wdt];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) out[blockIdx.x * 8 + threadIdx.x] = s[threadIdx.x][0];
}

template <typename T, int EOS, int TX, int S, int G>
cudaError_t batch_variant(bool configure, int *ctas_per_sm, int grid, const void *maps,
                          const void *lats, const BatchItem *items, int n_items, int phase,
                          int *errs, cudaStream_t st) {
    auto kern = k_batch_step<T, EOS, TX, S, G>;
    constexpr size_t smem = step_smem_bytes<T, TX, S, G>();
    if (configure) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kern, G * TX / 2, smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(G * TX / 2);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, static_cast<const CUtensorMap *>(maps),
                              static_cast<const BatchLattice<T> *>(lats), items, n_items, phase,
                              errs);
}

template <typename T, int TX, int S, int G>
cudaError_t batch_eos(int eos, bool configure, int *occ, int grid, const void *maps,
                      const void *lats, const BatchItem *items, int n_items, int phase, int *errs,
                      cudaStream_t st) {
    switch (eos) {
        case LB_EOS_CS:
            return batch_variant<T, LB_EOS_CS, TX, S, G>(configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case LB_EOS_EXP:
            return batch_variant<T, LB_EOS_EXP, TX, S, G>(configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        default:
            return batch_variant<T, LB_EOS_PIECEWISE, TX, S, G>(configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
    }
}

template <typename T>
cudaError_t batch_dispatch(int variant, int eos, bool configure, int *occ, int grid,
                           const void *maps, const void *lats, const BatchItem *items,
                           int n_items, int phase, int *errs, cudaStream_t st) {
    switch (variant) {
        case 0: return batch_eos<T, 128, 5, 1>(eos, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case 1: return batch_eos<T, 128, 6, 1>(eos, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case 2: return batch_eos<T, 240, 5, 1>(eos, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case 3: return batch_eos<T, 64, 6, 1>(eos, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case 4: return batch_eos<T, 128, 6, 2>(eos, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case 5: return batch_eos<T, 128, 8, 2>(eos, configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

int step_variant_count() { return 6; }

int step_variant_tx(int variant) {
    static const int tx[] = {128, 128, 240, 64, 128, 128};
    return (variant >= 0 && variant < 6) ? tx[variant] : 0;
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

cudaError_t configure_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l) {
    static const CUtensorMap dummy{};
    if (prec == LB_FP32) return step_dispatch<float>(c, g, l, 0, dummy, nullptr, nullptr, nullptr, true);
    return step_dispatch<double>(c, g, l, 0, dummy, nullptr, nullptr, nullptr, true);
}

cudaError_t launch_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l, int order,
                        const void *tensor_map_in, void *gout, int *err, cudaStream_t st) {
    const CUtensorMap &tin = *static_cast<const CUtensorMap *>(tensor_map_in);
    if (prec == LB_FP32) return step_dispatch<float>(c, g, l, order, tin, gout, err, st, false);
    return step_dispatch<double>(c, g, l, order, tin, gout, err, st, false);
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

namespace lbm {

cudaError_t configure_batch(int prec, int eos_kind, int variant, int *ctas_per_sm) {
    if (prec == LB_FP32)
        return batch_dispatch<float>(variant, eos_kind, true, ctas_per_sm, 0, nullptr, nullptr,
                                     nullptr, 0, 0, nullptr, nullptr);
    return batch_dispatch<double>(variant, eos_kind, true, ctas_per_sm, 0, nullptr, nullptr,
                                  nullptr, 0, 0, nullptr, nullptr);
}

cudaError_t launch_batch_step(int prec, int eos_kind, int variant, int grid, const void *maps,
                              const void *lats, const BatchItem *items, int n_items, int phase,
                              int *errs, cudaStream_t st) {
    if (prec == LB_FP32)
        return batch_dispatch<float>(variant, eos_kind, false, nullptr, grid, maps, lats, items,
                                     n_items, phase, errs, st);
    return batch_dispatch<double>(variant, eos_kind, false, nullptr, grid, maps, lats, items,
                                  n_items, phase, errs, st);
}

cudaError_t launch_batch_measure(int prec, int eos_kind, const void *lats, int n_lat, int phase,
                                 const double *radius, double *out, cudaStream_t st) {
#define LB_BM(T, EOSK)                                                                         \
    k_batch_measure<T, EOSK><<<n_lat, RED_THREADS, 0, st>>>(                                   \
        static_cast<const BatchLattice<T> *>(lats), phase, radius, out)
    if (prec == LB_FP32) {
        if (eos_kind == LB_EOS_CS) LB_BM(float, LB_EOS_CS);
        else if (eos_kind == LB_EOS_EXP) LB_BM(float, LB_EOS_EXP);
        else LB_BM(float, LB_EOS_PIECEWISE);
    } else {
        if (eos_kind == LB_EOS_CS) LB_BM(double, LB_EOS_CS);
        else if (eos_kind == LB_EOS_EXP) LB_BM(double, LB_EOS_EXP);
        else LB_BM(double, LB_EOS_PIECEWISE);
    }
#undef LB_BM
    return cudaGetLastError();
}

}  // namespace lbm
