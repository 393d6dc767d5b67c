// Templates of the step kernels shared by the translation units that instantiate them
// (lb_step_<type>.cu: the whole-row ring, lb_step_<type>_stage.cu: the stage ring, one
// pair per storage type; lb_batch_kernels.cu, lb_batch_stage.cu: the batched step) and by
// the auxiliary kernels (lb_kernels.cu). Everything here has internal linkage; each unit
// instantiates what it launches (LB_STEP_UNIT / LB_BATCH_UNIT at the end of this file).
//
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
// Population a lives in plane plane_of(a) (groups of three by the row it is pulled from,
// see lb_internal.h). Each plane has ny rows of `pitch` elements. Column x of the lattice
// lives at element x + GH<T> of its row (8 for float storage, 4 otherwise); elements GH-2,
// GH-1 and nx+GH, nx+GH+1 are ghost copies of columns nx-2, nx-1 and 0, 1 (periodic
// images), rewritten by every kernel that writes g.
//
// Hot kernels: a CTA owns a strip of TX columns (two per thread) and marches over `rows`
// rows. The populations arrive in shared memory through 3-D TMA loads
// (cp.async.bulk.tensor) completing on per-stage mbarriers: k_pull_collide_stage (the
// default) stages, per psi row, exactly the three plane groups that row is pulled from,
// one stage in use at a time; k_pull_collide stages whole rows of the strip (9 planes x
// (TX + AL + 4) columns: the strip, an apron of AL columns on the left, 8 for float
// storage and 4 otherwise, and 4 on the right), three rows in use at a time. From the
// stage a thread pulls f for its two sites, forms rho and psi (psi is never stored in
// HBM; a four-row psi ring with one halo column on each side lives in shared memory), then
// collides (Eqs. 3-8, 17-19) in packed two-lane arithmetic and stores f* as one 8-byte
// (FP32) or 16-byte (FP64) store per population. Both give identical results.



#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <type_traits>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace lbm {

namespace {

// elements before column 0 of each row (ghost_of_prec of the storage type)
template <typename T>
constexpr int GH = std::is_same<T, float>::value ? 8 : 4;
// ring rows of the step kernel: a strip of TX columns with AL<T> apron columns on the left
// and 4 on the right, so the TMA box starts at column x0 - AL<T>, i.e. at element x0 of the
// row (aligned like x0 itself), and ring column = x - x0 + AL<T>
template <typename T>
constexpr int AL = GH<T>;
template <typename T, int TX>
constexpr int ring_width() { return TX + AL<T> + 4; }
constexpr int RED_THREADS = 256;      // reduction blocks (diagnostics, batch measurement)
constexpr int RED_MAX_BLOCKS = 1024;

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

// Boundary kinds (template parameter BC, the lb_bc value): 0 periodic; 1 half-way
// bounce-back walls below row 0 and above row ny-1, periodic in x; 2 a bounce-back wall
// below row 0 and open boundaries above row ny-1 and beyond columns 0 and nx-1, where a
// population entering the lattice is pulled from the nearest lattice site (zero gradient).

// f_a(x, y) pulled from g in global memory.
template <typename T, int BC>
__device__ __forceinline__ T pull_global(const T *__restrict__ g, int a, int x, int y, int nx,
                                         int ny, int pitch, long long plane) {
    const int ex = EXv(a), ey = EYv(a);
    int sy = y - ey;
    if ((BC != 0 && sy < 0) || (BC == 1 && sy >= ny))
        return g[plane_of(opp(a)) * plane + (long long)y * pitch + x + GH<T>];
    if (BC == 0) sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
    if (BC == 2) sy = sy >= ny ? ny - 1 : sy;
    int sx = x - ex;
    if (BC == 2) sx = sx < 0 ? 0 : (sx >= nx ? nx - 1 : sx);
    else sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
    return g[plane_of(a) * plane + (long long)sy * pitch + sx + GH<T>];
}

// the value of f_a(x, y) (decoded from the storage type)
template <typename T, int BC>
__device__ __forceinline__ Arith<T> pull_val(const T *__restrict__ g, int a, int x, int y,
                                             int nx, int ny, int pitch, long long plane,
                                             const DevConsts<Arith<T>> &P) {
    // a bounced-back link reads the opposite population, whose storage shift is the same
    return pop_dec<T>(pull_global<T, BC>(g, a, x, y, nx, ny, pitch, plane), a, P);
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
    return (size_t)S * (((9u * ring_width<T, TX>() * sizeof(T)) + 127u) / 128u * 128u) +
           (((size_t)psi_ring_rows<G>() * (TX + 4) * sizeof(Arith<T>) + 15u) / 16u * 16u);
}
template <typename T, int TX, int S, int G>
__host__ __device__ constexpr size_t step_smem_bytes() {
    return step_bar_offset<T, TX, S, G>() + (size_t)S * 8 + 128;   // + room to align the base
}

// resident CTAs per SM a step kernel is compiled for (its __launch_bounds__ minimum): as
// many as its shared memory allows (with the 1 KB the hardware reserves per CTA, out of
// 228 KB), but no more than leave each thread 88 registers
__host__ __device__ constexpr int resident_ctas(size_t smem, int threads) {
    const int by_smem = (int)((228u * 1024u) / (smem + 1024u));
    const int by_regs = 65536 / (threads * 88);
    return by_smem < by_regs ? by_smem : by_regs;
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

// The step kernels work on the stored values themselves: for LB_BF16 the shifted
// f_a - w_a rho_s (exactly, as FP32), which the collision corrects in moment space
// (collide_pair with SH), so neither the loads nor the stores apply the shift.
template <typename T>
__device__ __forceinline__ Arith<T> stored_val(T v) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(v);
    else return v;
}

// an aligned pair of stored elements from shared memory, as stored values
template <typename T>
__device__ __forceinline__ V2<Arith<T>> ring_pair(const T *p) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        return V2<float>(__bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(p)));
    } else {
        return lds_pair<T>(p);
    }
}

// the density of two sites from their stored values (plus rho_s for LB_BF16)
template <typename T>
__device__ __forceinline__ V2<Arith<T>> site_rho(const V2<Arith<T>> (&f)[9],
                                                 const DevConsts<Arith<T>> &P) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value)
        return rho_pair(f) + V2<float>::all(P.rho_s);
    else
        return rho_pair(f);
}

// a stored value from the value of the shifted population (LB_BF16; nearest or, SR,
// stochastic rounding with the 16 random bits r16), the value itself otherwise
template <typename T, bool SR>
__device__ __forceinline__ T stored_enc(Arith<T> v, unsigned r16) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        if constexpr (SR) return bf16_stochastic(v, r16);
        else return __float2bfloat16_rn(v);
    } else {
        (void)r16;
        return v;
    }
}

// f of two sites at ring columns cA, cB (adjacent c, c+1 for a thread's own pair; the two
// strip-halo columns for the halo pair) pulled from the ring rows r.m, r.z, r.p (lattice
// rows Y-1, Y, Y+1); bounce-back at the walls. ADJ: cB == cA + 1 with cA even, so the
// unshifted populations come in one aligned 2-element load. A ring row holds the stored
// populations; the value of stored plane a is decoded with the shift of population a
// (a bounced-back link reads the opposite population, whose shift is the same).
template <typename T, int BC, int BW, bool ADJ>
__device__ __forceinline__ void pull2(V2<Arith<T>> (&f)[9], const Ring<T> &r, int cA, int cB,
                                      bool bottom, bool top, const DevConsts<Arith<T>> &P) {
    using A = Arith<T>;
    // stored population a sits in ring plane plane_of(a)
    auto two = [&](const T *row, int a, int dc) -> V2<A> {
        const T *pl = row + plane_of(a) * BW;
        if (ADJ && dc == 0) return ring_pair<T>(pl + cA);
        return V2<A>(stored_val<T>(pl[cA + dc]), stored_val<T>(pl[cB + dc]));
    };
    f[0] = two(r.z, 0, 0);
    f[1] = two(r.z, 1, -1);
    f[3] = two(r.z, 3, 1);
    if (BC != 0 && bottom) {   // links from below row 0 are wall links: bounce back
        f[2] = two(r.z, 4, 0);
        f[5] = two(r.z, 7, 0);
        f[6] = two(r.z, 8, 0);
    } else {
        f[2] = two(r.m, 2, 0);
        f[5] = two(r.m, 5, -1);
        f[6] = two(r.m, 6, 1);
    }
    if (BC == 1 && top) {
        f[4] = two(r.z, 2, 0);
        f[7] = two(r.z, 5, 0);
        f[8] = two(r.z, 6, 0);
    } else if (BC == 2 && top) {   // open top: from the top row itself (zero gradient)
        f[4] = two(r.z, 4, 0);
        f[7] = two(r.z, 7, 1);
        f[8] = two(r.z, 8, -1);
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

// stored pair from the pair of (shifted, for LB_BF16) values; SR: LB_BF16 with stochastic
// rounding, r32 its random bits for the pair (low half for the first site, high half for
// the second)
template <typename T, bool SR = false>
__device__ __forceinline__ void store_pop_pair(T *p, V2<Arith<T>> v, bool both, int a,
                                               const DevConsts<Arith<T>> &P, unsigned r32 = 0) {
    (void)a; (void)P;
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        const V2<float> d = v;
        if constexpr (SR) {
            const __nv_bfloat16 lo = bf16_stochastic(d.lo(), r32), hi = bf16_stochastic(d.hi(), r32 >> 16);
            if (both) *reinterpret_cast<__nv_bfloat162 *>(p) = __halves2bfloat162(lo, hi);
            else p[0] = lo;
        } else {
            if (both) *reinterpret_cast<__nv_bfloat162 *>(p) = __float22bfloat162_rn(d.v);
            else p[0] = __float2bfloat16_rn(d.lo());
        }
    } else {
        store_pair<T>(p, v, both);
    }
}

// the stochastic-rounding key of a site pair (SR: LB_BF16 with stochastic rounding), else 0
template <typename T, bool SR>
__device__ __forceinline__ unsigned store_key(int x, int y, const DevConsts<Arith<T>> &P) {
    if constexpr (SR && std::is_same<T, __nv_bfloat16>::value)
        return sr_pair_key(x, y, P.sr_step);
    else
        return 0u;
}
template <typename T, bool SR>
__device__ __forceinline__ unsigned store_bits(unsigned key, int a, const DevConsts<Arith<T>> &) {
    if constexpr (SR && std::is_same<T, __nv_bfloat16>::value)
        return sr_bits(key, a);
    else
        return 0u;
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
template <typename T, int EOS, int BC, int TX, int S, int G, bool SR = false>
__device__ __forceinline__ int march(const CUtensorMap *tmap, T *__restrict__ gout,
                                     const DevConsts<Arith<T>> &P, const int nx, const int ny,
                                     const int pitch, const unsigned plane, const int x0,
                                     const int w, const int yb, const int n, const int dir,
                                     unsigned char *smem_raw, bool &bad) {
    static_assert(G == 1 || G == 2, "one or two row groups");
    constexpr bool WALLS = BC != 0;   // rows outside the lattice are not periodic images
    static_assert(S >= G + 4, "ring rows of one iteration plus one row in flight");
    static_assert(TX % 4 == 0 && ring_width<T, TX>() <= 256,
                  "TMA box: 16-byte aligned start, at most 256 columns");
    constexpr int NT = TX / 2;      // threads per row group
    constexpr int L = AL<T>;        // left apron
    constexpr int BW = ring_width<T, TX>();   // ring row: columns x0-L .. x0+TX+3 -> col x - x0 + L
    constexpr int RW = TX + 4;      // psi row: columns x0-2 .. x0+TX+1 -> psi col = x - x0 + 2
    constexpr int PR = psi_ring_rows<G>();
    constexpr uint32_t STAGE_BYTES = 9u * BW * sizeof(T);
    constexpr int STAGE_ELEMS = (int)(((STAGE_BYTES + 127u) / 128u) * 128u / sizeof(T));
    using A = Arith<T>;
    T *ring = reinterpret_cast<T *>(smem_raw);                 // S stages, 128-byte aligned
    A *psis = reinterpret_cast<A *>(ring + S * STAGE_ELEMS);    // [PR][RW]
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
            // element x0 holds column x0 - L, the first of the box
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
    auto psi_row = [&](int Y, int j, V2<A> (&keep)[9]) {
        if (WALLS && (Y < 0 || Y >= ny)) return;
        A *ps = psis + (Y & (PR - 1)) * RW;
        const Ring<T> r = dir > 0 ? Ring<T>{stage(j - 1), stage(j), stage(j + 1)}
                                  : Ring<T>{stage(j + 1), stage(j), stage(j - 1)};
        const bool bottom = WALLS && Y == 0, top = WALLS && Y == ny - 1;
        if (act) {
            pull2<T, BC, BW, true>(keep, r, c0 + L, c0 + L + 1, bottom, top, P);
            const V2<A> psi = eos_psi2<A, EOS>(site_rho<T>(keep, P), P, both, bad);
            if (both) {
                store_pair<A>(ps + c0 + 2, psi, true);
            } else {
                ps[c0 + 2] = psi.lo();
            }
        }
        if (t == NT - 1) {   // the two halo columns x0-1 and x0+w as one packed pair
            V2<A> h[9];
            int ha = L - 1, hb = w + L;
            if (BC == 2) {   // open sides: psi beyond the lattice is that of its edge column
                if (x0 == 0) ha = L;
                if (x0 + w == nx) hb = w + L - 1;
            }
            pull2<T, BC, BW, false>(h, r, ha, hb, bottom, top, P);
            const V2<A> psi = eos_psi2<A, EOS>(site_rho<T>(h, P), P, true, bad);
            ps[1] = psi.lo();
            ps[w + 2] = psi.hi();
        }
    };
    // psi-ring row holding psi of lattice row Y (walls: rows -1 and ny read rows 0, ny-1)
    auto psi_at = [&](int Y) -> const A * {
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
    V2<A> fA[9], fB[9];
    if (!tmo) {
        psi_row(start + grp * dir, grp + 2, fA);
        if (grp == 0) psi_row(start - dir, 1, fB);
    }
    // ring rows 0 .. G are dead now: refill their slots at once
    tmo = __syncthreads_or(tmo);
    if (!tmo && lead) issue_upto(S + G);

    auto body = [&](int k, V2<A> (&fc)[9], V2<A> (&fn)[9]) -> bool {
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
            const A *pm = psi_at(yr - 1);
            const A *p0 = psi_at(yr);
            const A *pp = psi_at(yr + 1);
            const int c = c0 + 2;
            const V2<A> m0 = lds_pair<A>(pm + c), z0 = lds_pair<A>(p0 + c), q0 = lds_pair<A>(pp + c);
            const A mL = pm[c - 1], mR = pm[c + 2], zL = p0[c - 1], zR = p0[c + 2];
            const A qL = pp[c - 1], qR = pp[c + 2];
            V2<A> pn[9];
            pn[0] = z0;
            pn[1] = V2<A>(z0.hi(), zR);
            pn[2] = q0;
            pn[3] = V2<A>(zL, z0.lo());
            pn[4] = m0;
            pn[5] = V2<A>(q0.hi(), qR);
            pn[6] = V2<A>(qL, q0.lo());
            pn[7] = V2<A>(mL, m0.lo());
            pn[8] = V2<A>(m0.hi(), mR);
            collide_pair<A, BC == 2, std::is_same<T, __nv_bfloat16>::value>(fc, pn, P);

            const int x = x0 + c0;
            const unsigned idx = (unsigned)yr * (unsigned)pitch + (unsigned)(x + GH<T>);
            const unsigned key = store_key<T, SR>(x, yr, P);
#pragma unroll
            for (int a = 0; a < 9; ++a)
                store_pop_pair<T, SR>(gout + (idx + plane_of(a) * plane), fc[a], both, a, P,
                                  store_bits<T, SR>(key, a, P));
            if (BC == 2) {
                // open sides: the ghost columns repeat the edge columns (zero gradient)
                if (x == 0 || x + 1 >= nx - 1) {
                    const unsigned rowi = (unsigned)yr * (unsigned)pitch;
#pragma unroll
                    for (int a = 0; a < 9; ++a) {
                        const unsigned r = store_bits<T, SR>(key, a, P);
                        const T v0 = stored_enc<T, SR>(fc[a].lo(), r), v1 = stored_enc<T, SR>(fc[a].hi(), r >> 16);
                        T *rb = gout + (rowi + plane_of(a) * plane);
                        if (x == 0) rb[GH<T> - 1] = rb[GH<T> - 2] = v0;
                        if (x == nx - 1) rb[nx + GH<T>] = rb[nx + GH<T> + 1] = v0;
                        if (both && x + 1 == nx - 1) rb[nx + GH<T>] = rb[nx + GH<T> + 1] = v1;
                    }
                }
            } else if (x < 2 || x + 1 >= nx - 2) {
                // ghost images of columns 0, 1 (right of nx-1) and nx-2, nx-1 (left of 0)
                const unsigned rowi = (unsigned)yr * (unsigned)pitch;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const unsigned r = store_bits<T, SR>(key, a, P);
                    const T v0 = stored_enc<T, SR>(fc[a].lo(), r), v1 = stored_enc<T, SR>(fc[a].hi(), r >> 16);
                    T *rb = gout + (rowi + plane_of(a) * plane);
                    if (x < 2) rb[nx + GH<T> + x] = v0;
                    if (both && x + 1 < 2) rb[nx + GH<T> + x + 1] = v1;
                    if (x >= nx - 2) rb[x - nx + GH<T>] = v0;
                    if (both && x + 1 >= nx - 2) rb[x + 1 - nx + GH<T>] = v1;
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

// ---------------------------------------------------------------- stage ring

// Every stored value of the state is pulled exactly once per step: population a of stored
// row R feeds psi row R + e_a,y. The planes are stored in three groups of three by that
// row offset (plane_of): group 0 = populations 2, 5, 6 (pulled from the row below),
// group 1 = 0, 1, 3 (the same row), group 2 = 4, 7, 8 (the row above). Stage i of this
// ring holds exactly what psi row P_i consumes: group 0 of row P_i - 1, group 1 of row
// P_i and group 2 of row P_i + 1, fetched by three TMA loads of 3 planes each. At a wall
// the bounced-back group comes from row P_i itself with the opposite populations (group 2
// for group 0 at the bottom, group 0 for group 2 at the top; the positions inside the
// groups are opposite populations), and at an open top group 2 comes from row ny - 1.
// A stage is read by one iteration only, so one stage is in use while S - 1 are in flight.

// elements between the starts of two groups of a stage: a TMA destination must start on
// a 128-byte boundary
template <typename T, int TX>
__host__ __device__ constexpr int group_elems() {
    return (int)(((3u * ring_width<T, TX>() * sizeof(T) + 127u) / 128u) * 128u / sizeof(T));
}

template <typename T, int TX, int S>
__host__ __device__ constexpr size_t stage_bar_offset() {
    return (size_t)S * 3u * group_elems<T, TX>() * sizeof(T) +
           (((size_t)4 * (TX + 4) * sizeof(Arith<T>) + 15u) / 16u * 16u);
}
template <typename T, int TX, int S>
__host__ __device__ constexpr size_t stage_smem_bytes() {
    return stage_bar_offset<T, TX, S>() + (size_t)S * 8 + 128;
}
template <typename T, int TX, int S>
__host__ __device__ constexpr int stage_min_blocks() {
    return resident_ctas(stage_smem_bytes<T, TX, S>(), TX / 2);
}

// f of two sites at stage columns cA, cB (see pull2); population a sits at group
// plane_of(a) / 3, place plane_of(a) % 3 of the stage; only the column offset depends on
// the boundary (0 for a bounced-back link)
template <typename T, int BC, int BW, int GS, bool ADJ>
__device__ __forceinline__ void pull_stage(V2<Arith<T>> (&f)[9], const T *stg, int cA, int cB,
                                           bool bottom, bool top, const DevConsts<Arith<T>> &P) {
    using A = Arith<T>;
    auto two = [&](int a, int dc) -> V2<A> {
        const T *pl = stg + (plane_of(a) / 3) * GS + (plane_of(a) % 3) * BW;
        if (ADJ && dc == 0) return ring_pair<T>(pl + cA);
        return V2<A>(stored_val<T>(pl[cA + dc]), stored_val<T>(pl[cB + dc]));
    };
    f[0] = two(0, 0);
    f[1] = two(1, -1);
    f[3] = two(3, 1);
    f[2] = two(2, 0);
    f[4] = two(4, 0);
    if (BC != 0 && bottom) {
        f[5] = two(5, 0);
        f[6] = two(6, 0);
    } else {
        f[5] = two(5, -1);
        f[6] = two(6, 1);
    }
    if (BC == 1 && top) {
        f[7] = two(7, 0);
        f[8] = two(8, 0);
    } else {
        f[7] = two(7, 1);
        f[8] = two(8, -1);
    }
}

// One time step for one strip with the stage ring: the same work, order and arithmetic as
// march (identical results), for columns x0 .. x0+w-1 and rows yb .. yb+n-1 visited from
// `start` in direction dir. Psi row P_i = start + (i - 1) dir, i = 0 .. n + 1, is formed
// from stage i (slot i mod S). Iteration k waits for stage k + 2, forms psi of row
// P_{k+2} (keeping its populations for the next collision), passes a barrier, lets thread
// 0 request stages up to k + 2 + S into the freed slots, then collides row start + k dir.
template <typename T, int EOS, int BC, int TX, int S, bool SR = false>
__device__ __forceinline__ int march_stage(const CUtensorMap *tmap, T *__restrict__ gout,
                                           const DevConsts<Arith<T>> &P, const int nx,
                                           const int ny, const int pitch, const unsigned plane,
                                           const int x0, const int w, const int yb, const int n,
                                           const int dir, unsigned char *smem_raw, bool &bad) {
    constexpr bool WALLS = BC != 0;
    static_assert(S >= 2, "one stage in use and at least one in flight");
    static_assert(TX % 4 == 0 && ring_width<T, TX>() <= 256,
                  "TMA box: 16-byte aligned start, at most 256 columns");
    constexpr int NT = TX / 2;
    constexpr int L = AL<T>;
    constexpr int BW = ring_width<T, TX>();
    constexpr int RW = TX + 4;
    constexpr int PR = 4;           // psi ring rows
    constexpr int GS = group_elems<T, TX>();
    constexpr int STAGE_ELEMS = 3 * GS;
    constexpr uint32_t STAGE_BYTES = 9u * BW * sizeof(T);
    using A = Arith<T>;
    T *ring = reinterpret_cast<T *>(smem_raw);
    A *psis = reinterpret_cast<A *>(ring + S * STAGE_ELEMS);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + stage_bar_offset<T, TX, S>());

    const int t = (int)threadIdx.x;
    const bool lead = t == 0;             // requests the stages
    const int c0 = 2 * t;
    const bool act = c0 < w;
    const bool both = c0 + 1 < w;
    const int start = dir > 0 ? yb : yb + n - 1;
    const int ns = n + 2;                 // stages

    // the lead thread requests stages in order
    int ji = 0, si = 0;
    auto issue_upto = [&](int jmax) {
        for (; ji <= jmax && ji < ns; ++ji) {
            const int Y = start + (ji - 1) * dir;
            const uint32_t sl = (uint32_t)si;
            si = (si + 1 == S) ? 0 : si + 1;
            if (Y == P.stall_row) continue;   // test hook: the wait for this stage must time out
            int r0 = Y - 1, r1 = Y, r2 = Y + 1, p0 = 0, p2 = 6;
            if (BC == 0) {
                r0 = r0 < 0 ? r0 + ny : (r0 >= ny ? r0 - ny : r0);
                r1 = r1 < 0 ? r1 + ny : (r1 >= ny ? r1 - ny : r1);
                r2 = r2 < 0 ? r2 + ny : (r2 >= ny ? r2 - ny : r2);
            } else if (Y >= 0 && Y < ny) {
                // a psi row outside the lattice is never formed: its rows outside the lattice
                // are filled with zeros by the TMA unit
                if (Y == 0) { r0 = 0; p0 = 6; }                 // bounce-back below row 0
                if (Y == ny - 1) { r2 = ny - 1; p2 = BC == 1 ? 0 : 6; }   // wall / open top
            }
            T *dst = ring + sl * STAGE_ELEMS;
            mbar_arrive_expect_tx(&bar[sl], STAGE_BYTES);
            // element x0 holds column x0 - L, the first of the box
            tma_load_3d(dst, tmap, x0, r0, p0, &bar[sl]);
            tma_load_3d(dst + GS, tmap, x0, r1, 3, &bar[sl]);
            tma_load_3d(dst + 2 * GS, tmap, x0, r2, p2, &bar[sl]);
        }
    };
    if (lead) issue_upto(S - 1);

    // slot and phase parity of the stage awaited next (every thread tracks them)
    int ws = 0;
    uint32_t wpar = 0;
    auto wait_next = [&]() -> bool {
        const bool ok = mbar_wait_bounded(&bar[ws], wpar);
        if (++ws == S) { ws = 0; wpar ^= 1u; }
        return ok;
    };
    auto stage_of = [&](int j) -> const T * { return ring + (j % S) * STAGE_ELEMS; };

    auto psi_row = [&](int Y, const T *stg, V2<A> (&keep)[9]) {
        if (WALLS && (Y < 0 || Y >= ny)) return;
        A *ps = psis + (Y & (PR - 1)) * RW;
        const bool bottom = WALLS && Y == 0, top = WALLS && Y == ny - 1;
        if (act) {
            pull_stage<T, BC, BW, GS, true>(keep, stg, c0 + L, c0 + L + 1, bottom, top, P);
            const V2<A> psi = eos_psi2<A, EOS>(site_rho<T>(keep, P), P, both, bad);
            if (both) {
                store_pair<A>(ps + c0 + 2, psi, true);
            } else {
                ps[c0 + 2] = psi.lo();
            }
        }
        if (t == NT - 1) {   // the two halo columns x0-1 and x0+w as one packed pair
            V2<A> h[9];
            int ha = L - 1, hb = w + L;
            if (BC == 2) {   // open sides: psi beyond the lattice is that of its edge column
                if (x0 == 0) ha = L;
                if (x0 + w == nx) hb = w + L - 1;
            }
            pull_stage<T, BC, BW, GS, false>(h, stg, ha, hb, bottom, top, P);
            const V2<A> psi = eos_psi2<A, EOS>(site_rho<T>(h, P), P, true, bad);
            ps[1] = psi.lo();
            ps[w + 2] = psi.hi();
        }
    };
    auto psi_at = [&](int Y) -> const A * {
        if (WALLS) Y = Y < 0 ? 0 : (Y >= ny ? ny - 1 : Y);
        return psis + (Y & (PR - 1)) * RW;
    };

    // prologue: psi of rows start - dir (stage 0) and start (stage 1, populations kept)
    bool tmo = false;
    int jw = 0;                           // first stage not yet seen complete
#pragma unroll 1
    for (int j = 0; j < 2; ++j) {
        tmo |= !wait_next();
        if (!tmo) jw = j + 1;
    }
    V2<A> fA[9], fB[9];
    if (!tmo) {
        psi_row(start - dir, stage_of(0), fB);
        psi_row(start, stage_of(1), fA);
    }
    tmo = __syncthreads_or(tmo);
    if (!tmo && lead) issue_upto(S + 1);

    auto body = [&](int k, V2<A> (&fc)[9], V2<A> (&fn)[9]) -> bool {
        const int y = start + k * dir;
        const int j = k + 2;
        const T *stg = ring + ws * STAGE_ELEMS;   // stage j sits in slot j mod S
        if (!tmo) tmo = !wait_next();
        if (!tmo) jw = j + 1;
        if (!tmo) psi_row(y + dir, stg, fn);
        if (__syncthreads_or(tmo)) return false;
        if (lead) issue_upto(j + S);      // refill the slot of stage j and the earlier ones

        if (act) {
            const A *pm = psi_at(y - 1);
            const A *p0 = psi_at(y);
            const A *pp = psi_at(y + 1);
            const int c = c0 + 2;
            const V2<A> m0 = lds_pair<A>(pm + c), z0 = lds_pair<A>(p0 + c), q0 = lds_pair<A>(pp + c);
            const A mL = pm[c - 1], mR = pm[c + 2], zL = p0[c - 1], zR = p0[c + 2];
            const A qL = pp[c - 1], qR = pp[c + 2];
            V2<A> pn[9];
            pn[0] = z0;
            pn[1] = V2<A>(z0.hi(), zR);
            pn[2] = q0;
            pn[3] = V2<A>(zL, z0.lo());
            pn[4] = m0;
            pn[5] = V2<A>(q0.hi(), qR);
            pn[6] = V2<A>(qL, q0.lo());
            pn[7] = V2<A>(mL, m0.lo());
            pn[8] = V2<A>(m0.hi(), mR);
            collide_pair<A, BC == 2, std::is_same<T, __nv_bfloat16>::value>(fc, pn, P);

            const int x = x0 + c0;
            const unsigned idx = (unsigned)y * (unsigned)pitch + (unsigned)(x + GH<T>);
            const unsigned key = store_key<T, SR>(x, y, P);
            if (w == TX) {   // a whole strip (CTA-uniform): every thread stores two sites
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    store_pop_pair<T, SR>(gout + (idx + plane_of(a) * plane), fc[a], true, a, P,
                                      store_bits<T, SR>(key, a, P));
            } else {
#pragma unroll
                for (int a = 0; a < 9; ++a)
                    store_pop_pair<T, SR>(gout + (idx + plane_of(a) * plane), fc[a], both, a, P,
                                      store_bits<T, SR>(key, a, P));
            }
            if (BC == 2) {
                if (x == 0 || x + 1 >= nx - 1) {
                    const unsigned rowi = (unsigned)y * (unsigned)pitch;
#pragma unroll
                    for (int a = 0; a < 9; ++a) {
                        const unsigned r = store_bits<T, SR>(key, a, P);
                        const T v0 = stored_enc<T, SR>(fc[a].lo(), r), v1 = stored_enc<T, SR>(fc[a].hi(), r >> 16);
                        T *rb = gout + (rowi + plane_of(a) * plane);
                        if (x == 0) rb[GH<T> - 1] = rb[GH<T> - 2] = v0;
                        if (x == nx - 1) rb[nx + GH<T>] = rb[nx + GH<T> + 1] = v0;
                        if (both && x + 1 == nx - 1) rb[nx + GH<T>] = rb[nx + GH<T> + 1] = v1;
                    }
                }
            } else if (x < 2 || x + 1 >= nx - 2) {
                const unsigned rowi = (unsigned)y * (unsigned)pitch;
#pragma unroll
                for (int a = 0; a < 9; ++a) {
                    const unsigned r = store_bits<T, SR>(key, a, P);
                    const T v0 = stored_enc<T, SR>(fc[a].lo(), r), v1 = stored_enc<T, SR>(fc[a].hi(), r >> 16);
                    T *rb = gout + (rowi + plane_of(a) * plane);
                    if (x < 2) rb[nx + GH<T> + x] = v0;
                    if (both && x + 1 < 2) rb[nx + GH<T> + x + 1] = v1;
                    if (x >= nx - 2) rb[x - nx + GH<T>] = v0;
                    if (both && x + 1 >= nx - 2) rb[x + 1 - nx + GH<T>] = v1;
                }
            }
        }
        return true;
    };

    int k = 0;
    bool ok = !tmo;
    if (ok) {
        for (; k + 1 < n; k += 2) {
            if (!body(k, fA, fB) || !body(k + 1, fB, fA)) { ok = false; break; }
        }
        if (ok && k < n) ok = body(k, fA, fB);
    }
    if (!ok) {
        // a bounded wait gave up: let every requested stage land (each wait bounded; the
        // test hook's stage was never requested), then leave
        if (lead)
            for (int j = jw; j < ji; ++j)
                if (start + (j - 1) * dir != P.stall_row)
                    (void)mbar_wait_bounded(&bar[j % S], (uint32_t)((j / S) & 1));
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
// the stochastic-rounding kernels hold the hash state too: they are compiled for as many
// resident CTAs as 128 registers per thread allow (8 at 64 threads) rather than spill
__host__ __device__ constexpr int sr_blocks(int blocks, int threads, bool sr) {
    return !sr || blocks * threads * 128 <= 65536 ? blocks
                                                  : (65536 / (threads * 128) > 0 ? 65536 / (threads * 128) : 1);
}

template <typename T, int EOS, int BC, int TX, int S, int G, bool SR = false>
__global__ void __launch_bounds__(G * TX / 2,
                                  sr_blocks(resident_ctas(step_smem_bytes<T, TX, S, G>(), G * TX / 2), G * TX / 2, SR))
k_pull_collide(const __grid_constant__ CUtensorMap tin, T *__restrict__ gout,
               const DevConsts<Arith<T>> P, const int nx, const int ny, const int pitch,
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
    const int st = march<T, EOS, BC, TX, S, G, SR>(&tin, gout, P, nx, ny, pitch, plane, x0,
                                               min(TX, nx - x0), yb, min(yb + rows, ny) - yb,
                                               ((by & 1) ^ order) ? -1 : 1, smem_raw, bad);
    if (threadIdx.x == 0 && st) atomicOr(err, st);
    // one flag per CTA (a failing lattice would otherwise send every thread to one word)
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, ERR_DOMAIN);
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
        // phase 1 (every other step) visits the items, and the rows inside each, in reverse:
        // a step then starts on the rows the previous one wrote last (still in L2)
        const BatchItem it = items[phase ? n_items - 1 - i : i];
        const BatchLattice<T> &L = lats[it.lat];
        const DevConsts<Arith<T>> P = L.P;
        const CUtensorMap *map = maps + 2 * it.lat + phase;
        if (threadIdx.x == 0) prefetch_tensormap(map);
        bool bad = false;
        const int st = march<T, EOS, false, TX, S, G>(map, L.g[phase ^ 1], P, L.nx, L.ny, L.pitch,
                                                   L.plane, it.x0, it.w, it.yb, it.n,
                                                   phase ? -it.dir : it.dir, smem_raw, bad);
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&errs[it.lat], ERR_DOMAIN);
        if (st) {
            if (threadIdx.x == 0) atomicOr(&errs[it.lat], st);
            return;   // the ring is in an unknown state: this CTA stops
        }
        __syncthreads();                 // every thread is done with the ring of this item
        init_ring_barriers<S>(bar, true);
    }
}

// Single lattice with the stage ring (same grid, parameters and results as k_pull_collide).
template <typename T, int EOS, int BC, int TX, int S, bool SR = false>
__global__ void __launch_bounds__(TX / 2, sr_blocks(stage_min_blocks<T, TX, S>(), TX / 2, SR))
k_pull_collide_stage(const __grid_constant__ CUtensorMap tin, T *__restrict__ gout,
                     const DevConsts<Arith<T>> P, const int nx, const int ny, const int pitch,
                     const unsigned plane, const int rows, const int order, int *__restrict__ err) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char *smem_raw = align_smem128(smem_dyn);
    if (threadIdx.x == 0) prefetch_tensormap(&tin);
    init_ring_barriers<S>(reinterpret_cast<uint64_t *>(smem_raw + stage_bar_offset<T, TX, S>()),
                          false);
    grid_dependency_wait();
    grid_dependents_launch();
    const int bx = order ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int by = order ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    const int x0 = bx * TX;
    const int yb = by * rows;
    bool bad = false;
    const int st = march_stage<T, EOS, BC, TX, S, SR>(&tin, gout, P, nx, ny, pitch, plane, x0,
                                                  min(TX, nx - x0), yb, min(yb + rows, ny) - yb,
                                                  ((by & 1) ^ order) ? -1 : 1, smem_raw, bad);
    if (threadIdx.x == 0 && st) atomicOr(err, st);
    // one flag per CTA (a failing lattice would otherwise send every thread to one word)
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(err, ERR_DOMAIN);
}

// Many lattices with the stage ring (as k_batch_step).
// The item loop keeps the lattice's constants in registers on top of the single kernel's
// state: FP32 and BF16 storage are compiled for at most 10 resident CTAs (96 registers at
// 64 threads), FP64 for as many as 224 registers per thread allow, rather than re-read the
// constants from the table or spill.
template <typename T, int TX, int S>
__host__ __device__ constexpr int batch_stage_blocks() {
    constexpr int smb = stage_min_blocks<T, TX, S>();
    constexpr int cap = sizeof(T) == 8 ? 65536 / (TX / 2 * 224) : 10;
    return smb < cap ? smb : (cap > 0 ? cap : 1);
}
template <typename T, int EOS, int TX, int S>
__global__ void __launch_bounds__(TX / 2, batch_stage_blocks<T, TX, S>())
k_batch_step_stage(const CUtensorMap *__restrict__ maps, const BatchLattice<T> *__restrict__ lats,
                   const BatchItem *__restrict__ items, const int n_items, const int phase,
                   int *__restrict__ errs) {
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char *smem_raw = align_smem128(smem_dyn);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + stage_bar_offset<T, TX, S>());
    init_ring_barriers<S>(bar, false);
    grid_dependency_wait();
    grid_dependents_launch();
    for (int i = blockIdx.x; i < n_items; i += gridDim.x) {
        const BatchItem it = items[phase ? n_items - 1 - i : i];
        const BatchLattice<T> &L = lats[it.lat];
        const DevConsts<Arith<T>> P = L.P;
        const CUtensorMap *map = maps + 2 * it.lat + phase;
        if (threadIdx.x == 0) prefetch_tensormap(map);
        bool bad = false;
        const int st = march_stage<T, EOS, 0, TX, S>(map, L.g[phase ^ 1], P, L.nx, L.ny, L.pitch,
                                                     L.plane, it.x0, it.w, it.yb, it.n,
                                                     phase ? -it.dir : it.dir, smem_raw, bad);
        if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&errs[it.lat], ERR_DOMAIN);
        if (st) {
            if (threadIdx.x == 0) atomicOr(&errs[it.lat], st);
            return;
        }
        __syncthreads();
        init_ring_barriers<S>(bar, true);
    }
}

// ---------------------------------------------------------------- dispatch




// K: ring kind, 0 = whole stored rows (k_pull_collide), 1 = stages (k_pull_collide_stage)
// SR: LB_BF16 with stochastic rounding (compiled apart, so the nearest-rounding kernels
// carry none of its code)
template <typename T, int EOS, int BC, int TX, int S, int K, bool SR = false>
constexpr auto step_kernel() {
    if constexpr (K == 0) return k_pull_collide<T, EOS, BC, TX, S, 1, SR>;
    else return k_pull_collide_stage<T, EOS, BC, TX, S, SR>;
}
template <typename T, int TX, int S, int K>
constexpr size_t step_kernel_smem() {
    if constexpr (K == 0) return step_smem_bytes<T, TX, S, 1>();
    else return stage_smem_bytes<T, TX, S>();
}

template <typename T, int EOS, int BC, int TX, int S, int K>
cudaError_t step_variant(const Consts &c, const Geom &g, int rows, int order,
                         const CUtensorMap &tin, void *out, int *err, cudaStream_t st,
                         bool configure) {
    constexpr bool BF = std::is_same<T, __nv_bfloat16>::value;
    auto kern = (BF && c.stochastic) ? step_kernel<T, EOS, BC, TX, S, K, BF>()
                                     : step_kernel<T, EOS, BC, TX, S, K>();
    constexpr size_t smem = step_kernel_smem<T, TX, S, K>();
    if (configure) {
        cudaError_t e = cudaFuncSetAttribute(step_kernel<T, EOS, BC, TX, S, K>(),
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess && BF)
            e = cudaFuncSetAttribute(step_kernel<T, EOS, BC, TX, S, K, BF>(),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((g.nx + TX - 1) / TX, (g.ny + rows - 1) / rows);
    cfg.blockDim = dim3(TX / 2);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    // programmatic dependent launch: this grid's CTAs may start their set-up while the
    // previous step drains; they wait (griddepcontrol.wait) before touching global memory
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, tin, static_cast<T *>(out), to_dev<Arith<T>>(c), g.nx, g.ny,
                              g.pitch, (unsigned)g.plane, rows, order, err);
}

template <typename T, int EOS, int TX, int S, int K>
cudaError_t step_bc(const Consts &c, const Geom &g, int rows, int order, const CUtensorMap &tin,
                    void *out, int *err, cudaStream_t st, bool configure) {
    switch (g.walls) {
        case 0: return step_variant<T, EOS, 0, TX, S, K>(c, g, rows, order, tin, out, err, st, configure);
        case 1: return step_variant<T, EOS, 1, TX, S, K>(c, g, rows, order, tin, out, err, st, configure);
        default:
            // open boundaries (and nu(rho)) are compiled for FP32 and FP64 only
            if constexpr (std::is_same<T, __nv_bfloat16>::value) return cudaErrorInvalidValue;
            else return step_variant<T, EOS, 2, TX, S, K>(c, g, rows, order, tin, out, err, st, configure);
    }
}

template <typename T, int TX, int S, int K>
cudaError_t step_eos(const Consts &c, const Geom &g, int rows, int order, const CUtensorMap &tin,
                     void *out, int *err, cudaStream_t st, bool configure) {
    switch (c.eos_kind) {
        case LB_EOS_CS: return step_bc<T, LB_EOS_CS, TX, S, K>(c, g, rows, order, tin, out, err, st, configure);
        case LB_EOS_EXP: return step_bc<T, LB_EOS_EXP, TX, S, K>(c, g, rows, order, tin, out, err, st, configure);
        default: return step_bc<T, LB_EOS_PIECEWISE, TX, S, K>(c, g, rows, order, tin, out, err, st, configure);
    }
}

// The compiled launch variants: (strip width TX, ring depth S, ring kind K). The table is
// mirrored by step_variant_tx / step_variant_planes (lb_kernels.cu).
#define LB_STEP_VARIANTS(X) \
    X(0, 128, 5, 0)         \
    X(1, 128, 6, 0)         \
    X(2, 240, 5, 0)         \
    X(3, 64, 6, 0)          \
    X(4, 128, 3, 1)         \
    X(5, 128, 4, 1)         \
    X(6, 240, 3, 1)

// the variants of ring kind K (each kind is compiled in its own translation unit)
template <typename T, int K>
cudaError_t step_dispatch(const Consts &c, const Geom &g, const StepLaunch &l, int order,
                          const CUtensorMap &tin, void *out, int *err, cudaStream_t st,
                          bool configure) {
    switch (l.variant) {
#define LB_X(v, tx, s, k)                                                                   \
        case v:                                                                             \
            if constexpr (k == K)                                                           \
                return step_eos<T, tx, s, k>(c, g, l.rows, order, tin, out, err, st, configure); \
            else                                                                            \
                return cudaErrorInvalidValue;
        LB_STEP_VARIANTS(LB_X)
#undef LB_X
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int EOS, int BC, int TX, int S, int K>
int occupancy_variant() {
    int n = 0;
    constexpr size_t smem = step_kernel_smem<T, TX, S, K>();
    auto kern = step_kernel<T, EOS, BC, TX, S, K>();
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
        return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, TX / 2, smem) != cudaSuccess)
        return 0;
    return n;
}

template <typename T, int EOS, int TX, int S, int K>
int occupancy_bc(int bc) {
    switch (bc) {
        case 0: return occupancy_variant<T, EOS, 0, TX, S, K>();
        case 1: return occupancy_variant<T, EOS, 1, TX, S, K>();
        default:
            if constexpr (std::is_same<T, __nv_bfloat16>::value) return 0;
            else return occupancy_variant<T, EOS, 2, TX, S, K>();
    }
}

template <typename T, int TX, int S, int K>
int occupancy_eos(int eos, int bc) {
    switch (eos) {
        case LB_EOS_CS: return occupancy_bc<T, LB_EOS_CS, TX, S, K>(bc);
        case LB_EOS_EXP: return occupancy_bc<T, LB_EOS_EXP, TX, S, K>(bc);
        default: return occupancy_bc<T, LB_EOS_PIECEWISE, TX, S, K>(bc);
    }
}

template <typename T, int K>
int occupancy(int variant, int eos, int w) {
    switch (variant) {
#define LB_X(v, tx, s, k)                                        \
        case v:                                                  \
            if constexpr (k == K) return occupancy_eos<T, tx, s, k>(eos, w); \
            else return 0;
        LB_STEP_VARIANTS(LB_X)
#undef LB_X
        default: return 0;
    }
}

template <typename T, int EOS, int TX, int S, int K>
constexpr auto batch_kernel() {
    if constexpr (K == 0) return k_batch_step<T, EOS, TX, S, 1>;
    else return k_batch_step_stage<T, EOS, TX, S>;
}

template <typename T, int EOS, int TX, int S, int K>
cudaError_t batch_variant(bool configure, int *ctas_per_sm, int grid, const void *maps,
                          const void *lats, const BatchItem *items, int n_items, int phase,
                          int *errs, cudaStream_t st) {
    auto kern = batch_kernel<T, EOS, TX, S, K>();
    constexpr size_t smem = step_kernel_smem<T, TX, S, K>();
    if (configure) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, kern, TX / 2, smem);
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TX / 2);
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

template <typename T, int TX, int S, int K>
cudaError_t batch_eos(int eos, bool configure, int *occ, int grid, const void *maps,
                      const void *lats, const BatchItem *items, int n_items, int phase, int *errs,
                      cudaStream_t st) {
    switch (eos) {
        case LB_EOS_CS:
            return batch_variant<T, LB_EOS_CS, TX, S, K>(configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        case LB_EOS_EXP:
            return batch_variant<T, LB_EOS_EXP, TX, S, K>(configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
        default:
            return batch_variant<T, LB_EOS_PIECEWISE, TX, S, K>(configure, occ, grid, maps, lats, items, n_items, phase, errs, st);
    }
}

template <typename T, int K>
cudaError_t batch_dispatch(int variant, int eos, bool configure, int *occ, int grid,
                           const void *maps, const void *lats, const BatchItem *items,
                           int n_items, int phase, int *errs, cudaStream_t st) {
    switch (variant) {
#define LB_X(v, tx, s, k)                                                                    \
        case v:                                                                              \
            if constexpr (k == K)                                                            \
                return batch_eos<T, tx, s, k>(eos, configure, occ, grid, maps, lats, items,  \
                                              n_items, phase, errs, st);                     \
            else                                                                             \
                return cudaErrorInvalidValue;
        LB_STEP_VARIANTS(LB_X)
#undef LB_X
        default: return cudaErrorInvalidValue;
    }
}



}  // namespace

}  // namespace lbm

// The entry points of one step unit: the single-lattice step and its occupancy for storage
// type T and ring kind K (lb_internal.h declares them).
#define LB_STEP_UNIT(NAME, T, K)                                                                \
    cudaError_t step_##NAME##_k##K(const Consts &c, const Geom &g, const StepLaunch &l,        \
                                   int order, const void *tensor_map_in, void *gout, int *err, \
                                   cudaStream_t st, bool configure) {                          \
        return step_dispatch<T, K>(c, g, l, order,                                             \
                                   *static_cast<const CUtensorMap *>(tensor_map_in), gout, err, \
                                   st, configure);                                             \
    }                                                                                          \
    int occupancy_##NAME##_k##K(int variant, int eos_kind, int bc) {                          \
        return occupancy<T, K>(variant, eos_kind, bc);                                         \
    }

// The batched step of one unit (storage type T, ring kind K).
#define LB_BATCH_UNIT(NAME, T, K)                                                              \
    cudaError_t batch_##NAME##_k##K(int variant, int eos, bool configure, int *occ, int grid,  \
                                    const void *maps, const void *lats, const BatchItem *items, \
                                    int n_items, int phase, int *errs, cudaStream_t st) {      \
        return batch_dispatch<T, K>(variant, eos, configure, occ, grid, maps, lats, items,     \
                                    n_items, phase, errs, st);                                 \
    }
