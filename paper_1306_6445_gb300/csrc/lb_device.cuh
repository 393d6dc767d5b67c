// Device-side building blocks of the D2Q9 MRT pseudopotential update.
//
// Velocity order e_0..e_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1);
// moment order (rho, e, zeta, j_x, q_x, j_y, q_y, p_xx, p_xy) of the standard D2Q9
// transformation matrix M (Sec. II). All constants below are written out by hand.
//
// The collision works on PAIRS of sites held in a two-lane vector: in FP32 the lanes are
// packed into one register pair and every add / subtract / multiply / fma is a single
// packed instruction of sm_100-class GPUs (__fadd2_rn, sub.rn.f32x2, __fmul2_rn,
// __ffma2_rn, each lane rounded exactly like the scalar operation); in FP64 the two lanes
// are plain scalar doubles.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "lb_internal.h"

namespace lbm {

// Storage element -> arithmetic type: BF16 storage (LB_BF16) is worked on in FP32.
template <typename T>
struct ArithOf { using type = T; };
template <>
struct ArithOf<__nv_bfloat16> { using type = float; };
template <typename T>
using Arith = typename ArithOf<T>::type;

template <typename T>
struct DevConsts {
    T a, b4, RT;
    T psi0, rho0;
    T th_v, th_m, th_l, rho1, rho2, p_rho1, p_rho2;
    T two_over_G;
    T G, kG2, sig_coef;
    T s_e, s_z, s_q, s_v;
    // Eq. 17 coefficients per relaxed moment k: (1 - s_k), s_k, (1 - s_k/2) and the source
    // weights 3 s_k / 2 (e, zeta) and -s_v (p_xx, p_xy), rounded once from FP64
    T e_keep, e_half, e_src, z_keep, z_half, z_src, q_keep, q_half, v_keep, v_half, v_src;
    // storage shift w_a rho_s: LB_BF16 stores f_a - w_a rho_s (zero for FP32 / FP64)
    T wshift[9];
    T rho_s;
    // nu(rho) (open-boundary kernels only): sites with rho < rho_sw relax p_xx, p_xy at
    // s_vV; the Eq. 17 coefficients for that rate
    T rho_sw, s_vV, v_keep_V, v_half_V, v_src_V;
    int stall_row;
    // LB_BF16 stochastic rounding: the step of the launch (the counter)
    unsigned sr_step;
};

// Per-lattice record of the batched step (lives in a device table).
template <typename T>
struct BatchLattice {
    T *g[2];              // the lattice's two population buffers
    DevConsts<T> P;
    int nx, ny, pitch;
    unsigned plane;
    int frozen;           // 1: set inactive (not stepped); its state stays in g[0]
};

template <typename T>
inline DevConsts<T> to_dev(const Consts &c) {
    DevConsts<T> d;
    d.a = T(c.a); d.b4 = T(c.b4); d.RT = T(c.RT);
    d.psi0 = T(c.psi0); d.rho0 = T(c.rho0);
    d.th_v = T(c.th_v); d.th_m = T(c.th_m); d.th_l = T(c.th_l);
    d.rho1 = T(c.rho1); d.rho2 = T(c.rho2); d.p_rho1 = T(c.p_rho1); d.p_rho2 = T(c.p_rho2);
    d.two_over_G = T(c.two_over_G);
    d.G = T(c.G); d.kG2 = T(c.kG2); d.sig_coef = T(c.sig_coef);
    d.s_e = T(c.s_e); d.s_z = T(c.s_z); d.s_q = T(c.s_q); d.s_v = T(c.s_v);
    d.e_keep = T(1.0 - c.s_e); d.e_half = T(1.0 - 0.5 * c.s_e); d.e_src = T(1.5 * c.s_e);
    d.z_keep = T(1.0 - c.s_z); d.z_half = T(1.0 - 0.5 * c.s_z); d.z_src = T(1.5 * c.s_z);
    d.q_keep = T(1.0 - c.s_q); d.q_half = T(1.0 - 0.5 * c.s_q);
    d.v_keep = T(1.0 - c.s_v); d.v_half = T(1.0 - 0.5 * c.s_v); d.v_src = T(-c.s_v);
    for (int a = 0; a < 9; ++a)
        d.wshift[a] = T((a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0)) * c.shift_rho);
    d.rho_s = T(c.shift_rho);
    d.rho_sw = T(c.rho_sw);
    d.s_vV = T(c.s_v_vapour);
    d.v_keep_V = T(1.0 - c.s_v_vapour);
    d.v_half_V = T(1.0 - 0.5 * c.s_v_vapour);
    d.v_src_V = T(-c.s_v_vapour);
    d.stall_row = c.stall_row;
    d.sr_step = c.step_key;
    return d;
}

// ---- scalar helpers: FP32 uses the hardware approximations (a few ulp, far inside the
// FP32 error budget), FP64 IEEE-rounded operations (its division within one ulp: the
// product with the rounded reciprocal). Every add / multiply / fma is an
// explicit round-to-nearest intrinsic, so the compiler cannot contract them differently
// at different inline sites: a site's psi is bitwise the same wherever it is computed. --
__device__ __forceinline__ float lb_exp(float v) { return __expf(v); }
__device__ __forceinline__ double lb_exp(double v) { return exp(v); }
// FP32 reciprocal and reciprocal square root: one hardware approximation each (PTX
// rcp.approx / rsqrt.approx, within two ulp), subnormal inputs and results flushed to zero
// (.ftz): the update meets no subnormal density, pressure or potential, and the
// non-flushing forms add range fix-ups around every approximation.
__device__ __forceinline__ float rcp_ftz(float v) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float rsqrt_ftz(float v) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}
__device__ __forceinline__ float lb_div(float a, float b) { return __fmul_rn(a, rcp_ftz(b)); }
// FP64 a / b as a times the correctly rounded 1 / b (within one ulp of the quotient)
__device__ __forceinline__ double lb_div(double a, double b) { return __dmul_rn(a, __drcp_rn(b)); }
__device__ __forceinline__ float lb_rcp(float v) { return rcp_ftz(v); }
__device__ __forceinline__ double lb_rcp(double v) { return __drcp_rn(v); }   // = 1 / v rounded
__device__ __forceinline__ float lb_sqrt_pos(float v) { return __fmul_rn(v, rsqrt_ftz(v)); }   // v > 0
__device__ __forceinline__ double lb_sqrt_pos(double v) { return __dsqrt_rn(v); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }

// ---- stored population <-> value. FP32 / FP64 store f itself; LB_BF16 stores the FP32
// difference f_a - w_a rho_s rounded to BF16 (nearest even), and reads it back exactly
// as float(stored) + w_a rho_s (one FP32 rounding).
template <typename T>
__device__ __forceinline__ Arith<T> pop_dec(T v, int, const DevConsts<Arith<T>> &) { return v; }
template <>
__device__ __forceinline__ float pop_dec<__nv_bfloat16>(__nv_bfloat16 v, int a,
                                                         const DevConsts<float> &P) {
    return __fadd_rn(__bfloat162float(v), P.wshift[a]);
}
// MurmurHash3's 32-bit finaliser (fmix32; A. Appleby, public domain): a bijective mix of a
// 32-bit counter into well-spread bits, the generator of the stochastic rounding below.
__device__ __forceinline__ unsigned mix32(unsigned h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// The counter of a site pair (first column x, row y) in the step of the launch, and the 32
// random bits of its population a (16 per site of the pair): reproducible, and independent
// of the launch shape.
__device__ __forceinline__ unsigned sr_pair_key(int x, int y, unsigned step) {
    return mix32(mix32((unsigned)y * 0x9e3779b1u + (unsigned)x) ^ (step * 0x85ebca6bu));
}
__device__ __forceinline__ unsigned sr_bits(unsigned key, int a) {
    return mix32(key + (unsigned)(a + 1) * 0x9e3779b9u);
}

// BF16 of v rounded stochastically with the 16 random bits r16: r16 is added below the
// kept bits and the rest cut off, so the magnitude rounds up with probability (dropped
// bits) / 2^16 and the expected stored value is v.
__device__ __forceinline__ __nv_bfloat16 bf16_stochastic(float v, unsigned r16) {
    unsigned b = __float_as_uint(v);
    if ((b & 0x7f800000u) != 0x7f800000u) b += r16 & 0xffffu;   // not Inf / NaN
    __nv_bfloat16_raw raw;
    raw.x = (unsigned short)(b >> 16);
    return __nv_bfloat16(raw);
}

// SR: LB_BF16 with stochastic rounding, r16 its random bits; otherwise nearest even
template <typename T, bool SR = false>
__device__ __forceinline__ T pop_enc(Arith<T> v, int a, const DevConsts<Arith<T>> &P,
                                     unsigned r16 = 0) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        const float d = __fsub_rn(v, P.wshift[a]);
        if constexpr (SR) return bf16_stochastic(d, r16);
        else return __float2bfloat16_rn(d);
    } else {
        (void)a; (void)P; (void)r16;
        return v;
    }
}

// Interaction potential psi(rho) (Sec. II): psi0 exp(-rho0/rho), or
// sqrt(2 (p_EOS - rho c_s^2) / G) with p_EOS the Carnahan-Starling EOS or Eq. 23.
// Sets `bad` when rho <= 0 or psi^2 <= 0 (the value is then not usable).
template <typename T, int EOS>
__device__ __forceinline__ T eos_psi(T rho, const DevConsts<T> &P, bool &bad) {
    if constexpr (EOS == LB_EOS_EXP) {
        bad |= !(rho > T(0));
        return rmul(P.psi0, lb_exp(-lb_div(P.rho0, rho)));
    } else {
        T p;
        if constexpr (EOS == LB_EOS_CS) {
            // rho RT (1 + eta + eta^2 - eta^3) / (1 - eta)^3 - a rho^2
            const T eta = rmul(P.b4, rho);
            const T om = rsub(T(1), eta);
            const T poly = rfma(eta, rfma(eta, rsub(T(1), eta), T(1)), T(1));
            const T num = rmul(rmul(rho, P.RT), poly);
            p = rsub(lb_div(num, rmul(rmul(om, om), om)), rmul(P.a, rmul(rho, rho)));
        } else {
            p = (rho <= P.rho1) ? rmul(rho, P.th_v)
              : (rho < P.rho2) ? rfma(rsub(rho, P.rho1), P.th_m, P.p_rho1)
                               : rfma(rsub(rho, P.rho2), P.th_l, P.p_rho2);
        }
        const T arg = rmul(rsub(p, rmul(rho, T(1.0 / 3.0))), P.two_over_G);
        bad |= !(arg > T(0)) || !(rho > T(0));
        return lb_sqrt_pos(arg);
    }
}

// ---- two-lane vectors ---------------------------------------------------------------
template <typename T>
struct V2;

template <>
struct V2<float> {
    float2 v;
    __device__ __forceinline__ V2() {}
    __device__ __forceinline__ V2(float2 a) : v(a) {}
    __device__ __forceinline__ V2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ static V2 all(float a) { return V2(a, a); }
    __device__ __forceinline__ float lo() const { return v.x; }
    __device__ __forceinline__ float hi() const { return v.y; }
};
__device__ __forceinline__ V2<float> operator+(V2<float> a, V2<float> b) { return __fadd2_rn(a.v, b.v); }
__device__ __forceinline__ V2<float> operator*(V2<float> a, V2<float> b) { return __fmul2_rn(a.v, b.v); }
__device__ __forceinline__ V2<float> operator-(V2<float> a, V2<float> b) {
    // the packed subtraction (PTX sub.rn.f32x2), lane by lane the rounded a - b
    float2 r;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.v.x), "f"(a.v.y), "f"(b.v.x), "f"(b.v.y));
    return r;
}
__device__ __forceinline__ V2<float> vfma(V2<float> a, V2<float> b, V2<float> c) {
    return __ffma2_rn(a.v, b.v, c.v);
}
__device__ __forceinline__ V2<float> operator-(V2<float> a) { return V2<float>(-a.v.x, -a.v.y); }

template <>
struct V2<double> {
    double x, y;
    __device__ __forceinline__ V2() {}
    __device__ __forceinline__ V2(double a, double b) : x(a), y(b) {}
    __device__ __forceinline__ static V2 all(double a) { return V2(a, a); }
    __device__ __forceinline__ double lo() const { return x; }
    __device__ __forceinline__ double hi() const { return y; }
};
__device__ __forceinline__ V2<double> operator+(V2<double> a, V2<double> b) {
    return {__dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y)};
}
__device__ __forceinline__ V2<double> operator*(V2<double> a, V2<double> b) {
    return {__dmul_rn(a.x, b.x), __dmul_rn(a.y, b.y)};
}
__device__ __forceinline__ V2<double> operator-(V2<double> a, V2<double> b) {
    return {__dsub_rn(a.x, b.x), __dsub_rn(a.y, b.y)};
}
__device__ __forceinline__ V2<double> vfma(V2<double> a, V2<double> b, V2<double> c) {
    return {__fma_rn(a.x, b.x, c.x), __fma_rn(a.y, b.y, c.y)};
}
__device__ __forceinline__ V2<double> operator-(V2<double> a) { return {-a.x, -a.y}; }

// psi of two densities; lane by lane the same operations, in the same order and with
// the same rounding, as eos_psi (so a site's psi does not depend on which lane or which
// kernel computes it). `hi_valid` = false: the second lane is padding and is not checked.
template <typename T, int EOS>
__device__ __forceinline__ V2<T> eos_psi2(V2<T> rho, const DevConsts<T> &P, bool hi_valid,
                                          bool &bad) {
    if constexpr (EOS == LB_EOS_CS) {
        using V = V2<T>;
        const V one = V::all(T(1));
        const V eta = V::all(P.b4) * rho;
        const V om = one - eta;
        const V poly = vfma(eta, vfma(eta, one - eta, one), one);
        const V num = (rho * V::all(P.RT)) * poly;
        const V den = (om * om) * om;
        const V q(lb_div(num.lo(), den.lo()), lb_div(num.hi(), den.hi()));
        const V p = q - V::all(P.a) * (rho * rho);
        const V arg = (p - rho * V::all(T(1.0 / 3.0))) * V::all(P.two_over_G);
        bad |= !(arg.lo() > T(0)) || !(rho.lo() > T(0));
        if (hi_valid) bad |= !(arg.hi() > T(0)) || !(rho.hi() > T(0));
        return V(lb_sqrt_pos(arg.lo()), lb_sqrt_pos(arg.hi()));
    } else {
        bool b2 = false;
        const T lo = eos_psi<T, EOS>(rho.lo(), P, bad);
        const T hi = eos_psi<T, EOS>(rho.hi(), P, b2);
        if (hi_valid) bad |= b2;
        return V2<T>(lo, hi);
    }
}

// One collision for two sites: f[9] (populations after streaming, pre-collision) and the
// potential at the sites and their neighbours pn[a] = psi(x + e_a) (pn[0] = psi(x)) give
// f*[9] in place.
//
// Arithmetic (identical in exact arithmetic to Eqs. 3, 5-8, 17-19 and f* = M^-1 m*):
//   Sx, Sy = sum_a w_a psi(x+e_a) e_a,       F = -G psi(x) (Sx, Sy)                 (Eq. 7)
//   Q = kappa G/2 psi(x) sum_a w_a (psi_a - psi) e_a e_a                           (Eq. 19)
//   v = (j + F/2) / rho                                                             (Eq. 6)
//   |F|^2 / psi^2 in Eq. 8 is evaluated as G^2 (Sx^2 + Sy^2) (no division by psi)
//   m*_rho = rho and m*_j = j + F for every s_j (relaxing j towards rho v = j + F/2 and
//   adding (1 - s_j/2) F cancels s_j exactly), so s_rho and s_j drop out;
//   m*_k = (1 - s_k) m_k + s_k m_eq_k + (1 - s_k/2) S_k + C_k for the other moments.
//   VSW: nu(rho) of Sec. V.C, the rate of p_xx, p_xy (and the weight of their source
//   terms) taken per site as s_v where rho >= rho_sw, else s_vV.
//   SH (LB_BF16): f holds the stored shifted populations f_a - w_a rho_s. The shift only
//   moves the moments rho, e and zeta (M w = (1, -2, 1, 0, ..., 0)), so those are corrected
//   by rho_s, and the same is taken off m* before M^-1 gives the shifted f* that is stored;
//   f*_0 from mass conservation reads the same in shifted terms.
template <typename T, bool VSW = false, bool SH = false>
__device__ __forceinline__ void collide_pair(V2<T> (&f)[9], const V2<T> (&pn)[9],
                                             const DevConsts<T> &P) {
    using V = V2<T>;
    const V third = V::all(T(1.0 / 3.0)), twelfth = V::all(T(1.0 / 12.0));
    const V two = V::all(T(2)), four = V::all(T(4)), half = V::all(T(0.5));
    const V pc = pn[0];

    // Eq. 7 neighbour sums and Eq. 19 differences
    const V dg_pp = pn[5] - pn[7];
    const V dg_mp = pn[6] - pn[8];
    const V Sx = vfma(third, pn[1] - pn[3], twelfth * (dg_pp - dg_mp));
    const V Sy = vfma(third, pn[2] - pn[4], twelfth * (dg_pp + dg_mp));
    const V mGpc = V::all(-P.G) * pc;
    const V Fx = mGpc * Sx;
    const V Fy = mGpc * Sy;
    const V dsum = vfma(V::all(T(-4)), pc, (pn[5] + pn[6]) + (pn[7] + pn[8]));
    const V qpre = V::all(P.kG2) * pc;
    const V tdsum = twelfth * dsum;
    const V Qxx = qpre * vfma(third, vfma(V::all(T(-2)), pc, pn[1] + pn[3]), tdsum);
    const V Qyy = qpre * vfma(third, vfma(V::all(T(-2)), pc, pn[2] + pn[4]), tdsum);
    const V Qxy = qpre * (twelfth * ((pn[5] + pn[7]) - (pn[6] + pn[8])));

    // moments m = M f
    const V ax = f[1] + f[3], ay = f[2] + f[4];
    const V d13 = f[1] - f[3], d24 = f[2] - f[4];
    const V s57 = f[5] + f[7], s68 = f[6] + f[8];
    const V d57 = f[5] - f[7], d68 = f[6] - f[8];
    const V axis = ax + ay, diag = s57 + s68;
    const V rsum = f[0] + (axis + diag);       // sum of f (of the shifted f when SH)
    V rs;                                      // rho_s in both lanes (SH)
    if constexpr (SH) rs = V::all(P.rho_s);
    V rho = rsum;
    if constexpr (SH) rho = rsum + rs;
    const V jx = d13 + (d57 - d68);
    const V jy = d24 + (d57 + d68);
    V m1 = vfma(two, diag, vfma(V::all(T(-4)), f[0], -axis));
    V m2 = vfma(four, f[0], vfma(V::all(T(-2)), axis, diag));
    if constexpr (SH) {
        m1 = vfma(V::all(T(-2)), rs, m1);
        m2 = m2 + rs;
    }
    const V m4 = vfma(V::all(T(-2)), d13, d57 - d68);
    const V m6 = vfma(V::all(T(-2)), d24, d57 + d68);
    const V m7 = ax - ay;
    const V m8 = s57 - s68;

    // Eq. 6 velocity and Eq. 3 equilibria
    const V rinv(lb_rcp(rho.lo()), lb_rcp(rho.hi()));
    const V vx = vfma(half, Fx, jx) * rinv;
    const V vy = vfma(half, Fy, jy) * rinv;
    const V vxx = vx * vx, vyy = vy * vy;
    const V v2 = vxx + vyy;
    const V meq1 = rho * vfma(V::all(T(3)), v2, V::all(T(-2)));
    const V meq2 = rho * vfma(V::all(T(-3)), v2, V::all(T(1)));
    const V rvx = rho * vx, rvy = rho * vy;
    const V meq7 = rho * (vxx - vyy);
    const V meq8 = rvx * vy;

    // Eq. 5 forcing with S_1 of Eq. 8
    const V S1 = vfma(V::all(T(6)), vfma(vx, Fx, vy * Fy), V::all(P.sig_coef) * vfma(Sx, Sx, Sy * Sy));
    const V S7 = two * (vx * Fx - vy * Fy);
    const V S8 = vfma(vx, Fy, vy * Fx);

    // Eq. 18 source
    const V tr = Qxx + Qyy;

    // Eq. 17, written as (1 - s) m + s m_eq + (1 - s/2) S + C
    const V ms0 = rho;
    V ms1 = vfma(V::all(P.e_keep), m1, vfma(V::all(P.s_e), meq1,
                  vfma(V::all(P.e_half), S1, V::all(P.e_src) * tr)));
    V ms2 = vfma(V::all(P.z_keep), m2, vfma(V::all(P.s_z), meq2,
                  -vfma(V::all(P.z_half), S1, V::all(P.z_src) * tr)));
    const V ms3 = jx + Fx;
    const V ms4 = vfma(V::all(P.q_keep), m4, -vfma(V::all(P.s_q), rvx, V::all(P.q_half) * Fx));
    const V ms5 = jy + Fy;
    const V ms6 = vfma(V::all(P.q_keep), m6, -vfma(V::all(P.s_q), rvy, V::all(P.q_half) * Fy));
    V vkeep = V::all(P.v_keep), vs = V::all(P.s_v), vhalf = V::all(P.v_half);
    V vsrc = V::all(P.v_src);
    if constexpr (VSW) {
        const bool lo = rho.lo() >= P.rho_sw, hi = rho.hi() >= P.rho_sw;
        vkeep = V(lo ? P.v_keep : P.v_keep_V, hi ? P.v_keep : P.v_keep_V);
        vs = V(lo ? P.s_v : P.s_vV, hi ? P.s_v : P.s_vV);
        vhalf = V(lo ? P.v_half : P.v_half_V, hi ? P.v_half : P.v_half_V);
        vsrc = V(lo ? P.v_src : P.v_src_V, hi ? P.v_src : P.v_src_V);
    }
    const V ms7 = vfma(vkeep, m7, vfma(vs, meq7, vfma(vhalf, S7, vsrc * (Qxx - Qyy))));
    const V ms8 = vfma(vkeep, m8, vfma(vs, meq8, vfma(vhalf, S8, vsrc * Qxy)));

    // f* = M^-1 m*, M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    if constexpr (SH) {   // back to the moments of the shifted f*
        ms1 = vfma(two, rs, ms1);
        ms2 = ms2 - rs;
    }
    const V c9 = V::all(T(1.0 / 9.0)), c18 = V::all(T(1.0 / 18.0)), c36 = V::all(T(1.0 / 36.0));
    const V c6 = V::all(T(1.0 / 6.0)), c12 = V::all(T(1.0 / 12.0)), c4 = V::all(T(0.25));
    const V a0 = c9 * (SH ? rsum : ms0);
    const V base_axis = a0 - vfma(c36, ms1, c18 * ms2);
    const V base_diag = vfma(c18, ms1, vfma(c36, ms2, a0));
    const V jx6 = c6 * ms3, qx6 = c6 * ms4, jy6 = c6 * ms5, qy6 = c6 * ms6;
    const V pxx4 = c4 * ms7, pxy4 = c4 * ms8;
    const V ax1 = jx6 - qx6, ay1 = jy6 - qy6;
    f[1] = base_axis + (ax1 + pxx4);
    f[3] = base_axis + (pxx4 - ax1);
    f[2] = base_axis + (ay1 - pxx4);
    f[4] = base_axis - (ay1 + pxx4);
    const V xp = vfma(c12, ms4, jx6), yp = vfma(c12, ms6, jy6);
    const V xy_p = xp + yp, xy_m = xp - yp;
    f[5] = base_diag + (xy_p + pxy4);
    f[6] = base_diag - (xy_m + pxy4);
    f[7] = base_diag - (xy_p - pxy4);
    f[8] = base_diag + (xy_m - pxy4);
    // f*_0 from mass conservation, rho - sum_{a>0} f*_a, instead of (m*_0 - m*_1 + m*_2)/9:
    // with the rounded constants 1/9, 1/18, 1/36 the column sums of M^-1 are not exactly
    // (1, 0, ..., 0), which in FP32 adds mass at about 7e-9 per step; this way the only
    // error is one unbiased rounding.
    f[0] = rsum - (((f[1] + f[3]) + (f[2] + f[4])) + ((f[5] + f[7]) + (f[6] + f[8])));
}

}  // namespace lbm
