// Device-side building blocks of the D2Q9 MRT pseudopotential update.
//
// Velocity order e_0..e_8 = (0,0),(1,0),(0,1),(-1,0),(0,-1),(1,1),(-1,1),(-1,-1),(1,-1);
// moment order (rho, e, zeta, j_x, q_x, j_y, q_y, p_xx, p_xy) of the standard D2Q9
// transformation matrix M (Sec. II). All constants below are written out by hand.
#pragma once

#include <cuda_runtime.h>

#include "lb_internal.h"

namespace lbm {

template <typename T>
struct DevConsts {
    T a, b4, RT;
    T psi0, rho0;
    T th_v, th_m, th_l, rho1, rho2, p_rho1, p_rho2;
    T two_over_G;
    T G, kG2, sig_coef;
    T s_e, s_z, s_q, s_v;
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
    return d;
}

__device__ __forceinline__ float lb_exp(float v) { return expf(v); }
__device__ __forceinline__ double lb_exp(double v) { return exp(v); }
__device__ __forceinline__ float lb_sqrt(float v) { return sqrtf(v); }
__device__ __forceinline__ double lb_sqrt(double v) { return sqrt(v); }

// Interaction potential psi(rho) (Sec. II): psi0 exp(-rho0/rho), or
// sqrt(2 (p_EOS - rho c_s^2) / G) with p_EOS the Carnahan-Starling EOS or Eq. 23.
// Sets `bad` when rho <= 0 or psi^2 < 0 (the value is then NaN/inf and must not be used).
template <typename T, int EOS>
__device__ __forceinline__ T eos_psi(T rho, const DevConsts<T> &P, bool &bad) {
    if constexpr (EOS == LB_EOS_EXP) {
        bad |= !(rho > T(0));
        return P.psi0 * lb_exp(-P.rho0 / rho);
    } else {
        T p;
        if constexpr (EOS == LB_EOS_CS) {
            const T eta = P.b4 * rho;
            const T om = T(1) - eta;
            p = rho * P.RT * (T(1) + eta * (T(1) + eta * (T(1) - eta))) / (om * om * om)
                - P.a * rho * rho;
        } else {
            p = (rho <= P.rho1) ? rho * P.th_v
              : (rho < P.rho2) ? P.p_rho1 + (rho - P.rho1) * P.th_m
                               : P.p_rho2 + (rho - P.rho2) * P.th_l;
        }
        const T arg = (p - rho * T(1.0 / 3.0)) * P.two_over_G;
        bad |= !(arg >= T(0)) || !(rho > T(0));
        return lb_sqrt(arg);
    }
}

// One site's collision: f[9] (post-streaming populations at x) and the potential at x
// and its eight neighbours pn[a] = psi(x + e_a) (pn[0] = psi(x)) give f*[9] in place.
//
// Arithmetic (identical in exact arithmetic to Eqs. 3, 5-8, 17-19 and f* = M^-1 m*):
//   Sx, Sy = sum_a w_a psi(x+e_a) e_a,       F = -G psi(x) (Sx, Sy)                 (Eq. 7)
//   Q = kappa G/2 psi(x) sum_a w_a (psi_a - psi) e_a e_a                           (Eq. 19)
//   v = (j + F/2) / rho                                                             (Eq. 6)
//   |F|^2 / psi^2 in Eq. 8 is evaluated as G^2 (Sx^2 + Sy^2) (no division by psi)
//   m*_rho = rho and m*_j = j + F for every s_j (the relaxation of j towards
//   rho v = j + F/2 plus (1 - s_j/2) F cancels s_j exactly), so s_rho and s_j drop out.
template <typename T>
__device__ __forceinline__ void collide_site(T (&f)[9], const T (&pn)[9], const DevConsts<T> &P) {
    const T pc = pn[0];
    const T third = T(1.0 / 3.0), twelfth = T(1.0 / 12.0);

    // Eq. 7 neighbour sums and Eq. 19 differences
    const T dg_pp = pn[5] - pn[7];   // (1,1) - (-1,-1)
    const T dg_mp = pn[6] - pn[8];   // (-1,1) - (1,-1)
    const T Sx = third * (pn[1] - pn[3]) + twelfth * (dg_pp - dg_mp);
    const T Sy = third * (pn[2] - pn[4]) + twelfth * (dg_pp + dg_mp);
    const T Fx = -P.G * pc * Sx;
    const T Fy = -P.G * pc * Sy;
    const T dsum = (pn[5] + pn[6]) + (pn[7] + pn[8]) - T(4) * pc;
    const T qpre = P.kG2 * pc;
    const T Qxx = qpre * (third * (pn[1] + pn[3] - T(2) * pc) + twelfth * dsum);
    const T Qyy = qpre * (third * (pn[2] + pn[4] - T(2) * pc) + twelfth * dsum);
    const T Qxy = qpre * twelfth * ((pn[5] + pn[7]) - (pn[6] + pn[8]));

    // moments m = M f
    const T ax = f[1] + f[3], ay = f[2] + f[4];
    const T d13 = f[1] - f[3], d24 = f[2] - f[4];
    const T s57 = f[5] + f[7], s68 = f[6] + f[8];
    const T d57 = f[5] - f[7], d68 = f[6] - f[8];
    const T axis = ax + ay, diag = s57 + s68;
    const T rho = f[0] + axis + diag;
    const T jx = d13 + d57 - d68;
    const T jy = d24 + d57 + d68;
    const T m1 = T(-4) * f[0] - axis + T(2) * diag;
    const T m2 = T(4) * f[0] - T(2) * axis + diag;
    const T m4 = T(-2) * d13 + d57 - d68;
    const T m6 = T(-2) * d24 + d57 + d68;
    const T m7 = ax - ay;
    const T m8 = s57 - s68;

    // Eq. 6 velocity and Eq. 3 equilibria
    const T rinv = T(1) / rho;
    const T vx = (jx + T(0.5) * Fx) * rinv;
    const T vy = (jy + T(0.5) * Fy) * rinv;
    const T v2 = vx * vx + vy * vy;
    const T meq1 = rho * (T(-2) + T(3) * v2);
    const T meq2 = rho * (T(1) - T(3) * v2);
    const T meq4 = -rho * vx;
    const T meq6 = -rho * vy;
    const T meq7 = rho * (vx * vx - vy * vy);
    const T meq8 = rho * vx * vy;

    // Eq. 5 forcing with S_1 of Eq. 8
    const T S1 = T(6) * (vx * Fx + vy * Fy) + P.sig_coef * (Sx * Sx + Sy * Sy);
    const T S7 = T(2) * (vx * Fx - vy * Fy);
    const T S8 = vx * Fy + vy * Fx;

    // Eq. 18 source
    const T tr = Qxx + Qyy;

    // Eq. 17
    const T ms0 = rho;
    const T ms1 = m1 - P.s_e * (m1 - meq1) + (T(1) - T(0.5) * P.s_e) * S1 + T(1.5) * P.s_e * tr;
    const T ms2 = m2 - P.s_z * (m2 - meq2) - (T(1) - T(0.5) * P.s_z) * S1 - T(1.5) * P.s_z * tr;
    const T ms3 = jx + Fx;
    const T ms4 = m4 - P.s_q * (m4 - meq4) - (T(1) - T(0.5) * P.s_q) * Fx;
    const T ms5 = jy + Fy;
    const T ms6 = m6 - P.s_q * (m6 - meq6) - (T(1) - T(0.5) * P.s_q) * Fy;
    const T ms7 = m7 - P.s_v * (m7 - meq7) + (T(1) - T(0.5) * P.s_v) * S7 - P.s_v * (Qxx - Qyy);
    const T ms8 = m8 - P.s_v * (m8 - meq8) + (T(1) - T(0.5) * P.s_v) * S8 - P.s_v * Qxy;

    // f* = M^-1 m*, M^-1 = M^T diag(1/9, 1/36, 1/36, 1/6, 1/12, 1/6, 1/12, 1/4, 1/4)
    const T c9 = T(1.0 / 9.0), c18 = T(1.0 / 18.0), c36 = T(1.0 / 36.0);
    const T c6 = T(1.0 / 6.0), c12 = T(1.0 / 12.0), c4 = T(0.25);
    const T a0 = c9 * ms0;
    const T base_axis = a0 - c36 * ms1 - c18 * ms2;
    const T base_diag = a0 + c18 * ms1 + c36 * ms2;
    const T jx6 = c6 * ms3, qx6 = c6 * ms4, jy6 = c6 * ms5, qy6 = c6 * ms6;
    const T qx12 = c12 * ms4, qy12 = c12 * ms6;
    const T pxx4 = c4 * ms7, pxy4 = c4 * ms8;
    f[0] = a0 - c9 * ms1 + c9 * ms2;
    f[1] = base_axis + jx6 - qx6 + pxx4;
    f[3] = base_axis - jx6 + qx6 + pxx4;
    f[2] = base_axis + jy6 - qy6 - pxx4;
    f[4] = base_axis - jy6 + qy6 - pxx4;
    const T xp = jx6 + qx12, yp = jy6 + qy12;
    f[5] = base_diag + xp + yp + pxy4;
    f[6] = base_diag - xp + yp - pxy4;
    f[7] = base_diag - xp - yp + pxy4;
    f[8] = base_diag + xp - yp - pxy4;
}

}  // namespace lbm
