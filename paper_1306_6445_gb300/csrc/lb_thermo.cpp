// Host-side thermodynamic helpers used to set up initial states (no GPU work):
// the Carnahan-Starling critical point and the Maxwell coexistence densities.
//
// Methods: T_c is the maximum over rho of the spinodal temperature
// T_sp(rho) = 2 a rho / (R d(rho Z)/drho) (golden-section search); the Maxwell rule
// (Sec. II: equal area in the specific volume v = 1/rho) is solved by bisection on the
// bulk pressure, with the area integrated by composite Simpson in v.
#include <algorithm>
#include <cmath>
#include <functional>

#include "lb_internal.h"

namespace lbm {

namespace {

double cs_pressure(double a, double b, double R, double T, double rho) {
    const double eta = b * rho / 4.0;
    const double om = 1.0 - eta;
    return rho * R * T * (1.0 + eta + eta * eta - eta * eta * eta) / (om * om * om) - a * rho * rho;
}

// d(rho Z(eta))/drho for Carnahan-Starling, closed form.
double cs_dcompress(double b, double rho) {
    const double eta = b * rho / 4.0;
    const double om = 1.0 - eta;
    const double num = 1.0 + 4.0 * eta + 4.0 * eta * eta - 4.0 * eta * eta * eta + eta * eta * eta * eta;
    return num / (om * om * om * om);
}

double golden_max(const std::function<double(double)> &f, double lo, double hi) {
    const double g = 0.5 * (std::sqrt(5.0) - 1.0);
    double x1 = hi - g * (hi - lo), x2 = lo + g * (hi - lo);
    double f1 = f(x1), f2 = f(x2);
    for (int it = 0; it < 300 && hi - lo > 1e-15 * (1.0 + std::fabs(lo)); ++it) {
        if (f1 < f2) {
            lo = x1; x1 = x2; f1 = f2; x2 = lo + g * (hi - lo); f2 = f(x2);
        } else {
            hi = x2; x2 = x1; f2 = f1; x1 = hi - g * (hi - lo); f1 = f(x1);
        }
    }
    return 0.5 * (lo + hi);
}

template <typename F>
bool bisect(F f, double lo, double hi, double &root) {
    double flo = f(lo), fhi = f(hi);
    if (!(std::isfinite(flo) && std::isfinite(fhi)) || (flo > 0) == (fhi > 0)) return false;
    for (int it = 0; it < 400; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        const double fm = f(mid);
        if ((fm > 0) == (flo > 0)) { lo = mid; flo = fm; } else { hi = mid; }
    }
    root = 0.5 * (lo + hi);
    return true;
}

}  // namespace

double p_eos_host(const lb_eos &e, double G, double rho) {
    switch (e.kind) {
        case LB_EOS_CS:
            return cs_pressure(e.a, e.b, e.R, e.T, rho);
        case LB_EOS_EXP: {
            const double psi = e.psi0 * std::exp(-e.rho0 / rho);
            return rho / 3.0 + 0.5 * G * psi * psi;
        }
        default: {
            if (rho <= e.rho1) return rho * e.theta_v;
            const double p1 = e.rho1 * e.theta_v;
            if (rho < e.rho2) return p1 + (rho - e.rho1) * e.theta_m;
            return p1 + (e.rho2 - e.rho1) * e.theta_m + (rho - e.rho2) * e.theta_l;
        }
    }
}

}  // namespace lbm

extern "C" {

lb_status lb_cs_critical(double a, double b, double R, double *Tc, double *rhoc) {
    if (!(a > 0 && b > 0 && R > 0) || !Tc || !rhoc) return LB_EINVAL;
    auto tsp = [&](double rho) { return 2.0 * a * rho / (R * lbm::cs_dcompress(b, rho)); };
    const double r = lbm::golden_max(tsp, 1e-9, 0.999 * 4.0 / b);
    *Tc = tsp(r);
    *rhoc = r;
    return LB_OK;
}

lb_status lb_maxwell(const lb_eos *eos, double G, double *rho_v, double *rho_l, double *p_b) {
    if (!eos || !rho_v || !rho_l || !p_b) return LB_EINVAL;
    const lb_eos e = *eos;
    auto p = [&](double r) { return lbm::p_eos_host(e, G, r); };
    double rmax;
    switch (e.kind) {
        case LB_EOS_CS: rmax = 0.999 * 4.0 / e.b; break;
        case LB_EOS_EXP: rmax = 10.0 * e.rho0; break;
        case LB_EOS_PIECEWISE: rmax = 10.0 * e.rho2; break;
        default: return LB_EINVAL;
    }
    // spinodals: local maximum ra and local minimum rb of p on a fine scan
    double ra = 0, rb = 0;
    if (e.kind == LB_EOS_PIECEWISE) {
        ra = e.rho1;
        rb = e.rho2;
    } else {
        const int n = 40000;
        double prev = p(rmax * 1e-5);
        int phase = 0;
        for (int i = 1; i <= n; ++i) {
            const double r = rmax * (1e-5 + (1.0 - 1e-5) * i / n);
            const double cur = p(r);
            if (phase == 0 && cur < prev) { ra = r; phase = 1; }
            else if (phase == 1 && cur > prev) { rb = r; phase = 2; break; }
            prev = cur;
        }
        if (phase != 2) return LB_EINVAL;
        const double h = rmax / n;
        ra = lbm::golden_max(p, std::max(ra - 2 * h, 1e-12), ra + h);
        rb = lbm::golden_max([&](double r) { return -p(r); }, rb - 2 * h, rb + h);
    }
    const double p_hi = p(ra);
    const double p_lo = std::max(p(rb), 1e-9 * p_hi);
    auto roots = [&](double pb, double &rv, double &rl) {
        double lo = ra * 1e-3;
        while (p(lo) > pb && lo > 1e-300) lo *= 1e-3;
        const bool a = lbm::bisect([&](double r) { return p(r) - pb; }, lo, ra, rv);
        const bool b2 = lbm::bisect([&](double r) { return p(r) - pb; }, rb, rmax, rl);
        return a && b2;
    };
    // area in v = 1/rho: A(pb) = int_{1/rl}^{1/rv} (p(1/v) - pb) dv, zero at coexistence
    auto area = [&](double pb) {
        double rv, rl;
        if (!roots(pb, rv, rl)) return std::nan("");
        const double v0 = 1.0 / rl, v1 = 1.0 / rv;
        // split at the kinks of Eq. 23 so that Simpson sees smooth pieces
        double cuts[4] = {v0, v1, v1, v1};
        int nc = 2;
        if (e.kind == LB_EOS_PIECEWISE) {
            nc = 0;
            cuts[nc++] = v0;
            if (1.0 / e.rho2 > v0 && 1.0 / e.rho2 < v1) cuts[nc++] = 1.0 / e.rho2;
            if (1.0 / e.rho1 > v0 && 1.0 / e.rho1 < v1) cuts[nc++] = 1.0 / e.rho1;
            cuts[nc++] = v1;
        }
        double total = 0.0;
        for (int k = 0; k + 1 < nc; ++k) {
            const double lo = cuts[k], hi = cuts[k + 1];
            // geometric spacing in v resolves the steep liquid end; Simpson on log(v)
            const int m = 4000;
            const double l0 = std::log(lo), l1 = std::log(hi), hstep = (l1 - l0) / m;
            double s = 0.0;
            for (int i = 0; i <= m; ++i) {
                const double lv = l0 + i * hstep, v = std::exp(lv);
                const double w = (i == 0 || i == m) ? 1.0 : (i % 2 ? 4.0 : 2.0);
                s += w * (p(1.0 / v) - pb) * v;  // dv = v d(log v)
            }
            total += s * hstep / 3.0;
        }
        return total;
    };
    const double span = p_hi - p_lo;
    double pb;
    if (!lbm::bisect(area, p_lo + 1e-12 * span, p_hi - 1e-12 * span, pb)) return LB_EINVAL;
    double rv, rl;
    if (!roots(pb, rv, rl)) return LB_EINVAL;
    *rho_v = rv;
    *rho_l = rl;
    *p_b = pb;
    return LB_OK;
}

}  // extern "C"
