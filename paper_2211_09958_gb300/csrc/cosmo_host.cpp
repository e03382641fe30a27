// Host FP64 background cosmology of the PM library: growth functions,
// growth-matched KDK factors, BBKS linear power normalised to sigma8.
//
// The paper (pmwd, arXiv:2211.09958) names growth-factor based integration
// of a cosmological PM simulation but prints no formulas.  This file uses the
// standard flat-LCDM forms (H0 = 1):
//   E(a)^2 = Om a^-3 + 1 - Om
//   D'' + (3/a + E'/E) D' - 3 Om / (2 a^5 E^2) D = 0              (D1)
//   same operator on D2 with source -3 Om / (2 a^5 E^2) D1^2      (D2)
//   started at a = 1e-5 with D1 = a, D2 = -3/7 a^2, normalised to D1(1) = 1.
//   g_p = a^3 E D1', g_f = 3/2 Om D1 (force growth)
//   kick  K(a->b; c) = (g_p(b) - g_p(a)) / g_f(c)
//   drift Dr(a->b; c) = (D1(b) - D1(a)) / g_p(c)
//   step n: K_a = K(a_n -> a_h; a_n), Dr = Dr(a_n -> a_{n+1}; a_h),
//           K_b = K(a_h -> a_{n+1}; a_{n+1}), a_h = (a_n + a_{n+1}) / 2,
//           a_n uniform between a_init and a_final (or, with the log-a
//           solver flag, uniform in ln a with a_h the geometric midpoint).
//   P(k) = A k^ns T_BBKS(k / (Om h))^2, A from the top-hat sigma8 integral.
// Integration: classical RK4 in ln a with steps <= 1e-3; sigma8 integral:
// composite Simpson in ln k over [1e-5, 1e3] h/Mpc, 10^4 intervals.
// Om derivatives: central differences with dOm = 1e-5.  With solver flag 16
// the growth quantities come from the growth-function emulator
// (growth_emulator.cpp) instead of the ODE solve.

#include <algorithm>
#include <cmath>
#include <vector>

#include "pm_internal.h"

namespace pmgb {

namespace {

constexpr double kAStart = 1e-5;
constexpr double kMaxStep = 1e-3;  // in ln a
constexpr double kFdOmega = 1e-5;

struct GrowthState {
    double d1, v1, d2, v2;  // D1, dD1/da, D2, dD2/da
};

GrowthState deriv_lna(double lna, const GrowthState &y, double om) {
    const double a = std::exp(lna);
    const double e2 = om / (a * a * a) + (1.0 - om);
    const double dlne = -1.5 * om / (a * a * a * a) / e2;
    const double damp = 3.0 / a + dlne;
    const double src = 1.5 * om / (a * a * a * a * a * e2);
    GrowthState r;
    r.d1 = a * y.v1;
    r.v1 = a * (-damp * y.v1 + src * y.d1);
    r.d2 = a * y.v2;
    r.v2 = a * (-damp * y.v2 + src * (y.d2 - y.d1 * y.d1));
    return r;
}

GrowthState axpy(const GrowthState &y, double h, const GrowthState &k) {
    return {y.d1 + h * k.d1, y.v1 + h * k.v1, y.d2 + h * k.d2, y.v2 + h * k.v2};
}

void rk4(double &t, GrowthState &y, double h, double om) {
    GrowthState k1 = deriv_lna(t, y, om);
    GrowthState k2 = deriv_lna(t + 0.5 * h, axpy(y, 0.5 * h, k1), om);
    GrowthState k3 = deriv_lna(t + 0.5 * h, axpy(y, 0.5 * h, k2), om);
    GrowthState k4 = deriv_lna(t + h, axpy(y, h, k3), om);
    y.d1 += h / 6.0 * (k1.d1 + 2 * k2.d1 + 2 * k3.d1 + k4.d1);
    y.v1 += h / 6.0 * (k1.v1 + 2 * k2.v1 + 2 * k3.v1 + k4.v1);
    y.d2 += h / 6.0 * (k1.d2 + 2 * k2.d2 + 2 * k3.d2 + k4.d2);
    y.v2 += h / 6.0 * (k1.v2 + 2 * k2.v2 + 2 * k3.v2 + k4.v2);
    t += h;
}

}  // namespace

double hubble_e(double a, double om) { return std::sqrt(om / (a * a * a) + (1.0 - om)); }

void growth_at(double om, const std::vector<double> &a, std::vector<Growth> *out) {
    std::vector<double> pts(a);
    pts.push_back(1.0);
    std::sort(pts.begin(), pts.end());
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    std::vector<GrowthState> at(pts.size());
    GrowthState y{kAStart, 1.0, -3.0 / 7.0 * kAStart * kAStart, -6.0 / 7.0 * kAStart};
    double t = std::log(kAStart);
    for (size_t i = 0; i < pts.size(); ++i) {
        const double t1 = std::log(pts[i]);
        const double span = t1 - t;
        if (span > 0) {
            const int nsub = std::max(1, (int)std::ceil(span / kMaxStep));
            const double h = span / nsub;
            for (int k = 0; k < nsub; ++k) rk4(t, y, h, om);
        }
        t = t1;
        at[i] = y;
    }
    const size_t i1 = std::lower_bound(pts.begin(), pts.end(), 1.0) - pts.begin();
    const double norm = at[i1].d1;
    out->resize(a.size());
    for (size_t i = 0; i < a.size(); ++i) {
        const size_t j = std::lower_bound(pts.begin(), pts.end(), a[i]) - pts.begin();
        const GrowthState &g = at[j];
        const double e = hubble_e(a[i], om);
        const double ai = a[i];
        Growth r;
        r.D1 = g.d1 / norm;
        r.dD1 = g.v1 / norm;
        r.D2 = g.d2 / (norm * norm);
        r.dD2 = g.v2 / (norm * norm);
        r.gp = ai * ai * ai * e * r.dD1;
        r.gp2 = ai * ai * ai * e * r.dD2;
        r.gf = 1.5 * om * r.D1;
        (*out)[i] = r;
    }
}

double step_a(const Params &p, int n) {
    if (p.solver & 4) return p.a_init * std::pow(p.a_final / p.a_init, (double)n / p.n_steps);
    return p.a_init + (p.a_final - p.a_init) * n / p.n_steps;
}

double half_step_a(const Params &p, int n) {
    if (p.solver & 4) return std::sqrt(step_a(p, n) * step_a(p, n + 1));
    return 0.5 * (step_a(p, n) + step_a(p, n + 1));
}

namespace {
// Growth quantities at a: the ODE solve, or with the emulator solver flag
// (16) the growth-function emulator.
void growth_values(const Params &p, double om, const std::vector<double> &a, std::vector<Growth> *out) {
    if (p.solver & 16)
        growth_emulated(om, a, out);
    else
        growth_at(om, a, out);
}

void kdk_factors(double om, const Params &p, std::vector<double> *ka, std::vector<double> *dr,
                 std::vector<double> *kb) {
    const int n_steps = p.n_steps;
    std::vector<double> a(n_steps + 1), ah(n_steps);
    for (int n = 0; n <= n_steps; ++n) a[n] = step_a(p, n);
    for (int n = 0; n < n_steps; ++n) ah[n] = half_step_a(p, n);
    std::vector<double> all(a);
    all.insert(all.end(), ah.begin(), ah.end());
    std::vector<Growth> g;
    growth_values(p, om, all, &g);
    ka->resize(n_steps);
    dr->resize(n_steps);
    kb->resize(n_steps);
    for (int n = 0; n < n_steps; ++n) {
        const Growth &g0 = g[n], &g1 = g[n + 1], &gh = g[n_steps + 1 + n];
        (*ka)[n] = (gh.gp - g0.gp) / g0.gf;
        (*dr)[n] = (g1.D1 - g0.D1) / gh.gp;
        (*kb)[n] = (g1.gp - gh.gp) / g1.gf;
    }
}
}  // namespace

void lpt_factors(double om, double a_init, double out[4], const Params *p) {
    std::vector<Growth> g;
    if (p)
        growth_values(*p, om, {a_init}, &g);
    else
        growth_at(om, {a_init}, &g);
    out[0] = g[0].D1;
    out[1] = g[0].D2;
    out[2] = g[0].gp;
    out[3] = g[0].gp2;
}

double bbks_transfer(double k, double om, double h) {
    const double q = k / (om * h);
    const double x = 2.34 * q;
    const double lead = x > 1e-8 ? std::log1p(x) / x : 1.0 - 0.5 * x;
    const double poly = 1.0 + 3.89 * q + std::pow(16.1 * q, 2) + std::pow(5.46 * q, 3) + std::pow(6.71 * q, 4);
    return lead * std::pow(poly, -0.25);
}

namespace {
// 3 (sin x - x cos x) / x^3.  The closed form cancels below x ~ 0.1 (relative
// error ~ eps / x^2), so there it is summed as its Taylor series
// sum_m (-1)^m 6 (m + 1) x^(2m) / (2m + 3)!, m = 0..4.
double tophat(double x) {
    if (std::fabs(x) < 0.1) {
        const double y = x * x;
        return 1.0 - y / 10.0 + y * y / 280.0 - y * y * y / 15120.0 + y * y * y * y / 1330560.0;
    }
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}
}  // namespace

double power_amplitude(double om, double s8, double h, double ns) {
    const int m = 10000;
    const double lo = std::log(1e-5), hi = std::log(1e3), dl = (hi - lo) / m;
    double acc = 0.0;
    for (int i = 0; i <= m; ++i) {
        const double k = std::exp(lo + i * dl);
        const double t = bbks_transfer(k, om, h);
        const double w = tophat(8.0 * k);
        const double f = k * k * k * std::pow(k, ns) * t * t * w * w;
        const double c = (i == 0 || i == m) ? 1.0 : (i % 2 ? 4.0 : 2.0);
        acc += c * f;
    }
    const double sig2_unit = acc * dl / 3.0 / (2.0 * M_PI * M_PI);
    return s8 * s8 / sig2_unit;
}

void host_tables(const Params &p, double om, double s8, HostTables *t) {
    kdk_factors(om, p, &t->ka, &t->dr, &t->kb);
    std::vector<double> ka_u, dr_u, kb_u, ka_d, dr_d, kb_d;
    kdk_factors(om + kFdOmega, p, &ka_u, &dr_u, &kb_u);
    kdk_factors(om - kFdOmega, p, &ka_d, &dr_d, &kb_d);
    t->dka.resize(p.n_steps);
    t->ddr.resize(p.n_steps);
    t->dkb.resize(p.n_steps);
    for (int n = 0; n < p.n_steps; ++n) {
        t->dka[n] = (ka_u[n] - ka_d[n]) / (2 * kFdOmega);
        t->ddr[n] = (dr_u[n] - dr_d[n]) / (2 * kFdOmega);
        t->dkb[n] = (kb_u[n] - kb_d[n]) / (2 * kFdOmega);
    }
    lpt_factors(om, p.a_init, t->lpt, &p);
    double up[4], dn[4];
    lpt_factors(om + kFdOmega, p.a_init, up, &p);
    lpt_factors(om - kFdOmega, p.a_init, dn, &p);
    for (int i = 0; i < 4; ++i) t->dlpt[i] = (up[i] - dn[i]) / (2 * kFdOmega);
    t->amp = power_amplitude(om, s8, p.h, p.n_s);
    t->dlnamp = (std::log(power_amplitude(om + kFdOmega, s8, p.h, p.n_s)) -
                 std::log(power_amplitude(om - kFdOmega, s8, p.h, p.n_s))) /
                (2 * kFdOmega);
}

}  // namespace pmgb
