// Growth-function emulator: D1, D2, their derivatives in a and in Omega_m,
// over Omega_m in [0.1, 0.6] and a in [1e-3, 1], from a two-dimensional
// Chebyshev series instead of one growth ODE solve per cosmology.
//
// The paper (pmwd, arXiv:2211.09958) names a growth-function emulator as
// separate, adjacent work (Statement of Need) without describing it; this
// is the library's own.  It is built once per process from the ODE solve of
// cosmo_host.cpp (growth_at): the smooth functions
//   f0 = D1 / a,  f1 = dD1/da,  f2 = D2 / a^2,  f3 = (dD2/da) / a
// (f0 -> 1, f1 -> 1, f2 -> -3/7, f3 -> -6/7 in matter domination) are sampled
// at the tensor product of NU Chebyshev-Gauss nodes in u (a in [0, 1] mapped
// to [-1, 1]) and NV in v (Omega_m mapped to [-1, 1]), NV ODE solves in all,
// and their Chebyshev coefficients c_q[m][n] follow from the discrete
// orthogonality of T_n at those nodes.  Evaluation sums
// f = sum_mn c[m][n] T_m(v) T_n(u); d/dv takes T_m' = m U_{m-1}.
// The series converge geometrically, at a rate set by the nearest complex
// singularity: in a, where E(a)^2 = 0 (a^3 = -Om / (1 - Om), |a| ~ 0.75, well
// off the interval; in ln a it would sit only pi/3 away and the series would
// need hundreds of terms), in Omega_m at 0 and 1.  48 x 32 terms reproduce
// the ODE solve to ~1e-11.

#include <cmath>
#include <vector>

#include "../../include/pmgb.h"
#include "pm_internal.h"

namespace pmgb {

namespace {

constexpr int kNU = 48, kNV = 32, kNQ = 4;
constexpr double kOmLo = 0.1, kOmHi = 0.6, kALo = 1e-3, kAHi = 1.0;

struct Series {
    double c[kNQ][kNV][kNU];
};

// T_0 .. T_{N-1} and their derivatives at x.
template <int N>
void cheb(double x, double (&t)[N], double (&dt)[N]) {
    double u[N];  // U_0 .. U_{N-1}
    t[0] = 1.0;
    u[0] = 1.0;
    if (N > 1) {
        t[1] = x;
        u[1] = 2.0 * x;
    }
    for (int n = 2; n < N; ++n) {
        t[n] = 2.0 * x * t[n - 1] - t[n - 2];
        u[n] = 2.0 * x * u[n - 1] - u[n - 2];
    }
    dt[0] = 0.0;
    for (int n = 1; n < N; ++n) dt[n] = n * u[n - 1];
}

const Series &build() {
    static Series s;
    std::vector<double> a(kNU);
    double xv[kNV];
    for (int j = 0; j < kNU; ++j) a[j] = 0.5 * (1.0 + std::cos(M_PI * (j + 0.5) / kNU));  // a in (0, 1)
    for (int i = 0; i < kNV; ++i) xv[i] = std::cos(M_PI * (i + 0.5) / kNV);
    static double f[kNQ][kNV][kNU];
    for (int i = 0; i < kNV; ++i) {
        const double om = 0.5 * (kOmLo + kOmHi) + 0.5 * (kOmHi - kOmLo) * xv[i];
        std::vector<Growth> g;
        growth_at(om, a, &g);
        for (int j = 0; j < kNU; ++j) {
            f[0][i][j] = g[j].D1 / a[j];
            f[1][i][j] = g[j].dD1;
            f[2][i][j] = g[j].D2 / (a[j] * a[j]);
            f[3][i][j] = g[j].dD2 / a[j];
        }
    }
    // c[m][n] = (2 - delta_m0)(2 - delta_n0) / (NV NU) sum_ij f_ij T_m(v_i) T_n(u_j)
    for (int q = 0; q < kNQ; ++q)
        for (int m = 0; m < kNV; ++m)
            for (int n = 0; n < kNU; ++n) {
                double acc = 0.0;
                for (int i = 0; i < kNV; ++i) {
                    const double tv = std::cos(m * M_PI * (i + 0.5) / kNV);
                    for (int j = 0; j < kNU; ++j) acc += f[q][i][j] * tv * std::cos(n * M_PI * (j + 0.5) / kNU);
                }
                s.c[q][m][n] = (m ? 2.0 : 1.0) * (n ? 2.0 : 1.0) / (kNV * kNU) * acc;
            }
    return s;
}

const Series &series() {
    static const Series &s = build();  // built once, thread-safe initialisation
    return s;
}

}  // namespace

bool growth_emulator_covers(double om, double a) {
    return om >= kOmLo && om <= kOmHi && a >= kALo && a <= kAHi;
}

// out[8]: D1, D2, dD1/da, dD2/da, dD1/dOm, dD2/dOm, d(dD1/da)/dOm, d(dD2/da)/dOm.
void growth_emulate(double om, double a, double out[8]) {
    const Series &s = series();
    const double u = 2.0 * a - 1.0;
    const double v = (2.0 * om - (kOmLo + kOmHi)) / (kOmHi - kOmLo);
    const double dvdom = 2.0 / (kOmHi - kOmLo);
    double tu[kNU], dtu[kNU], tv[kNV], dtv[kNV];  // dtu unused: dD/da is emulated directly
    cheb<kNU>(u, tu, dtu);
    cheb<kNV>(v, tv, dtv);
    double f[kNQ], fv[kNQ];
    for (int q = 0; q < kNQ; ++q) {
        double acc = 0.0, accv = 0.0;
        for (int m = 0; m < kNV; ++m) {
            double row = 0.0;
            for (int n = 0; n < kNU; ++n) row += s.c[q][m][n] * tu[n];
            acc += tv[m] * row;
            accv += dtv[m] * row;
        }
        f[q] = acc;
        fv[q] = accv * dvdom;
    }
    out[0] = a * f[0];
    out[1] = a * a * f[2];
    out[2] = f[1];
    out[3] = a * f[3];
    out[4] = a * fv[0];
    out[5] = a * a * fv[2];
    out[6] = fv[1];
    out[7] = a * fv[3];
}

void growth_emulated(double om, const std::vector<double> &a, std::vector<Growth> *out) {
    out->resize(a.size());
    for (size_t i = 0; i < a.size(); ++i) {
        double e[8];
        growth_emulate(om, a[i], e);
        const double ai = a[i], h = hubble_e(ai, om);
        Growth &r = (*out)[i];
        r.D1 = e[0];
        r.D2 = e[1];
        r.dD1 = e[2];
        r.dD2 = e[3];
        r.gp = ai * ai * ai * h * r.dD1;
        r.gp2 = ai * ai * ai * h * r.dD2;
        r.gf = 1.5 * om * r.D1;
    }
}

}  // namespace pmgb

extern "C" int pm_growth_emulate(double omega_m, int32_t n, const double *a, double *out) {
    if (n < 0 || (n > 0 && (!a || !out))) return PM_EINVAL;
    for (int32_t i = 0; i < n; ++i)
        if (!pmgb::growth_emulator_covers(omega_m, a[i])) return PM_ERANGE;
    for (int32_t i = 0; i < n; ++i) pmgb::growth_emulate(omega_m, a[i], out + 8 * (size_t)i);
    return PM_OK;
}
