"""Background cosmology for the PM oracle (FP64, test infrastructure only).

The paper (Summary) names a cosmological PM simulation with gradients with
respect to cosmological parameters but prints no formulas; everything below
is the standard flat-LCDM reading:

* E(a) = sqrt(Om a^-3 + 1 - Om), Hubble units H0 = 1            [reading]
* growth ODE in a for D1 and the second-order D2                 [reading]
    D'' + (3/a + E'/E) D' - 3 Om / (2 a^5 E^2) D = 0
    D2'' + (3/a + E'/E) D2' - 3 Om / (2 a^5 E^2) D2 = -3 Om / (2 a^5 E^2) D1^2
  started in matter domination (D1 = a, D2 = -3/7 a^2) and normalised to
  D1(1) = 1, D2 by the same factor squared.
* momentum p = a^3 E dx/da; growth of p: g_p(a) = a^3 E D1'(a); force growth
  g_f(a) = a^2 E g_p'(a) = 3/2 Om D1(a) (by the ODE)                [reading]
* growth-matched kick/drift factors (FastPM form, cited by the paper in its
  Statement of Need):                                              [reading]
    kick  K(a->b; c) = (g_p(b) - g_p(a)) / g_f(c)
    drift Dr(a->b; c) = (D1(b) - D1(a)) / g_p(c)
* BBKS linear transfer with shape Gamma = Om h, P = A k^ns T^2, A fixed by
  sigma8 (top hat, R = 8 Mpc/h), Simpson in ln k on [1e-5, 1e3] h/Mpc with
  1e4 intervals                                                     [reading]
"""

from dataclasses import dataclass, replace

import numpy as np
from scipy.integrate import solve_ivp

A_START = 1e-5          # start of the growth integration (matter era)
SIGMA8_R = 8.0          # Mpc/h
LNK_MIN, LNK_MAX, LNK_INTERVALS = np.log(1e-5), np.log(1e3), 10000
FD_OMEGA = 1e-5         # central-difference step for d/dOm of host tables


@dataclass(frozen=True)
class Cosmology:
    omega_m: float = 0.3
    sigma8: float = 0.8
    h: float = 0.7
    n_s: float = 0.96

    def with_omega_m(self, om):
        return replace(self, omega_m=float(om))


def hubble_e(a, om):
    """E(a) = H(a)/H0 for flat LCDM without radiation [reading]."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(om * a ** -3 + (1.0 - om))


def _dlne_da(a, om):
    e2 = om * a ** -3 + (1.0 - om)
    return -1.5 * om * a ** -4 / e2


def _growth_rhs(lna, y, om):
    # y = (D1, dD1/da, D2, dD2/da); returns d/dlna = a d/da
    a = np.exp(lna)
    d1, v1, d2, v2 = y
    e2 = om * a ** -3 + (1.0 - om)
    damp = 3.0 / a + _dlne_da(a, om)
    src = 1.5 * om / (a ** 5 * e2)
    acc1 = -damp * v1 + src * d1
    acc2 = -damp * v2 + src * (d2 - d1 * d1)
    return a * np.array([v1, acc1, v2, acc2])


def growth(a, om):
    """D1, D1', D2, D2' (prime = d/da) at scale factors ``a``, normalised to
    D1(1) = 1.  Returns a dict of arrays shaped like ``a``."""
    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    pts = np.unique(np.concatenate([a.ravel(), [1.0]]))
    y0 = [A_START, 1.0, -3.0 / 7.0 * A_START ** 2, -6.0 / 7.0 * A_START]
    sol = solve_ivp(_growth_rhs, (np.log(A_START), np.log(pts[-1])), y0,
                    method="DOP853", t_eval=np.log(pts), rtol=1e-13,
                    atol=1e-30, args=(om,))
    if not sol.success:
        raise RuntimeError(sol.message)
    ys = sol.y
    i1 = np.searchsorted(pts, 1.0)
    norm = ys[0, i1]
    idx = np.searchsorted(pts, a.ravel())
    out = {
        "D1": ys[0, idx] / norm,
        "dD1": ys[1, idx] / norm,
        "D2": ys[2, idx] / norm ** 2,
        "dD2": ys[3, idx] / norm ** 2,
    }
    return {k: v.reshape(a.shape) for k, v in out.items()}


def growth_tables(a, om):
    """Growth quantities used by the integrator at scale factors ``a``."""
    g = growth(a, om)
    e = hubble_e(a, om)
    a = np.asarray(a, dtype=np.float64)
    g["E"] = e
    g["gp"] = a ** 3 * e * g["dD1"]          # momentum growth of the 1st order
    g["gp2"] = a ** 3 * e * g["dD2"]         # momentum growth of the 2nd order
    g["gf"] = 1.5 * om * g["D1"]             # force growth = a^2 E gp'
    return g


def time_grid(a_init, a_final, n_steps, log_a=False):
    """Uniform steps in a, half steps at the arithmetic midpoint [reading];
    with ``log_a`` uniform in ln a, half steps at the geometric midpoint (the
    solver variant)."""
    if log_a:
        a = a_init * (a_final / a_init) ** (np.arange(n_steps + 1) / n_steps)
        return a, np.sqrt(a[:-1] * a[1:])
    a = a_init + (a_final - a_init) * np.arange(n_steps + 1) / n_steps
    return a, 0.5 * (a[:-1] + a[1:])


def kdk_coefficients(cosmo, a_init, a_final, n_steps, log_a=False):
    """Per step n: K_a (first half kick, force at a_n), Dr (drift, momentum at
    a_{n+1/2}), K_b (second half kick, force at a_{n+1})."""
    a, ah = time_grid(a_init, a_final, n_steps, log_a)
    g = growth_tables(np.concatenate([a, ah]), cosmo.omega_m)
    n = n_steps
    gp_a, gp_h = g["gp"][: n + 1], g["gp"][n + 1:]
    gf_a = g["gf"][: n + 1]
    d1_a = g["D1"][: n + 1]
    k_a = (gp_h - gp_a[:-1]) / gf_a[:-1]
    drift = (d1_a[1:] - d1_a[:-1]) / gp_h
    k_b = (gp_a[1:] - gp_h) / gf_a[1:]
    return {"a": a, "ah": ah, "K_a": k_a, "Dr": drift, "K_b": k_b}


def kdk_coefficients_domega(cosmo, a_init, a_final, n_steps, log_a=False):
    """d(K_a, Dr, K_b)/dOm by central differences of the FP64 tables."""
    up = kdk_coefficients(cosmo.with_omega_m(cosmo.omega_m + FD_OMEGA), a_init, a_final, n_steps, log_a)
    dn = kdk_coefficients(cosmo.with_omega_m(cosmo.omega_m - FD_OMEGA), a_init, a_final, n_steps, log_a)
    return {k: (up[k] - dn[k]) / (2 * FD_OMEGA) for k in ("K_a", "Dr", "K_b")}


def lpt_growth(cosmo, a_init):
    """(D1, D2, g1, g2) at a_init: s = D1 s1 + D2 s2, p = g1 s1 + g2 s2."""
    g = growth_tables(np.array([a_init]), cosmo.omega_m)
    return np.array([g["D1"][0], g["D2"][0], g["gp"][0], g["gp2"][0]])


def lpt_growth_domega(cosmo, a_init):
    up = lpt_growth(cosmo.with_omega_m(cosmo.omega_m + FD_OMEGA), a_init)
    dn = lpt_growth(cosmo.with_omega_m(cosmo.omega_m - FD_OMEGA), a_init)
    return (up - dn) / (2 * FD_OMEGA)


# ---------------------------------------------------------------- power ----

def bbks_transfer(k, om, h):
    """BBKS transfer function with Gamma = Om h, k in h/Mpc [reading]."""
    k = np.asarray(k, dtype=np.float64)
    q = k / (om * h)
    with np.errstate(divide="ignore", invalid="ignore"):
        x = 2.34 * q
        lead = np.where(x > 1e-8, np.log1p(x) / np.where(x > 0, x, 1.0), 1.0 - 0.5 * x)
    poly = 1.0 + 3.89 * q + (16.1 * q) ** 2 + (5.46 * q) ** 3 + (6.71 * q) ** 4
    return lead * poly ** -0.25


def tophat_window(x):
    """W(x) = 3 (sin x - x cos x) / x^3.  Below x = 0.1 the closed form loses
    about eps / x^2 to cancellation, so there it takes the Taylor series
    W = sum_m (-1)^m 6 (m + 1) x^(2m) / (2m + 3)!, through m = 4 (the next
    term is below 1e-18)."""
    x = np.asarray(x, dtype=np.float64)
    small = np.abs(x) < 0.1
    xs = np.where(small, 1.0, x)
    big = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs ** 3
    x2 = x * x
    series = 1.0 + x2 * (-1.0 / 10.0 + x2 * (1.0 / 280.0 + x2 * (-1.0 / 15120.0 + x2 / 1330560.0)))
    return np.where(small, series, big)


def _simpson_lnk(f_of_k):
    lnk = np.linspace(LNK_MIN, LNK_MAX, LNK_INTERVALS + 1)
    k = np.exp(lnk)
    y = f_of_k(k)
    w = np.ones_like(lnk)
    w[1:-1:2] = 4.0
    w[2:-1:2] = 2.0
    return (lnk[1] - lnk[0]) / 3.0 * np.sum(w * y)


def unnormalised_power(k, cosmo):
    k = np.asarray(k, dtype=np.float64)
    return k ** cosmo.n_s * bbks_transfer(k, cosmo.omega_m, cosmo.h) ** 2


def sigma8_integral(power_fn):
    """sigma_8^2 = 1/(2 pi^2) int k^3 P(k) W(kR)^2 dlnk (Simpson in ln k)."""
    return _simpson_lnk(lambda k: k ** 3 * power_fn(k) * tophat_window(k * SIGMA8_R) ** 2) / (2 * np.pi ** 2)


def power_amplitude(cosmo):
    """A such that A k^ns T^2 has the requested sigma8 at a = 1."""
    return cosmo.sigma8 ** 2 / sigma8_integral(lambda k: unnormalised_power(k, cosmo))


def linear_power(k, cosmo):
    """Linear matter power at a = 1, (Mpc/h)^3."""
    k = np.asarray(k, dtype=np.float64)
    kk = np.where(k > 0, k, 1.0)
    return np.where(k > 0, power_amplitude(cosmo) * unnormalised_power(kk, cosmo), 0.0)
