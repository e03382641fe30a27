"""Pins of the oracle's background cosmology against closed forms and
independent quadratures (growth ODE, BBKS/sigma8, KDK coefficients)."""

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import cosmology as C
from oracle.pm import Setup, integrate


A = np.array([1 / 64, 0.05, 0.2, 0.5, 0.9, 1.0])


def test_einstein_de_sitter_closed_form():
    # Omega_m = 1: D1 = a, D2 = -3/7 a^2 exactly.
    g = C.growth(A, 1.0)
    np.testing.assert_allclose(g["D1"], A, rtol=1e-10)
    np.testing.assert_allclose(g["dD1"], np.ones_like(A), rtol=1e-10)
    np.testing.assert_allclose(g["D2"], -3 / 7 * A ** 2, rtol=1e-9)
    np.testing.assert_allclose(g["dD2"], -6 / 7 * A, rtol=1e-9)


@pytest.mark.parametrize("om", [0.2, 0.3, 0.45])
def test_lcdm_growth_matches_heath_integral(om):
    # Linear growing mode of flat LCDM: D1 ∝ E(a) ∫_0^a da' / (a' E(a'))^3.
    def heath(a):
        val, _ = quad(lambda x: (x * C.hubble_e(x, om)) ** -3, 0.0, a, epsabs=0, epsrel=1e-13, limit=200)
        return C.hubble_e(a, om) * val

    ref = np.array([heath(a) for a in A]) / heath(1.0)
    np.testing.assert_allclose(C.growth(A, om)["D1"], ref, rtol=1e-8)


def test_force_growth_identity():
    # g_f = a^2 E d(g_p)/da must equal 3/2 Om D1 (the growth ODE itself).
    om = 0.3
    a = np.array([0.05, 0.3, 0.7])
    eps = 1e-5
    gp = lambda x: C.growth_tables(x, om)["gp"]
    dgp = (gp(a * (1 + eps)) - gp(a * (1 - eps))) / (2 * eps * a)
    lhs = a ** 2 * C.hubble_e(a, om) * dgp
    np.testing.assert_allclose(lhs, C.growth_tables(a, om)["gf"], rtol=1e-7)


def test_bbks_limits():
    assert abs(C.bbks_transfer(1e-12, 0.3, 0.7) - 1.0) < 1e-10
    t = C.bbks_transfer(np.logspace(-3, 1, 50), 0.3, 0.7)
    assert np.all(np.diff(t) < 0)


def test_bbks_series_and_asymptote():
    # The BBKS fit (Bardeen, Bond, Kaiser & Szalay 1986, ApJ 304, 15, App. G):
    # T(q) = ln(1 + 2.34 q)/(2.34 q) [1 + 3.89 q + (16.1 q)^2 + (5.46 q)^3 + (6.71 q)^4]^(-1/4),
    # q = k / (Om h).  Expanded by hand: near q = 0 the slope is -(2.34/2 + 3.89/4) and the q^2
    # coefficient 2.34^2/3 + (2.34/2)(3.89/4) - 16.1^2/4 + (5/32) 3.89^2; for q >> 1,
    # T -> ln(1 + 2.34 q)/(2.34 q) / (6.71 q) * (1 - 5.46^3 / (4 * 6.71^4 q)).  Each coefficient
    # enters one of these, so a wrong one, a wrong exponent or a wrong log argument fails.
    om, h = 0.3, 0.7
    q = np.linspace(1e-4, 2e-3, 60)
    co = np.polynomial.polynomial.polyfit(q, C.bbks_transfer(q * om * h, om, h), 7)
    assert abs(co[0] - 1.0) < 1e-12
    assert abs(co[1] - (-(2.34 / 2 + 3.89 / 4))) < 1e-8
    c2 = 2.34 ** 2 / 3 + (2.34 / 2) * (3.89 / 4) - 16.1 ** 2 / 4 + 5 / 32 * 3.89 ** 2
    assert abs(co[2] - c2) < 1e-6 * abs(c2)
    for qq in (1e5, 1e6):
        x = 2.34 * qq
        asym = np.log1p(x) / x / (6.71 * qq) * (1 - 5.46 ** 3 / (4 * 6.71 ** 4 * qq))
        assert abs(C.bbks_transfer(qq * om * h, om, h) / asym - 1) < 1e-10
    # k enters only through Gamma = Om h
    k = np.logspace(-3, 1, 9)
    np.testing.assert_allclose(C.bbks_transfer(k, 0.3, 0.7), C.bbks_transfer(k * 0.25 * 0.8 / 0.21, 0.25, 0.8),
                               rtol=1e-13)


@pytest.mark.parametrize("cosmo", [C.Cosmology(), C.Cosmology(0.25, 0.9, 0.7, 0.96)])
def test_sigma8_normalisation_independent_quadrature(cosmo):
    amp = C.power_amplitude(cosmo)

    def integrand(lnk):
        k = np.exp(lnk)
        return k ** 3 * amp * C.unnormalised_power(k, cosmo) * C.tophat_window(k * 8.0) ** 2 / (2 * np.pi ** 2)

    val = sum(quad(integrand, lo, hi, epsabs=0, epsrel=1e-12, limit=400)[0]
              for lo, hi in zip(np.log([1e-5, 1e-2, 1e-1, 1, 10]), np.log([1e-2, 1e-1, 1, 10, 1e3])))
    assert abs(np.sqrt(val) - cosmo.sigma8) < 1e-8


def test_tophat_series_matches_closed_form():
    x = np.array([5e-3, 9e-3, 1.1e-2, 0.09, 0.11, 0.5])
    direct = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    np.testing.assert_allclose(C.tophat_window(x), direct, rtol=1e-9)


def test_tophat_window_to_double_precision():
    # The closed form evaluated in 50-digit arithmetic, on both sides of the
    # switch to the small-x series (where the closed form cancels in FP64).
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    x = np.array([1e-4, 3e-3, 9.9e-3, 1.01e-2, 0.099, 0.101, 0.3, 2.0, 7.5])
    ref = np.array([float(3 * (mp.sin(mp.mpf(v)) - mp.mpf(v) * mp.cos(mp.mpf(v))) / mp.mpf(v) ** 3) for v in x])
    np.testing.assert_allclose(C.tophat_window(x), ref, rtol=2e-14)


@pytest.mark.parametrize("n_steps", [1, 7, 50])
@pytest.mark.parametrize("solver", [0, 4])
def test_kdk_exact_for_linear_force(n_steps, solver):
    # With the linear-theory force F = 3/2 Om s, growth-matched KDK reproduces
    # the growing mode s = D1(a) s1, p = g_p(a) s1 exactly for any step count,
    # with steps uniform in a or (solver flag 4) in ln a.
    cosmo = C.Cosmology(0.3)
    st = Setup(4, 8, 100.0, cosmo, a_init=1 / 64, a_final=1.0, n_steps=n_steps, solver=solver)
    s1 = np.random.default_rng(3).standard_normal((64, 3))
    gi = C.growth_tables(np.array([st.a_init, st.a_final]), cosmo.omega_m)
    s0, p0 = gi["D1"][0] * s1, gi["gp"][0] * s1
    s, p, _ = integrate(s0, p0, st, force_fn=lambda y: 1.5 * cosmo.omega_m * y)
    np.testing.assert_allclose(s, gi["D1"][1] * s1, rtol=1e-11, atol=1e-12)
    np.testing.assert_allclose(p, gi["gp"][1] * s1, rtol=1e-11, atol=1e-12)


def test_coefficient_domega_step_independent():
    cosmo = C.Cosmology(0.3)
    d1 = C.kdk_coefficients_domega(cosmo, 1 / 64, 1.0, 5)
    up = C.kdk_coefficients(cosmo.with_omega_m(0.3 + 1e-3), 1 / 64, 1.0, 5)
    dn = C.kdk_coefficients(cosmo.with_omega_m(0.3 - 1e-3), 1 / 64, 1.0, 5)
    for k in ("K_a", "Dr", "K_b"):
        np.testing.assert_allclose(d1[k], (up[k] - dn[k]) / 2e-3, rtol=1e-5)


def test_log_a_grid_is_geometric():
    a, ah = C.time_grid(1 / 64, 1.0, 6, log_a=True)
    assert a[0] == 1 / 64 and abs(a[-1] - 1.0) < 1e-15
    np.testing.assert_allclose(np.diff(np.log(a)), np.log(64) / 6, rtol=1e-12)
    np.testing.assert_allclose(np.log(ah), 0.5 * (np.log(a[:-1]) + np.log(a[1:])), rtol=1e-12)
