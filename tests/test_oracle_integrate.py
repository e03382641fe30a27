"""Pins of the oracle's KDK integration, reverse time integration and
discrete adjoint (finite differences of the FP64 forward, reversibility,
plane-wave growth)."""

import numpy as np
import pytest

from oracle import lpt, pm
from oracle.cosmology import Cosmology, growth
from oracle.pm import Setup


def _ics(st, seed):
    noise = np.random.default_rng(seed).standard_normal((st.n_p,) * 3)
    return noise, lpt.initial_conditions(noise, st)


def test_forward_then_reverse_returns_initial_state():
    st = Setup(16, 32, 128.0, n_steps=10)
    _, (s0, p0) = _ics(st, 0)
    s, p, f = pm.integrate(s0, p0, st)
    assert np.max(np.abs(s - s0)) > 0.1 * st.spacing        # it moved
    sr, pr, _ = pm.reverse_integrate(s, p, f, st)
    assert np.max(np.abs(sr - s0)) < 1e-10 * st.spacing
    assert np.max(np.abs(pr - p0)) < 1e-10 * np.sqrt(np.mean(p0 ** 2))


def test_adjoint_matches_finite_differences_of_state():
    rng = np.random.default_rng(1)
    st = Setup(4, 8, 32.0, n_steps=2)
    _, (s0, p0) = _ics(st, 1)
    lam, mu = rng.standard_normal(s0.shape), rng.standard_normal(p0.shape)
    s, p, f = pm.integrate(s0, p0, st)
    sr, pr, lam0, mu0, _ = pm.adjoint_integrate(s, p, f, lam, mu, st)
    np.testing.assert_allclose(sr, s0, atol=1e-12)

    def obj(a, b):
        y, z, _ = pm.integrate(a, b, st)
        return np.sum(lam * y) + np.sum(mu * z)

    eps = 1e-6
    for i in range(s0.shape[0]):            # full Jacobian-transpose rows
        for d in range(3):
            e = np.zeros_like(s0)
            e[i, d] = eps
            fd_s = (obj(s0 + e, p0) - obj(s0 - e, p0)) / (2 * eps)
            fd_p = (obj(s0, p0 + e) - obj(s0, p0 - e)) / (2 * eps)
            assert abs(fd_s - lam0[i, d]) < 1e-6 * max(1, abs(fd_s))
            assert abs(fd_p - mu0[i, d]) < 1e-6 * max(1, abs(fd_p))


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    st = Setup(8, 16, 64.0, Cosmology(0.3, 0.8), n_steps=3)
    noise = rng.standard_normal((8, 8, 8))
    target = rng.standard_normal((16, 16, 16))
    loss, g_noise, g_om, g_s8 = pm.loss_and_grad(noise, target, st)

    def loss_of(nz, cosmo):
        stc = Setup(8, 16, 64.0, cosmo, n_steps=3)
        s, _, _ = pm.simulate(nz, stc)
        return pm.mse_loss(s, target, stc)

    c = st.cosmo
    eps = 1e-6
    for _ in range(8):
        v = rng.standard_normal(noise.shape)
        fd = (loss_of(noise + eps * v, c) - loss_of(noise - eps * v, c)) / (2 * eps)
        assert abs(fd - np.sum(g_noise * v)) < 1e-6 * max(abs(fd), 1e-3)
    eps = 1e-6
    fd_om = (loss_of(noise, Cosmology(c.omega_m + eps, c.sigma8)) - loss_of(noise, Cosmology(c.omega_m - eps, c.sigma8))) / (2 * eps)
    fd_s8 = (loss_of(noise, Cosmology(c.omega_m, c.sigma8 + eps)) - loss_of(noise, Cosmology(c.omega_m, c.sigma8 - eps))) / (2 * eps)
    assert abs(fd_om - g_om) < 1e-5 * abs(fd_om)
    assert abs(fd_s8 - g_s8) < 1e-6 * abs(fd_s8)


@pytest.mark.parametrize("n_p", [32])
def test_plane_wave_grows_as_d1(n_p):
    # One fundamental longitudinal mode, amplitude 1 % of the wavelength,
    # well before shell crossing: its amplitude must follow D1(a) for any
    # step count (growth-matched KDK); the PM force differs from the linear
    # 3/2 Om s only by the CIC/mesh window, a small (k h)^2 effect.
    box = 128.0
    cosmo = Cosmology(0.3)
    ratios = {}
    for n_m in (n_p, 2 * n_p):
        for steps in (10, 100):
            st = Setup(n_p, n_m, box, cosmo, n_steps=steps)
            q = pm.lattice(n_p, box, n_m)
            k = 2 * np.pi / box
            d = growth(np.array([st.a_init, 1.0]), cosmo.omega_m)
            gp = lambda a, dd: a ** 3 * np.sqrt(cosmo.omega_m / a ** 3 + 1 - cosmo.omega_m) * dd
            amp1 = 0.01 * box                 # s1 amplitude at a = 1
            s1 = np.zeros_like(q)
            s1[:, 0] = amp1 * np.sin(k * q[:, 0])
            s0 = d["D1"][0] * s1
            p0 = gp(st.a_init, d["dD1"][0]) * s1
            s, _, _ = pm.integrate(s0, p0, st)
            proj = np.sum(s[:, 0] * np.sin(k * q[:, 0])) / np.sum(np.sin(k * q[:, 0]) ** 2)
            ratios[(n_m, steps)] = proj / amp1
    # Only the CIC window and the difference gradient enter, both small at
    # k = k_Nyquist(particles) / 16; growth-matched KDK makes the step count
    # irrelevant for a linear mode.
    tol = {n_p: 1.5e-2, 2 * n_p: 5e-3}
    steps_tol = {n_p: 2e-3, 2 * n_p: 2e-3}
    for (n_m, steps), r in ratios.items():
        assert abs(r - 1.0) < tol[n_m], (n_m, steps, r)
    for n_m in (n_p, 2 * n_p):
        assert abs(ratios[(n_m, 10)] - ratios[(n_m, 100)]) < steps_tol[n_m], ratios
