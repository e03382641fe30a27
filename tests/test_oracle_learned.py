"""Pins of the oracle's learned force correction: bfloat16 rounding against
its definition, feature layout against explicit periodic neighbours, and the
backpropagated gradient against central finite differences of the FP64
loss."""

import numpy as np

from oracle import learned as L
from oracle import pm
from oracle.pm import Setup


def test_bf16_round_to_nearest_even():
    one = 1.0
    ulp = 2.0 ** -7                      # bfloat16 spacing at 1
    vals = np.array([one, one + ulp / 2, one + 1.5 * ulp, one + 0.49 * ulp, -3.0, 0.0])
    want = np.array([one, one, one + 2 * ulp, one, -3.0, 0.0])
    np.testing.assert_array_equal(L.bf16(vals), want)


def test_features_are_periodic_neighbours():
    rng = np.random.default_rng(0)
    n = 6
    rho = rng.uniform(0.2, 3.0, (n, n, n))
    f = L.features(rho, 0.37)
    c = (1, 5, 0)
    row = f[(c[0] * n + c[1]) * n + c[2]]
    for q, o in enumerate(L.OFFSETS):
        nb = tuple((c[d] + o[d]) % n for d in range(3))
        assert abs(row[q] - np.arcsinh(rho[nb] - 1.0)) < 1e-15
    assert row[27] == 0.37 and np.all(row[28:] == 0)


def test_loss_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    st = Setup(4, 8, 16.0)
    s = rng.normal(0, 0.8, (64, 3))
    target = rng.normal(0, 0.05, (64, 3))
    theta = L.init_params(2)
    theta[-(L.N_HID * 3 + 3):] = rng.normal(0, 0.1, L.N_HID * 3 + 3)    # nonzero last layer
    _, g = L.loss_and_grad(s, target, 0.5, theta, st, rounding=False)
    eps = 1e-7            # small enough that no ReLU input changes sign
    for _ in range(6):
        v = rng.standard_normal(theta.size)
        fd = (L.loss(s, target, 0.5, theta + eps * v, st, rounding=False)
              - L.loss(s, target, 0.5, theta - eps * v, st, rounding=False)) / (2 * eps)
        assert abs(fd - g @ v) < 1e-5 * max(1.0, abs(fd)), (fd, g @ v)   # rare ReLU crossings within eps


def test_untrained_network_is_zero_correction():
    st = Setup(4, 8, 16.0)
    s = np.random.default_rng(3).normal(0, 0.5, (64, 3))
    assert np.all(L.predict(s, 0.5, L.init_params(4), st) == 0.0)


def test_correction_vjp_matches_finite_differences():
    rng = np.random.default_rng(21)
    st = Setup(4, 8, 16.0, pm.Cosmology(0.3), n_steps=2)
    theta = rng.standard_normal(L.n_params()) * 0.2
    s = rng.normal(0, 0.8, (64, 3))
    v = rng.standard_normal((64, 3))
    g_s, g_t = L.correction_vjp(s, v, 0.6, theta, st, rounding=False)
    obj = lambda ss, th: np.sum(v * L.predict(ss, 0.6, th, st, rounding=False))
    eps = 1e-7
    for _ in range(4):
        d = rng.standard_normal(s.shape)
        fd = (obj(s + eps * d, theta) - obj(s - eps * d, theta)) / (2 * eps)
        assert abs(fd - np.sum(g_s * d)) < 1e-5 * max(1.0, abs(fd))
        dt = rng.standard_normal(theta.shape)
        fd = (obj(s, theta + eps * dt) - obj(s, theta - eps * dt)) / (2 * eps)
        assert abs(fd - g_t @ dt) < 1e-5 * max(1.0, abs(fd))


def test_corrected_adjoint_matches_finite_differences():
    rng = np.random.default_rng(22)
    st = Setup(4, 8, 16.0, pm.Cosmology(0.3), n_steps=2)
    theta = rng.standard_normal(L.n_params()) * 0.05     # a gentle network: FD along theta stays on one ReLU piece
    s0 = rng.normal(0, 0.5, (64, 3))
    p0 = rng.normal(0, 0.05, (64, 3))
    lam, mu = rng.standard_normal((64, 3)), rng.standard_normal((64, 3))
    s, p, f = L.integrate_corrected(s0, p0, theta, st, rounding=False)
    sr, pr, lam0, mu0, g_t = L.adjoint_corrected(s, p, f, lam, mu, theta, st, rounding=False)
    np.testing.assert_allclose(sr, s0, atol=1e-10)

    def obj(a, b, th):
        y, z, _ = L.integrate_corrected(a, b, th, st, rounding=False)
        return np.sum(lam * y) + np.sum(mu * z)

    # two steps through ReLU and CIC kinks: the central difference needs a
    # small step to stay on one smooth piece (at 1e-7 it is still 7e-4 off,
    # at 1e-8 it agrees to 3e-8)
    eps = 1e-8
    for _ in range(3):
        d = rng.standard_normal(s0.shape)
        fd = (obj(s0 + eps * d, p0, theta) - obj(s0 - eps * d, p0, theta)) / (2 * eps)
        assert abs(fd - np.sum(lam0 * d)) < 1e-5 * max(1.0, abs(fd))
        fd = (obj(s0, p0 + eps * d, theta) - obj(s0, p0 - eps * d, theta)) / (2 * eps)
        assert abs(fd - np.sum(mu0 * d)) < 1e-5 * max(1.0, abs(fd))
        dt = rng.standard_normal(theta.shape)
        fd = (obj(s0, p0, theta + eps * dt) - obj(s0, p0, theta - eps * dt)) / (2 * eps)
        assert abs(fd - g_t @ dt) < 1e-5 * max(1.0, abs(fd))
