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
