"""Pins of the oracle's counter-based white noise: the Philox4x32-10 round
function bit for bit against the generator's published known-answer vectors
(tests/golden/philox4x32_10_kat.txt), and the Gaussian field it yields
statistically."""

import os

import numpy as np
from scipy import stats

from oracle import philox

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def test_philox_matches_the_published_known_answers():
    rows = [line.split() for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    assert len(rows) == 3
    for row in rows:
        ctr = [np.array([int(x, 16)], dtype=np.uint64) for x in row[:4]]
        k0, k1 = int(row[4], 16), int(row[5], 16)
        out = philox.philox4x32_10(*ctr, k0, k1)
        assert [int(o[0]) for o in out] == [int(x, 16) for x in row[6:10]], row


def test_white_noise_is_unit_gaussian():
    z = philox.white_noise(48, 2022).ravel()
    n = z.size
    assert abs(z.mean()) < 5 / np.sqrt(n)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / n)
    assert stats.kstest(z, "norm").pvalue > 1e-4
    # no lattice correlation between neighbouring sites
    f = z.reshape(48, 48, 48)
    for ax in range(3):
        assert abs(np.mean(f * np.roll(f, 1, axis=ax))) < 5 / np.sqrt(n)


def test_white_noise_depends_on_seed_and_site_only():
    a = philox.white_noise(8, 7)
    b = philox.white_noise(8, 7)
    c = philox.white_noise(8, 8)
    np.testing.assert_array_equal(a, b)
    assert np.corrcoef(a.ravel(), c.ravel())[0, 1] < 0.2
    # site index is the counter: a 4^3 field is not a sub-block of the 8^3 one
    # but its first 64 sites equal the first 64 sites of the larger stream.
    np.testing.assert_array_equal(philox.white_noise(4, 7).ravel(), a.ravel()[:64])


def test_round_function_is_a_bijection_on_samples():
    ctr = np.arange(1 << 16, dtype=np.uint64)
    z = np.zeros_like(ctr)
    out = philox.philox4x32_10(ctr, z, z, z, 123, 456)
    packed = (out[0] << np.uint64(32)) | out[1]
    assert np.unique(packed).size == ctr.size
