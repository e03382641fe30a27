"""Counter-based white noise for the oracle (test infrastructure only).

The paper constrains the initial conditions of the Universe (Statement of
Need) but does not say how its white noise is drawn.  Reading: unit Gaussian
white noise on the particle lattice from Philox4x32-10 (Salmon, Moraes, Dror
& Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3"), one counter per
lattice site, followed by the Box-Muller transform.           [reading]

  counter = (site & 0xffffffff, site >> 32, 0, 0), key = (seed lo, seed hi)
  u1 = (x0 + 1/2) / 2^32,  u2 = (x1 + 1/2) / 2^32
  z  = sqrt(-2 ln u1) cos(2 pi u2)

The round function and constants are the published ones; this file is written
from that definition.  Pinned bit for bit against the generator's published
known-answer vectors; the Gaussian field it yields is pinned statistically.
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds; counters are uint64 arrays holding 32-bit
    values, the key two Python ints.  Returns four uint64 arrays."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 &= 0xFFFFFFFF
    k1 &= 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1,
                          hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def white_noise(n_side, seed):
    """(n_side, n_side, n_side) unit Gaussian field in lattice order."""
    site = np.arange(n_side ** 3, dtype=np.uint64)
    x0, x1, _, _ = philox4x32_10(site & _MASK, site >> np.uint64(32),
                                 np.zeros_like(site), np.zeros_like(site),
                                 int(seed) & 0xFFFFFFFF, (int(seed) >> 32) & 0xFFFFFFFF)
    u1 = (x0.astype(np.float64) + 0.5) * 2.0 ** -32
    u2 = (x1.astype(np.float64) + 0.5) * 2.0 ** -32
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return z.reshape(n_side, n_side, n_side)
