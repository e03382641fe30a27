"""Seeded synthetic inputs shared by the tests, the benchmark and the
reference (oracle) checks.

Holds none of the method's arithmetic: only numpy's seeded generator for unit
white noise on the particle lattice and for the target density field of the
MSE loss, and the cosmology draws of the batched workload.  Values are
rounded to float32 so that the CUDA path and the FP64 oracle see identical
inputs.
"""

import numpy as np


def white_noise(n_p, seed):
    """(n_p, n_p, n_p) unit Gaussian white noise, float32, lattice order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n_p, n_p, n_p)).astype(np.float32)


def target_field(n_m, seed):
    """(n_m, n_m, n_m) unit Gaussian target density for the MSE loss."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.standard_normal((n_m, n_m, n_m)).astype(np.float32)


def batch_cosmologies(n_batch, seed=99):
    """Omega_m ~ U[0.2, 0.4] and sigma8 ~ U[0.6, 1.0] for a batch of runs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    om = rng.uniform(0.2, 0.4, n_batch)
    s8 = rng.uniform(0.6, 1.0, n_batch)
    return om, s8


def random_displacements(n_p, box, seed, scale=0.3):
    """Smooth-free random displacements (units of the lattice spacing times
    ``scale``), float32, shape (n_p^3, 3): a stand-in state for unit tests of
    single operations."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return (rng.standard_normal((n_p ** 3, 3)) * scale * box / n_p).astype(np.float32)


def clustered_displacements(n_p, box, seed, frac=0.5, volume=0.01, jitter=0.1):
    """Stress state for the paint and read kernels: the lattice cube that
    holds ``frac`` of the particles (side round(n_p frac^(1/3)) sites, corner
    drawn from the seed, periodic) is pulled towards its centre until it
    spans ``volume`` of the box; every particle also gets N(0, jitter^2)
    spacings of noise.  With the defaults half of the particles sit in 1 % of
    the volume, about 50 times the mean density.  Built from lattice index
    differences only (no lattice offset enters), float32, shape (n_p^3, 3)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    h = box / n_p
    side = max(1, int(round(n_p * frac ** (1.0 / 3.0))))
    kappa = volume ** (1.0 / 3.0) * n_p / side       # compressed side / lattice side
    corner = rng.integers(0, n_p, 3)
    s = rng.standard_normal((n_p ** 3, 3), dtype=np.float32) * np.float32(jitter * h)
    idx = np.arange(n_p)
    off = [(idx - corner[d]) % n_p for d in range(3)]
    cube = (off[0] < side)[:, None, None] & (off[1] < side)[None, :, None] & (off[2] < side)[None, None, :]
    for d, shape in enumerate(((n_p, 1, 1), (1, n_p, 1), (1, 1, n_p))):
        shift = ((kappa - 1.0) * (off[d] - (side - 1) / 2.0) * h).astype(np.float32).reshape(shape)
        s[:, d] += np.where(cube, shift, np.float32(0.0)).ravel()
    return s


def mlp_params(sizes, seed, bias_scale=0.1):
    """Flat float32 parameters of a dense network with layer widths
    ``sizes``: per layer a weight matrix [fan_in][fan_out] drawn N(0, 2 /
    fan_in), then a bias vector drawn N(0, bias_scale^2)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for fi, fo in zip(sizes[:-1], sizes[1:]):
        out.append(rng.standard_normal(fi * fo) * np.sqrt(2.0 / fi))
        out.append(rng.standard_normal(fo) * bias_scale)
    return np.concatenate(out).astype(np.float32)
