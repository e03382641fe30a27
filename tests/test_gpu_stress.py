"""Paint and read kernels under clustering: half of the particles in 1 % of
the volume (about 50 times the mean density; the float atomics of the paints
then hit the same cells from many particles).

Tolerances follow the uniform-state parity tests, with the density bound
scaled by the local density.  A cell sums k FP32 weights, each at most
alpha = (n_m / n_p)^3; the rounding grows with the sum, 1 + delta, so the
bound is 1e-5 of max(alpha, 1 + delta) per cell.
"""

import numpy as np
import pytest
import torch

from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300 import inputs

GEOMS = [(16, 32, 64.0), (32, 64, 128.0)]


def test_clustered_state_has_half_the_particles_in_one_percent_of_the_volume():
    n_p, box, bins = 32, 128.0, 64
    h, w = box / n_p, box / bins
    s = inputs.clustered_displacements(n_p, box, seed=1).astype(np.float64).reshape(n_p, n_p, n_p, 3)
    # positions relative to lattice site (0, 0, 0): index differences times the spacing, plus s
    rel = np.stack(np.meshgrid(*(np.arange(n_p) * h,) * 3, indexing="ij"), axis=-1) + s
    ix = np.floor((rel.reshape(-1, 3) % box) / w).astype(np.int64) % bins
    hist = np.zeros((bins,) * 3)
    np.add.at(hist, (ix[:, 0], ix[:, 1], ix[:, 2]), 1.0)
    # densest periodic window of k^3 bins (k w just above the cube side 0.01^(1/3) L), summed-area table
    k = int(np.ceil(0.01 ** (1.0 / 3.0) * box / w)) + 1
    pad = np.pad(hist, ((0, k), (0, k), (0, k)), mode="wrap")
    c = np.pad(pad.cumsum(0).cumsum(1).cumsum(2), ((1, 0), (1, 0), (1, 0)))
    sums = (c[k:, k:, k:] - c[:-k, k:, k:] - c[k:, :-k, k:] - c[k:, k:, :-k]
            + c[:-k, :-k, k:] + c[:-k, k:, :-k] + c[k:, :-k, :-k] - c[:-k, :-k, :-k])
    assert (k * w / box) ** 3 < 0.013
    assert sums.max() >= 0.45 * n_p ** 3, sums.max() / n_p ** 3


def _pm(n_p, n_m, box, steps=4, a_init=1.0 / 64):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps, a_init)


def _setup(pm, a_init=1.0 / 64):
    return opm.Setup(pm.n_p, pm.n_m, pm.box, Cosmology(0.3, 0.8), a_init=a_init, n_steps=pm.n_steps)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.gpu
@pytest.mark.parametrize("n_p,n_m,box", GEOMS)
def test_clustered_density_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    s = inputs.clustered_displacements(n_p, box, seed=n_p)
    d = _host(pm.density(_cuda(s)[None]))[0]
    ref = opm.density(s.astype(np.float64), _setup(pm))
    alpha = (n_m / n_p) ** 3
    assert ref.max() > 20.0                                   # the cluster is there
    err = np.abs(d - ref) / np.maximum(alpha, 1.0 + ref)
    assert err.max() < 1e-5, err.max()
    pm.close()


@pytest.mark.gpu
@pytest.mark.parametrize("n_p,n_m,box", GEOMS)
def test_clustered_force_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    s = inputs.clustered_displacements(n_p, box, seed=n_p + 1)
    f = _host(pm.pm_force(_cuda(s)[None]))[0]
    ref = opm.force(s.astype(np.float64), _setup(pm))
    err = np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    assert err < 2e-5, err
    pm.close()


@pytest.mark.gpu
def test_clustered_adjoint_parity():
    # the last two KDK steps (a = 0.9 -> 1, where clusters exist) from the
    # clustered state and their adjoint: the 4-field adjoint paint and the
    # adjoint read under clustering.  (From a = 1/64 the 50x overdensity would
    # throw particles thousands of Mpc/h, where FP32 spacing alone exceeds the
    # 1e-4 bound.)
    n_p, n_m, box, steps, a_init = 16, 32, 64.0, 2, 0.9
    pm = _pm(n_p, n_m, box, steps, a_init)
    st = _setup(pm, a_init)
    rng = np.random.default_rng(8)
    s0 = inputs.clustered_displacements(n_p, box, seed=9)
    p0 = (rng.standard_normal((n_p ** 3, 3)) * 0.01).astype(np.float32)
    lam0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    mu0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    s, p = _cuda(s0)[None], _cuda(p0)[None]
    f = pm.integrate(s, p)
    rs, rp, rf = opm.integrate(s0.astype(np.float64), p0.astype(np.float64), st)
    spacing = box / n_p
    assert np.max(np.abs(_host(s)[0] - rs)) < 1e-4 * spacing
    lam, mu = _cuda(lam0)[None], _cuda(mu0)[None]
    pm.adjoint_integrate(s, p, f, lam, mu)
    _, _, olam, omu, _ = opm.adjoint_integrate(rs, rp, rf, lam0.astype(np.float64), mu0.astype(np.float64), st)
    for got, ref in ((_host(lam)[0], olam), (_host(mu)[0], omu)):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < 1e-3, rel
    pm.close()
