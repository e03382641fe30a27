"""Binned, tile-owned CIC deposit (tuning family "deposit" = 2, for
own-transform meshes whose side is a multiple of 16; the default is the
atomic scatter, deposit = 1) against the FP64 oracle's density and against
the atomic scatter.

  * density (pm_density, delta = alpha sum W - 1) of seeded states that
    cross tile faces and the periodic box edges (random displacements of up
    to several spacings) and of a clustered state (half of the particles in
    1 % of the volume: most bins empty, a few holding thousands), on meshes
    of 1, 4 and 8 tiles per side, for a batch of 3 runs with different
    states: element by element within 1e-5 of max(alpha, 1 + delta), the
    density bound of the small-size tests, and mass conserved;
  * a mesh that is not a multiple of the tile (n_m = 8) runs the atomic
    scatter under deposit = 2 and matches the oracle the same way;
  * the force with the binned paint equals that of the atomic scatter
    within 2e-5 of max |F| (one evaluation: FP32 summation order only); a
    4-step trajectory and the reverse-time adjoint's cotangents and dL/dOm,
    whose 4-field paint (alpha, mu) is the binned kernel's other
    instantiation, within the oracle parity bounds (state 1e-4 of the
    spacing, lam and mu 1e-3 relative L2, dL/dOm 5e-3 relative).  Two runs
    of the atomic scatter with different block sizes differ by 1e-6 to 1e-5
    of the spacing and 1e-4 to 1e-3 in dL/dOm here (FP32 sums amplified by
    the giant steps), and so do the binned and the atomic paints.
"""

import numpy as np
import pytest
import torch

from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _pm(n_p, n_m, box, B=1, steps=4):
    from paper_2211_09958_gb300.pm import ParticleMesh
    om, s8 = ([0.3] * B, [0.8] * B) if B > 1 else (0.3, 0.8)
    return ParticleMesh(n_p, n_m, box, om, s8, steps)


def _states(n_p, box):
    return [inputs.random_displacements(n_p, box, seed=21, scale=3.0),
            inputs.clustered_displacements(n_p, box, seed=22),
            inputs.random_displacements(n_p, box, seed=23, scale=0.5)]


@pytest.mark.parametrize("n_p,n_m,box", [(8, 16, 32.0), (32, 64, 96.0), (64, 128, 128.0), (8, 8, 40.0)])
def test_binned_density_against_oracle(n_p, n_m, box):
    pm = _pm(n_p, n_m, box, B=3)
    assert pm.get_tuning()["deposit"] == 1                           # the atomic scatter by default
    pm.set_tuning(deposit=2)
    states = _states(n_p, box)
    d = _host(pm.density(_cuda(np.stack(states))))
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8))
    for b, s in enumerate(states):
        ref = opm.density(s.astype(np.float64), st)
        err = np.abs(d[b].ravel() - ref.ravel()) / np.maximum(st.alpha, 1.0 + ref.ravel())
        print(f"n_m {n_m}, run {b}: max err {err.max():.2e} of max(alpha, 1 + delta)")
        assert err.max() < 1e-5, (b, err.max())
        assert abs(d[b].sum()) < 1e-6 * d[b].size * st.alpha
    pm.close()


def test_binned_and_atomic_paints_agree_in_force_trajectory_and_adjoint():
    n_p, n_m, box = 32, 64, 256.0
    pm = _pm(n_p, n_m, box)
    s0 = _cuda(inputs.clustered_displacements(n_p, box, seed=4))[None]
    rng = np.random.default_rng(8)
    lam0 = rng.standard_normal((1, n_p ** 3, 3)).astype(np.float32)
    out = {}
    for dep in (1, 2):
        pm.set_tuning(deposit=dep)
        f = pm.pm_force(s0)
        s, p = pm.init_lpt(seed=6)
        fs = pm.integrate(s, p)
        lam, mu = _cuda(lam0), torch.zeros_like(p)
        dom = pm.adjoint_integrate(s, p, fs, lam, mu)
        out[dep] = (_host(f), _host(s), _host(lam), _host(mu), float(dom[0]))
    f1, s1, l1, m1, d1 = out[1]
    f2, s2, l2, m2, d2 = out[2]
    print(f"binned vs atomic: force {np.abs(f2 - f1).max() / np.abs(f1).max():.2e} of max |F|, "
          f"state {np.abs(s2 - s1).max() / (box / n_p):.2e} of the spacing, "
          f"lam {np.linalg.norm(l2 - l1) / np.linalg.norm(l1):.2e}, mu {np.linalg.norm(m2 - m1) / np.linalg.norm(m1):.2e}, "
          f"dOm {abs(d2 - d1) / abs(d1):.2e}")
    assert np.abs(f2 - f1).max() <= 2e-5 * np.abs(f1).max()
    assert np.abs(s2 - s1).max() <= 1e-4 * box / n_p
    for a, b in ((l2, l1), (m2, m1)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 1e-3
    assert abs(d2 - d1) <= 5e-3 * abs(d1)
    pm.close()
