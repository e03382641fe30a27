"""Degenerate cases of the method on the GPU path.

* The unperturbed lattice.  With the lattice half a mesh cell off the nodes
  and n_m = n_p or 2 n_p, every cell receives exactly one particle's worth of
  CIC weight.  The sums (eighths, or one eighth per particle times alpha) are
  exact in FP32 in any order, so delta = 0 exactly.  The force transforms
  the constant rho = 1.  The library's own FFT (power-of-two meshes) maps a
  constant exactly to its k = 0 mode: sums of equal values are exact,
  differences vanish, and every twiddle multiplies a zero.  The Green's
  function removes k = 0, so the force is exactly 0 there.  cuFFT (other
  meshes) may leave rounding-level residues: 1e-6 of the force of a
  perturbed lattice.
* A single KDK step, where the merged-kick loop reduces to one half kick,
  one drift and one half kick, against the FP64 oracle at the parity bounds.
"""

import numpy as np
import pytest
import torch

from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pm(n_p, n_m, box, steps=2):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps)


@pytest.mark.parametrize("n_p,n_m", [(16, 16), (16, 32), (32, 64), (12, 24)])
def test_unperturbed_lattice_has_no_density_and_no_force(n_p, n_m):
    pm = _pm(n_p, n_m, 2.0 * n_p)
    s = torch.zeros((1, n_p ** 3, 3), dtype=torch.float32, device="cuda")
    d = pm.density(s)
    assert torch.count_nonzero(d).item() == 0
    f = pm.pm_force(s)
    if n_m & (n_m - 1) == 0:                               # own FFT: exact
        assert torch.count_nonzero(f).item() == 0
    else:                                                  # cuFFT
        s1 = torch.from_numpy(inputs.random_displacements(n_p, 2.0 * n_p, seed=1, scale=0.3)).cuda()[None]
        scale = pm.pm_force(s1).abs().max().item()
        assert f.abs().max().item() <= 1e-6 * scale
    pm.close()


@pytest.mark.parametrize("n_p,n_m", [(16, 32), (18, 36)])
def test_single_step_matches_the_oracle(n_p, n_m):
    box = 4.0 * n_p
    pm = _pm(n_p, n_m, box, steps=1)
    noise = inputs.white_noise(n_p, 5)
    s, p = pm.init_lpt(torch.from_numpy(noise).cuda()[None])
    f = pm.integrate(s, p)
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8), n_steps=1)
    rs, rp, rf = opm.simulate(noise.astype(np.float64), st)
    ds = np.max(np.abs(s[0].cpu().numpy() - rs)) / (box / n_p)
    dp = np.max(np.abs(p[0].cpu().numpy() - rp)) / np.max(np.abs(rp))
    assert ds < 1e-4 and dp < 1e-4, (ds, dp)
    assert np.max(np.abs(f[0].cpu().numpy() - rf)) < 1e-3 * np.max(np.abs(rf))
    pm.close()
