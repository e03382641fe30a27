"""Failure path of the bounded device waits, with the failure made on the
host.  Two kernels wait on an mbarrier with an iteration limit and set a
device error flag when it runs out: the z-pass inverse (its TMA copy of the
spectrum) and the learned correction (its MMA completion).  Making a real
copy or MMA stall would need a faulting GPU, so pm_inject_wait_timeout sets
the flag as the kernel would, with no kernel made to wait.  Checks: the next
reporting call returns PM_ECUDA, the flag is cleared, the context keeps
working, and the hook rejects what it cannot do."""

import numpy as np
import pytest
import torch

from paper_2211_09958_gb300 import _pmgb, inputs

pytestmark = pytest.mark.gpu

SIZES = (32, 128, 128, 3)


def _pm(n_p, n_m, box=64.0, steps=2):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps)


def test_a_timed_out_spectrum_copy_is_reported_and_the_context_recovers():
    from paper_2211_09958_gb300.pm import PMError
    pm = _pm(16, 256)
    s, p = pm.init_lpt(seed=1)
    target = torch.from_numpy(inputs.target_field(256, 2)).cuda()[None]
    loss0, _ = pm.mse_loss(s, target)
    assert pm._lib.pm_inject_wait_timeout(pm._ctx, 0) == _pmgb.PM_OK
    with pytest.raises(PMError, match="timed out"):
        pm.mse_loss(s, target)
    loss1, _ = pm.mse_loss(s, target)                         # the flag was cleared
    assert abs(loss1[0] - loss0[0]) <= 1e-6 * loss0[0]
    s2, p2 = s.clone(), p.clone()
    pm.integrate(s2, p2)                                      # the context keeps working
    assert torch.isfinite(s2).all()
    pm.close()


def test_a_timed_out_correction_mma_is_reported_and_the_context_recovers():
    from paper_2211_09958_gb300.pm import PMError
    pm = _pm(16, 32)
    pm.nn_set_params(inputs.mlp_params(SIZES, seed=4))
    s = torch.from_numpy(inputs.random_displacements(16, 64.0, seed=5, scale=0.5)).cuda()[None]
    d0 = pm.nn_predict(s, 0.5)
    assert pm._lib.pm_inject_wait_timeout(pm._ctx, 1) == _pmgb.PM_OK
    with pytest.raises(PMError, match="timed out"):
        pm.nn_predict(s, 0.5)
    d1 = pm.nn_predict(s, 0.5)
    assert torch.equal(d0, d1) or (d0 - d1).abs().max().item() <= 1e-6 * d0.abs().max().item()
    pm.close()


def test_the_hook_rejects_what_it_cannot_do():
    pm = _pm(16, 32)
    assert pm._lib.pm_inject_wait_timeout(None, 0) == _pmgb.PM_EINVAL
    assert pm._lib.pm_inject_wait_timeout(pm._ctx, 2) == _pmgb.PM_EINVAL
    assert pm._lib.pm_inject_wait_timeout(pm._ctx, 1) == _pmgb.PM_ESTATE   # no network parameters yet
    pm.close()
    cu = _pm(12, 24, 48.0)                                                  # cuFFT mesh: no bounded copy
    assert cu._lib.pm_inject_wait_timeout(cu._ctx, 0) == _pmgb.PM_ESTATE
    s, p = cu.init_lpt(seed=3)
    cu.integrate(s, p)
    cu.close()
