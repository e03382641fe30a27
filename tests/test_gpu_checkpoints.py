"""Sparse checkpoints against FP32 reversal drift (a solver variant).

The adjoint reconstructs the forward trajectory by reverse time integration
(paper, Summary: adjoint method with reverse time integration).  In FP32 every
reverse step adds rounding, so the reconstructed states drift from the forward
ones.  With checkpoints every k steps the library stores s_m and p_{m+1/2}
during the forward run and restores them when the adjoint enters step m.

Checks (the density paint adds with float atomics in arbitrary order, so two
forward runs agree to rounding, not bit for bit: 1e-5 of the spacing):
  * the forward run is the same with and without checkpoints (they only copy);
  * a stored s_m is the state after integrating steps [0, m);
  * with every = 1 the state reconstructed at a_init is within 1e-6 of the
    spacing of the forward one (a single reverse drift of rounding), far below
    the drift of the unchecked reversal;
  * gradients with checkpoints match the FP64 oracle at the parity bounds;
  * dL/dOm of the dynamics with steps uniform in ln a: a small sum of large
    cancelling per-step terms, some weighted by the early, small momenta
    whose FP32 reconstruction drifts most (up to ~1e-3 of the sum of the
    terms' magnitudes without checkpoints); with a checkpoint at every step
    it meets the oracle at 1e-4 of that sum, the bound of the parity tests;
  * bad arguments are rejected and leave the context usable.
"""

import ctypes

import numpy as np
import pytest
import torch

from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300 import _pmgb, inputs

pytestmark = pytest.mark.gpu


def _pm(n_p, n_m, box, steps):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps)


def _ic(pm, seed):
    noise = torch.from_numpy(inputs.white_noise(pm.n_p, seed)).cuda()[None]
    return noise, *pm.init_lpt(noise)


def test_checkpoints_leave_the_forward_run_unchanged():
    pm = _pm(32, 64, 128.0, 12)
    _, s0, p0 = _ic(pm, 3)
    s1, p1 = s0.clone(), p0.clone()
    f1 = pm.integrate(s1, p1)
    buf = pm.set_checkpoints(4)
    assert buf is not None and buf.numel() == pm._lib.pm_checkpoint_floats(pm._ctx, 4) == 2 * 2 * 32 ** 3 * 3
    s2, p2 = s0.clone(), p0.clone()
    f2 = pm.integrate(s2, p2)
    tol = 1e-5 * pm.box / pm.n_p
    assert torch.max(torch.abs(s1 - s2)).item() <= tol
    assert torch.max(torch.abs(p1 - p2)).item() <= 1e-5 * torch.max(torch.abs(p1)).item()
    assert torch.max(torch.abs(f1 - f2)).item() <= 1e-5 * torch.max(torch.abs(f1)).item()
    pm.close()


def test_stored_states_are_the_forward_states():
    steps, every = 9, 3
    pm = _pm(16, 32, 64.0, steps)
    _, s0, p0 = _ic(pm, 4)
    buf = pm.set_checkpoints(every)
    s, p = s0.clone(), p0.clone()
    pm.integrate(s, p)
    ck = buf.view(-1, 2, 1, pm.n_part, 3).clone()
    assert ck.shape[0] == (steps - 1) // every == 2
    pm.set_checkpoints(0)
    for slot, m in enumerate(range(every, steps, every)):
        sm, pm_ = s0.clone(), p0.clone()
        pm.integrate(sm, pm_, 0, m)
        assert torch.max(torch.abs(ck[slot, 0] - sm)).item() <= 1e-5 * pm.box / pm.n_p, m
    pm.close()


def _reversal_error(pm, s0, p0):
    s, p = s0.clone(), p0.clone()
    f = pm.integrate(s, p)
    lam, mu = torch.zeros_like(s), torch.zeros_like(p)
    pm.adjoint_integrate(s, p, f, lam, mu, mu_zero=True)
    return torch.max(torch.abs(s - s0)).item(), torch.max(torch.abs(p - p0)).item()


def test_checkpoints_bound_the_reversal_drift():
    pm = _pm(32, 64, 128.0, 24)
    _, s0, p0 = _ic(pm, 5)
    ds_plain, dp_plain = _reversal_error(pm, s0, p0)
    pm.set_checkpoints(1)
    ds_ck, dp_ck = _reversal_error(pm, s0, p0)
    spacing = pm.box / pm.n_p
    assert ds_ck <= 1e-6 * spacing, (ds_ck, ds_plain)
    assert ds_ck < 0.1 * ds_plain, (ds_ck, ds_plain)
    assert dp_ck <= 1e-5 * torch.max(torch.abs(p0)).item(), (dp_ck, dp_plain)
    assert dp_ck < dp_plain, (dp_ck, dp_plain)
    pm.close()


@pytest.mark.parametrize("every", [1, 2])
def test_checkpointed_gradients_match_the_oracle(every):
    from paper_2211_09958_gb300.pm import density, simulate
    n_p, n_m, box, steps = 16, 32, 64.0, 4
    pm = _pm(n_p, n_m, box, steps)
    pm.set_checkpoints(every)
    noise = inputs.white_noise(n_p, 0)
    target = inputs.target_field(n_m, 1)
    nz = torch.from_numpy(noise).cuda()[None].requires_grad_(True)
    om = torch.tensor([0.3], dtype=torch.float64, requires_grad=True)
    s8 = torch.tensor([0.8], dtype=torch.float64, requires_grad=True)
    s, _ = simulate(pm, nz, om, s8)
    loss = torch.mean((density(pm, s) - torch.from_numpy(target).cuda()[None]) ** 2)
    loss.backward()
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8), n_steps=steps)
    o_loss, o_gn, _, o_s8 = opm.loss_and_grad(noise.astype(np.float64), target.astype(np.float64), st)
    assert abs(loss.item() - o_loss) < 1e-4 * o_loss
    g = nz.grad[0].cpu().numpy().astype(np.float64).ravel()
    rel = np.linalg.norm(g - o_gn.ravel()) / np.linalg.norm(o_gn)
    cos = np.dot(g, o_gn.ravel()) / np.linalg.norm(g) / np.linalg.norm(o_gn)
    assert rel < 1e-3 and cos > 0.9999, (rel, cos)
    assert abs(s8.grad.item() - o_s8) < 1e-3 * abs(o_s8), (s8.grad, o_s8)
    pm.close()


def test_bad_checkpoint_arguments_are_rejected():
    from paper_2211_09958_gb300.pm import PMError
    pm = _pm(16, 32, 64.0, 6)
    with pytest.raises(PMError):
        pm.set_checkpoints(-1)
    assert pm._lib.pm_set_checkpoints(pm._ctx, 2, None) == _pmgb.PM_EINVAL
    assert pm._lib.pm_set_checkpoints(pm._ctx, 6, None) == _pmgb.PM_OK     # no slot: off, no buffer needed
    assert pm._lib.pm_checkpoint_floats(pm._ctx, 6) == 0
    assert pm._lib.pm_checkpoint_floats(None, 2) == -1
    bad = torch.empty(pm._lib.pm_checkpoint_floats(pm._ctx, 2) + 1, dtype=torch.float32, device="cuda")
    assert pm._lib.pm_set_checkpoints(pm._ctx, 2, ctypes.c_void_p(bad.data_ptr() + 2)) == _pmgb.PM_EINVAL
    _, s0, p0 = _ic(pm, 6)
    pm.integrate(s0, p0)                                                  # still usable
    pm.close()


@pytest.mark.parametrize("n_p,n_m,solver", [(16, 16, 4), (16, 32, 6)])
def test_checkpoints_remove_the_drift_from_the_omega_gradient(n_p, n_m, solver):
    from oracle.cosmology import kdk_coefficients_domega
    from paper_2211_09958_gb300.pm import ParticleMesh
    box, steps = 4.0 * n_p, 4
    pm = ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps, solver=solver)
    pm.set_checkpoints(1)
    noise = inputs.white_noise(n_p, 9)
    rng = np.random.default_rng(3)
    lam0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    mu0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    s, p = pm.init_lpt(torch.from_numpy(noise).cuda()[None])
    f = pm.integrate(s, p)
    lam, mu = torch.from_numpy(lam0).cuda()[None], torch.from_numpy(mu0).cuda()[None]
    dom = pm.adjoint_integrate(s, p, f, lam, mu)[0]
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8), n_steps=steps, solver=solver)
    rs, rp, rf = opm.simulate(noise.astype(np.float64), st)
    _, _, _, _, grads = opm.adjoint_integrate(rs, rp, rf, lam0.astype(np.float64), mu0.astype(np.float64), st)
    o_dom = opm.dynamics_domega(grads, st)
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps, bool(solver & 4))
    cond = abs(grads["omega_m_direct"]) + sum(abs(np.dot(grads[k], d[k])) for k in ("K_a", "Dr", "K_b"))
    assert abs(dom - o_dom) <= 1e-4 * cond, (dom, o_dom, cond)
    pm.close()
