"""Parity at the full size of the benchmark workload, 512^3 particles on a
1024^3 mesh (1 Gpc/h, 100 KDK steps), in the launch configuration the
benchmark times (the autotuner's launch shapes, CUDA graphs on).  The oracle
cannot run this size whole, so the checks use outputs it computes one by
one, and properties that hold at any size:

  * density: 96 sampled cells of the 2LPT state, each summed in FP64 over
    the lattice sites that can reach it (oracle.pm.density_at); bound
    1e-5 of max(alpha, 1 + delta) per cell, as in the small-size test;
  * force on a plane wave along x, y or z (uniform across the other two
    axes): the exact PM force reduces to a 1D problem along the wave
    (oracle.pm.force_uniform_yz, pinned against the 3D oracle on the CPU;
    the cubic symmetry of box, lattice and mesh makes it the same function
    for every axis).  The force component along the wave matches it within
    2e-5 of max |F| (the small-size force bound) for every particle; the
    other two vanish to 1e-5 of it.  Each orientation sends non-zero modes
    through the 1024-point transforms of its own axis;
  * momentum conservation on the 2LPT state: with the same assignment for
    paint and read and an odd gradient multiplier (zero at k = 0 and at the
    Nyquist indices), sum_i F_i = 0 exactly; FP32 rounding leaves
    |sum_i F_i| far below 1e-6 of sum_i |F_i| (expected ~1e-9);
  * gradient: dL/dsigma8 and dL/dOm of the MSE density loss from the
    reverse-time adjoint (the benchmark's hot path) against central
    differences of two forward runs each (step 1e-3 relative): agreement to
    1e-2, the accuracy of the differences themselves (FP32 trajectory
    rounding over 100 steps divided by the 1e-3 step).  The adjoint runs
    without stored states, as the benchmark times it, and with a checkpoint
    every 4, 10 and 25 steps (all held to the same bound; the errors are
    printed).  dL/dOm is a small sum of large cancelling per-step terms, so
    it shows the FP32 reversal drift first; with the potential force
    pipeline the reverse steps recompute the force through the same
    arithmetic as the forward ones, which keeps that drift below the
    accuracy of the differences.
"""

import numpy as np
import pytest
import torch

from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300.configs import WORKLOADS

pytestmark = pytest.mark.gpu

W = WORKLOADS["pm512_mesh1024"]


@pytest.fixture(scope="module")
def full():
    from paper_2211_09958_gb300.pm import ParticleMesh
    pm = ParticleMesh(W.n_p, W.n_m, W.box, W.omega_m, W.sigma8, W.n_steps, W.a_init, W.a_final, W.h, W.n_s)
    gen = torch.Generator(device=pm.device)
    gen.manual_seed(W.ic_seed)
    noise = torch.randn((1, W.n_p, W.n_p, W.n_p), generator=gen, device=pm.device, dtype=torch.float32)
    s, p = pm.init_lpt(noise)
    pm.autotune(s)
    st = opm.Setup(W.n_p, W.n_m, W.box, Cosmology(W.omega_m, W.sigma8, W.h, W.n_s), a_init=W.a_init,
                   a_final=W.a_final, n_steps=W.n_steps)
    yield pm, st, noise, gen
    pm.close()
    torch.cuda.empty_cache()


def test_full_size_density_on_sampled_cells(full):
    pm, st, noise, _ = full
    s, _ = pm.init_lpt(noise)
    d = pm.density(s).reshape(-1)
    cells = np.random.default_rng(7).integers(0, W.n_m ** 3, 96)
    got = d[torch.from_numpy(cells).to(d.device)].double().cpu().numpy()
    del d
    s_host = s[0].cpu().numpy()
    ref = opm.density_at(cells, s_host, st, float(np.abs(s_host).max()))
    err = np.abs(got - ref) / np.maximum(st.alpha, 1.0 + ref)
    print(f"density: max err {err.max():.3e} of max(alpha, 1 + delta)")
    assert err.max() < 1e-5, err.max()


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_full_size_plane_wave_force(full, axis):
    # a plane wave along x, y or z: the state is uniform across the other two
    # axes, so each orientation puts non-zero modes through the 1024-point
    # transforms of its own axis (the same 1D reduction holds by the cubic
    # symmetry of box, lattice and mesh)
    pm, st, _, _ = full
    n_p, h_p = W.n_p, W.box / W.n_p
    i = np.arange(n_p)
    sx = (0.4 * h_p * np.sin(2 * np.pi * 8 * (i + 0.25) / n_p) + 0.1 * h_p * np.cos(2 * np.pi * 21 * i / n_p))
    sx = sx.astype(np.float32)
    shape = [1, 1, 1]
    shape[axis] = n_p
    s = torch.zeros((1, n_p, n_p, n_p, 3), dtype=torch.float32, device=pm.device)
    s[0, ..., axis] = torch.from_numpy(sx).to(pm.device).reshape(shape)
    f = pm.pm_force(s.reshape(1, -1, 3)).reshape(n_p, n_p, n_p, 3)
    f = f.movedim(axis, 0).reshape(n_p, n_p * n_p, 3)
    ref = opm.force_uniform_yz(sx.astype(np.float64), st)
    scale = np.abs(ref).max()
    fa = f[..., axis]
    others = [j for j in range(3) if j != axis]
    spread = (fa.max(dim=1).values - fa.min(dim=1).values).max().item()
    assert spread < 2e-5 * scale, spread / scale                        # F_axis depends on that axis alone
    assert f[..., others].abs().max().item() < 1e-5 * scale
    plane = fa[:, 0].double().cpu().numpy()
    print(f"plane wave along axis {axis}: spread {spread / scale:.3e}, "
          f"|F_other| {f[..., others].abs().max().item() / scale:.3e}, "
          f"|F - ref| {np.abs(plane - ref).max() / scale:.3e} of max |F|")
    assert np.abs(plane - ref).max() < 2e-5 * scale, np.abs(plane - ref).max() / scale


def test_full_size_momentum_conservation(full):
    pm, _, noise, _ = full
    s, _ = pm.init_lpt(noise)
    f = pm.pm_force(s)[0].double()
    total = f.sum(dim=0).abs()
    mag = f.abs().sum(dim=0)
    ratio = (total / mag).max().item()
    print(f"momentum: |sum F| / sum |F| = {ratio:.3e}")
    assert ratio < 1e-6, ratio


def _loss(pm, noise, target, om, s8):
    pm.set_cosmology(om, s8)
    s, p = pm.init_lpt(noise)
    pm.integrate(s, p)
    loss, _ = pm.mse_loss(s, target, want_grad=False)
    return float(loss[0])


def test_full_size_cosmology_gradients_against_differences(full):
    pm, _, noise, gen = full
    target = torch.randn((1, W.n_m, W.n_m, W.n_m), generator=gen, device=pm.device, dtype=torch.float32)
    om, s8 = W.omega_m, W.sigma8
    pm.set_cosmology(om, s8)
    grads = {}
    for every in (0, 4, 10, 25):
        pm.set_checkpoints(every)
        s, p = pm.init_lpt(noise)
        f = pm.integrate(s, p)
        _, lam = pm.mse_loss(s, target)
        mu = torch.zeros_like(p)
        dom = pm.adjoint_integrate(s, p, f, lam, mu, mu_zero=True)
        _, dcos = pm.init_lpt_adjoint(lam, mu, noise, want_noise_grad=False)
        del s, p, f, lam, mu
        grads[every] = (dom[0] + dcos[0, 0], dcos[0, 1])
    pm.set_checkpoints(0)
    g_om, g_s8 = grads[0]                # the benchmark's configuration: no stored states
    e8, eo = 1e-3 * s8, 1e-3 * om
    fd_s8 = (_loss(pm, noise, target, om, s8 + e8) - _loss(pm, noise, target, om, s8 - e8)) / (2 * e8)
    fd_om = (_loss(pm, noise, target, om + eo, s8) - _loss(pm, noise, target, om - eo, s8)) / (2 * eo)
    pm.set_cosmology(om, s8)
    print(f"gradients: dL/ds8 {g_s8:.6e} vs {fd_s8:.6e}, dL/dOm {g_om:.6e} vs {fd_om:.6e}")
    for every, (go, gs) in grads.items():
        print(f"  checkpoint every {every}: dL/dOm off by {abs(go - fd_om) / abs(fd_om):.2e}, "
              f"dL/ds8 by {abs(gs - fd_s8) / abs(fd_s8):.2e}")
    for every, (go, gs) in grads.items():
        assert abs(gs - fd_s8) < 1e-2 * abs(fd_s8), (every, gs, fd_s8)
        assert abs(go - fd_om) < 1e-2 * abs(fd_om), (every, go, fd_om)
