"""Batched runs (one context, n_batch simulations of different cosmologies
and seeds in every launch) against the FP64 oracle run by run.

  * three runs with distinct (Omega_m, sigma8) and seeds: the final state
    after 4 KDK steps (1e-4 of the spacing), and the reverse-time adjoint from
    seeded cotangents: lam, mu within 1e-3 relative L2 and dL/dOm of each
    run's dynamics within 1e-4 of the sum of its terms' magnitudes;
  * the shape of the batched workload (32 runs, Omega_m ~ U[0.2, 0.4],
    sigma8 ~ U[0.6, 1.0] from seed 99, IC seeds 5000 + i, 20 KDK steps, mesh
    twice the particle lattice, 2 Mpc/h spacing) at a reduced size (16^3
    particles on 32^3 meshes), through the autograd front end with the
    autotuner's launch shapes and the CUDA graphs on: the MSE loss of each run's final
    density, and its gradients with respect to that run's white noise
    (relative L2 1e-3, cosine 0.9999), Omega_m (1e-4 of the sum of the terms'
    magnitudes) and sigma8 (1e-3 relative).  The oracle runs the 32 runs in a
    pool of spawned processes.
"""

import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest
import torch

from oracle import lpt as olpt
from oracle import pm as opm
from oracle.cosmology import Cosmology, kdk_coefficients_domega
from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def test_batched_runs_and_adjoint_against_oracle_per_run():
    from paper_2211_09958_gb300.pm import ParticleMesh
    n_p, n_m, box, steps, B = 16, 32, 64.0, 4, 3
    om, s8 = [0.22, 0.37, 0.3], [0.65, 0.95, 0.8]
    pm = ParticleMesh(n_p, n_m, box, om, s8, steps)
    noise = np.stack([inputs.white_noise(n_p, 300 + b) for b in range(B)])
    rng = np.random.default_rng(17)
    lam0 = rng.standard_normal((B, n_p ** 3, 3)).astype(np.float32)
    mu0 = rng.standard_normal((B, n_p ** 3, 3)).astype(np.float32)
    s, p = pm.init_lpt(_cuda(noise))
    f = pm.integrate(s, p)
    fin = _host(s)
    lam, mu = _cuda(lam0), _cuda(mu0)
    dom = pm.adjoint_integrate(s, p, f, lam, mu)
    for b in range(B):
        st = opm.Setup(n_p, n_m, box, Cosmology(om[b], s8[b]), n_steps=steps)
        rs, rp, rf = opm.simulate(noise[b].astype(np.float64), st)
        assert np.max(np.abs(fin[b] - rs)) < 1e-4 * box / n_p, b
        _, _, olam, omu, g = opm.adjoint_integrate(rs, rp, rf, lam0[b].astype(np.float64),
                                                   mu0[b].astype(np.float64), st)
        for got, ref in ((_host(lam)[b], olam), (_host(mu)[b], omu)):
            assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-3, b
        d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps)
        cond = abs(g["omega_m_direct"]) + sum(abs(np.dot(g[k], d[k])) for k in ("K_a", "Dr", "K_b"))
        assert abs(dom[b] - opm.dynamics_domega(g, st)) < 1e-4 * cond, (b, dom[b], opm.dynamics_domega(g, st))


N_P, N_M, BOX, STEPS, RUNS = 16, 32, 32.0, 20, 32


def _oracle_run(b, om, s8):
    # FP64 loss and gradients of run b of the reduced batched workload, with
    # the magnitudes of the terms of dL/dOm
    st = opm.Setup(N_P, N_M, BOX, Cosmology(om, s8), n_steps=STEPS)
    noise = inputs.white_noise(N_P, 5000 + b).astype(np.float64)
    target = inputs.target_field(N_M, 6000 + b).astype(np.float64)
    s, p, f = opm.simulate(noise, st)
    loss = opm.mse_loss(s, target, st)
    lam = opm.mse_loss_grad(s, target, st)
    _, _, lam0, mu0, g = opm.adjoint_integrate(s, p, f, lam, np.zeros_like(p), st)
    g_noise, g_om_ic, g_s8 = olpt.initial_conditions_vjp(noise, lam0, mu0, st)
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps)
    terms = abs(g["omega_m_direct"]) + sum(abs(np.dot(g[k], d[k])) for k in ("K_a", "Dr", "K_b")) + abs(g_om_ic)
    return loss, g_noise, g_om_ic + opm.dynamics_domega(g, st), g_s8, terms


def test_batched_workload_shape_gradients_against_oracle():
    from paper_2211_09958_gb300.pm import ParticleMesh, density, simulate
    om, s8 = inputs.batch_cosmologies(RUNS, seed=99)
    with cf.ProcessPoolExecutor(max_workers=min(8, mp.cpu_count()), mp_context=mp.get_context("spawn")) as pool:
        futures = [pool.submit(_oracle_run, b, float(om[b]), float(s8[b])) for b in range(RUNS)]
        ref = [fu.result() for fu in futures]
    pm = ParticleMesh(N_P, N_M, BOX, om, s8, STEPS)
    noise = _cuda(np.stack([inputs.white_noise(N_P, 5000 + b) for b in range(RUNS)]))
    target = _cuda(np.stack([inputs.target_field(N_M, 6000 + b) for b in range(RUNS)]))
    s, _ = pm.init_lpt(noise)
    pm.autotune(s)
    nz = noise.clone().requires_grad_(True)
    omt = torch.tensor(om, dtype=torch.float64, requires_grad=True)
    s8t = torch.tensor(s8, dtype=torch.float64, requires_grad=True)
    s, _ = simulate(pm, nz, omt, s8t)
    d = density(pm, s)
    losses = torch.mean((d - target) ** 2, dim=(1, 2, 3))
    losses.sum().backward()
    gn = _host(nz.grad)
    worst = {"loss": 0.0, "noise": 0.0, "om": 0.0, "s8": 0.0}
    for b in range(RUNS):
        o_loss, o_gn, o_om, o_s8, terms = ref[b]
        g = gn[b].ravel()
        rel = np.linalg.norm(g - o_gn.ravel()) / np.linalg.norm(o_gn)
        cos = np.dot(g, o_gn.ravel()) / np.linalg.norm(g) / np.linalg.norm(o_gn)
        worst["loss"] = max(worst["loss"], abs(losses[b].item() - o_loss) / o_loss)
        worst["noise"] = max(worst["noise"], rel)
        worst["om"] = max(worst["om"], abs(omt.grad[b].item() - o_om) / terms)
        worst["s8"] = max(worst["s8"], abs(s8t.grad[b].item() - o_s8) / abs(o_s8))
        assert cos > 0.9999, (b, cos)
    print("batched workload shape, worst run:", {k: f"{v:.2e}" for k, v in worst.items()})
    assert worst["loss"] < 1e-4 and worst["noise"] < 1e-3, worst
    assert worst["om"] < 1e-4 and worst["s8"] < 1e-3, worst
