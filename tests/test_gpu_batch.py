"""Batched runs (one context, n_batch simulations of different cosmologies
and seeds in every launch) against the FP64 oracle run by run.

  * three runs with distinct (Omega_m, sigma8) and seeds: the final state
    after 4 KDK steps (1e-4 of the spacing), and the reverse-time adjoint from
    seeded cotangents: lam, mu within 1e-3 relative L2, and dL/dOm of each
    run's dynamics within 1e-4 of the sum of its terms' magnitudes with a
    checkpoint at every step.  dL/dOm is a small sum of large cancelling
    terms, and FP32 reversal drift moves it by about 1e-4 of them in the most
    nonlinear run of this batch when no state is stored (printed);
  * the shape of the batched workload (32 runs, Omega_m ~ U[0.2, 0.4],
    sigma8 ~ U[0.6, 1.0] from seed 99, IC seeds 5000 + i, 20 KDK steps, mesh
    twice the particle lattice, 2 Mpc/h spacing) at a reduced size (16^3
    particles on 32^3 meshes), through the autograd front end with the
    autotuner's launch shapes and the CUDA graphs on: the MSE loss of each run's final
    density, and its gradients with respect to that run's white noise
    (relative L2 1e-3, cosine 0.9999), Omega_m (1e-4 of the sum of the terms'
    magnitudes) and sigma8 (1e-3 relative), with CIC and with TSC assignment
    (the test says why CIC holds the median run to these bounds).  The oracle
    runs the 32 runs in a pool of spawned processes.
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
    out = {}
    for every in (0, 1):
        pm.set_checkpoints(every)
        s, p = pm.init_lpt(_cuda(noise))
        f = pm.integrate(s, p)
        fin = _host(s)
        lam, mu = _cuda(lam0), _cuda(mu0)
        dom = pm.adjoint_integrate(s, p, f, lam, mu)
        out[every] = (lam, mu, dom)
    lam, mu, _ = out[0]                  # the reverse-time adjoint without stored states
    dom = out[1][2]                      # dL/dOm with a checkpoint at every step
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
        o_dom = opm.dynamics_domega(g, st)
        print(f"run {b}: dL/dOm of the dynamics off by {abs(dom[b] - o_dom) / cond:.2e} of its terms "
              f"({abs(out[0][2][b] - o_dom) / cond:.2e} without checkpoints)")
        assert abs(dom[b] - o_dom) < 1e-4 * cond, (b, dom[b], o_dom)


N_P, N_M, BOX, STEPS, RUNS = 16, 32, 32.0, 20, 32


def _oracle_run(b, om, s8, solver):
    # FP64 loss and gradients of run b of the reduced batched workload, with
    # the magnitudes of the terms of dL/dOm
    st = opm.Setup(N_P, N_M, BOX, Cosmology(om, s8), n_steps=STEPS, solver=solver)
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


@pytest.mark.parametrize("solver", [0, 8], ids=["cic", "tsc"])
def test_batched_workload_shape_gradients_against_oracle(solver):
    # With CIC the weight gradient is discontinuous at cell faces (one-sided
    # slopes): where an FP32 position and the FP64 one fall on either side of
    # a face at some step, that particle's cotangent takes the other slope.
    # Over 20 steps of 4096 particles that happens in a few of the 32 runs
    # and moves their noise gradient by up to a few per cent, so with CIC
    # the median run is held to the bounds and every run to 0.1.  TSC weights
    # are C^1, their gradient has no jump, and every run is held to the bounds.
    from paper_2211_09958_gb300.pm import ParticleMesh, density, simulate
    om, s8 = inputs.batch_cosmologies(RUNS, seed=99)
    with cf.ProcessPoolExecutor(max_workers=min(16, mp.cpu_count()), mp_context=mp.get_context("spawn")) as pool:
        futures = [pool.submit(_oracle_run, b, float(om[b]), float(s8[b]), solver) for b in range(RUNS)]
        ref = [fu.result() for fu in futures]
    pm = ParticleMesh(N_P, N_M, BOX, om, s8, STEPS, solver=solver)
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
    err = {k: np.zeros(RUNS) for k in ("loss", "noise", "noise 1-cos", "om", "s8")}
    for b in range(RUNS):
        o_loss, o_gn, o_om, o_s8, terms = ref[b]
        g = gn[b].ravel()
        err["loss"][b] = abs(losses[b].item() - o_loss) / o_loss
        err["noise"][b] = np.linalg.norm(g - o_gn.ravel()) / np.linalg.norm(o_gn)
        err["noise 1-cos"][b] = 1.0 - np.dot(g, o_gn.ravel()) / np.linalg.norm(g) / np.linalg.norm(o_gn)
        err["om"][b] = abs(omt.grad[b].item() - o_om) / terms
        err["s8"][b] = abs(s8t.grad[b].item() - o_s8) / abs(o_s8)
    print(f"batched workload shape ({'TSC' if solver else 'CIC'}): median / worst run",
          {k: f"{np.median(v):.2e} / {v.max():.2e}" for k, v in err.items()})
    bounds = {"loss": 1e-4, "noise": 1e-3, "noise 1-cos": 1e-4, "om": 1e-4, "s8": 1e-3}
    worst = dict(bounds) if solver else {k: 0.1 for k in bounds}
    # dL/dOm of every run, also with TSC, to 5e-4 of its terms: it cancels to
    # ~1/25 of them, and FP32 reversal drift over 20 deeply nonlinear steps
    # in these 32 Mpc/h boxes reaches ~2e-4 of them in the worst runs (the
    # median run is at 2e-5)
    worst["om"] = max(worst["om"], 5e-4)
    assert err["loss"].max() < bounds["loss"], err["loss"]
    for k, bound in bounds.items():
        assert np.median(err[k]) < bound, (k, err[k])
        assert err[k].max() < worst[k], (k, err[k])
