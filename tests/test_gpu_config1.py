"""Parity of the 128^3-particle, 256^3-mesh gradient workload (256 Mpc/h,
63 KDK steps from 2LPT at a = 1/64, MSE of the final CIC density against a
seeded N(0, 1) target) against the FP64 oracle, in the autotuner's launch
shapes with the CUDA graphs on.

The oracle's full run takes over an hour on host cores, so its results come
from ``tests/golden/pm128_mesh256.npz``, written by the committed script
``tests/golden/make_pm128_mesh256.py`` (oracle calls only), on fixed samples
of 8192 particles and 32768 white-noise sites.  Bounds (FP32 against FP64):

  * after 10 steps: |ds| <= 1e-4 of the inter-particle spacing, |dp| <= 1e-4
    of max |p| (the small-size state bounds);
  * at a = 1: at least 99.9 % of the sampled particles within 1e-3 of the
    spacing.  FP32 rounding differences are amplified by the nonlinear
    evolution (shell crossing in collapsed regions) over 63 steps, so the
    bound is relaxed here and the measured maximum is printed;
  * the loss within 1e-4 relative and dL/dsigma8 within 1e-3 relative;
    the white-noise gradient within 2e-3 relative L2 on the sample with
    cosine >= 0.9999; dL/dOm within 1e-4 of the sum of its terms'
    magnitudes.  The gradients come from the reverse-time adjoint without
    stored states (the benchmark's configuration) and with a checkpoint every
    4 steps.  Measured on a GB300: noise gradient 1.5e-3 either way, which
    checkpoints do not change: CIC weight slopes are one-sided, so a particle
    whose FP32 position and FP64 one straddle a cell face at some step takes
    the other slope, and over 2M particles and 63 steps that happens (the
    batched test shows the same gradients with TSC weights, which have no
    jump, within 1e-4).  dL/dOm cancels to 1/300 of its terms here, so its
    relative error is 300 times the terms' FP32 accuracy: 1.4e-2 without
    stored states (4.6e-5 of the terms), 1.0e-3 to 1.6e-3 with a checkpoint
    every 4 steps (3e-6 to 5e-6 of the terms; the read's block shape sets the
    order of the per-block reduction sums), held to 3e-3 for that run.  The cotangents (lam, mu) of the initial
    state carry the reversal drift: within 1e-2 relative L2 without stored
    states (measured 4e-3) and 2e-3 with checkpoints (measured 1.3e-3).
"""

import os

import numpy as np
import pytest
import torch

from paper_2211_09958_gb300 import inputs
from paper_2211_09958_gb300.configs import WORKLOADS

pytestmark = pytest.mark.gpu

W = WORKLOADS["pm128_mesh256"]
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "pm128_mesh256.npz")


@pytest.fixture(scope="module")
def run():
    from paper_2211_09958_gb300.pm import ParticleMesh
    ref = dict(np.load(GOLDEN))
    pm = ParticleMesh(W.n_p, W.n_m, W.box, W.omega_m, W.sigma8, W.n_steps, W.a_init, W.a_final, W.h, W.n_s)
    noise = torch.from_numpy(inputs.white_noise(W.n_p, W.ic_seed)).cuda()[None]
    target = torch.from_numpy(inputs.target_field(W.n_m, W.target_seed)).cuda()[None]
    s, _ = pm.init_lpt(noise)
    pm.autotune(s)
    part = torch.from_numpy(ref["part"]).cuda()
    out = {}
    for every in (0, 4):
        pm.set_checkpoints(every)
        s, p = pm.init_lpt(noise)
        pm.integrate(s, p, 0, 10)
        out[every, "s10"], out[every, "p10"] = s[0, part].double().cpu().numpy(), p[0, part].double().cpu().numpy()
        f = pm.integrate(s, p, 10, W.n_steps)
        out[every, "s63"], out[every, "p63"] = s[0, part].double().cpu().numpy(), p[0, part].double().cpu().numpy()
        loss, lam = pm.mse_loss(s, target)
        mu = torch.zeros_like(p)
        dom = pm.adjoint_integrate(s, p, f, lam, mu, mu_zero=True)
        out[every, "lam0"], out[every, "mu0"] = (lam[0, part].double().cpu().numpy(),
                                                 mu[0, part].double().cpu().numpy())
        dnoise, dcos = pm.init_lpt_adjoint(lam, mu, noise)
        out[every, "loss"] = loss[0]
        out[every, "g_om"] = dom[0] + dcos[0, 0]
        out[every, "g_s8"] = dcos[0, 1]
        out[every, "g_noise"] = dnoise.reshape(-1)[torch.from_numpy(ref["cells"]).cuda()].double().cpu().numpy()
    pm.set_checkpoints(0)
    yield ref, out
    pm.close()
    torch.cuda.empty_cache()


def test_state_after_ten_steps(run):
    ref, out = run
    spacing = W.box / W.n_p
    ds = np.abs(out[0, "s10"] - ref["s10"]).max() / spacing
    dp = np.abs(out[0, "p10"] - ref["p10"]).max() / ref["p10_max"]
    print(f"10 steps: max |ds| {ds:.2e} of the spacing, max |dp| {dp:.2e} of max |p|")
    assert ds < 1e-4 and dp < 1e-4, (ds, dp)


def test_state_at_a_equal_one(run):
    ref, out = run
    spacing = W.box / W.n_p
    ds = np.abs(out[0, "s63"] - ref["s63"]).max(axis=1) / spacing
    frac = np.mean(ds <= 1e-3)
    print(f"a = 1: {100 * frac:.3f} % of particles within 1e-3 of the spacing; max {ds.max():.2e}, "
          f"median {np.median(ds):.2e}")
    assert frac >= 0.999, (frac, ds.max())


@pytest.mark.parametrize("every", [0, 4])
def test_gradients(run, every):
    ref, out = run
    rel = {}
    for k in ("lam0", "mu0", "g_noise"):
        got, want = out[every, k].ravel(), ref[k].astype(np.float64).ravel()
        rel[k] = np.linalg.norm(got - want) / np.linalg.norm(want)
        rel[k + " cos"] = np.dot(got, want) / np.linalg.norm(got) / np.linalg.norm(want)
    rel["loss"] = abs(out[every, "loss"] - float(ref["loss"])) / float(ref["loss"])
    rel["s8"] = abs(out[every, "g_s8"] - float(ref["g_s8"])) / abs(float(ref["g_s8"]))
    rel["om"] = abs(out[every, "g_om"] - float(ref["g_om"])) / abs(float(ref["g_om"]))
    rel["om/terms"] = abs(out[every, "g_om"] - float(ref["g_om"])) / float(ref["g_om_terms"])
    print(f"checkpoint every {every}: " + ", ".join(f"{k} {v:.6g}" for k, v in rel.items()))
    assert rel["loss"] < 1e-4, rel
    assert rel["g_noise"] < 2e-3 and rel["g_noise cos"] > 0.9999, rel
    for k in ("lam0", "mu0"):
        assert rel[k] < (2e-3 if every else 1e-2) and rel[k + " cos"] > 0.9999, (k, rel)
    assert rel["s8"] < 1e-3, rel
    assert rel["om/terms"] < 1e-4, rel
    if every:
        assert rel["om"] < 3e-3, rel
