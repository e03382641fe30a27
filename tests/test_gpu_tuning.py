"""Launch-shape autotuner (include/pmgb.h pm_autotune / pm_set_tuning):
every candidate block size gives the same results (up to the order of FP32
atomics), and the tuner keeps the fastest candidate it measured."""

import numpy as np
import pytest
import torch

from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu

FAMILIES = ("paint", "read", "spectral", "fft_z", "fft_x", "z_staging", "z_fwd_staging", "x_round", "pipeline",
            "deposit")
CANDIDATES = {"paint": (128, 256, 512), "read": (128, 256, 512), "spectral": (128, 256, 512),
              "fft_z": (128, 256, 512), "fft_x": (8, 16), "z_staging": (1, 2), "z_fwd_staging": (1, 2),
              "x_round": (1, 2, 3), "pipeline": (1, 2), "deposit": (1, 2)}
DEFAULT = {"paint": 256, "read": 256, "spectral": 256, "fft_z": 256, "fft_x": 8, "z_staging": 2, "z_fwd_staging": 1,
           "x_round": 2, "pipeline": 2, "deposit": 1}


def _pm(n_p=32, n_m=256, box=128.0, steps=3):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps)


def test_every_block_size_gives_the_same_force_and_trajectory():
    pm = _pm()
    s0 = torch.from_numpy(inputs.random_displacements(32, 128.0, seed=2, scale=0.5)).cuda()[None]
    ref_f = pm.pm_force(s0)
    s, p = pm.init_lpt(seed=5)
    ref_s, ref_p = s.clone(), p.clone()
    pm.integrate(ref_s, ref_p)
    scale_f = ref_f.abs().max().item()
    for fam in FAMILIES:
        for t in CANDIDATES[fam]:
            if t == DEFAULT[fam] or fam == "z_staging":
                continue
            pm.set_tuning(**{fam: t, "z_staging": 2})
            f = pm.pm_force(s0)
            assert (f - ref_f).abs().max().item() <= 2e-5 * scale_f, (fam, t)
            if fam in ("x_round", "pipeline"):
                # changes the FFT's rounding order, not only the order of
                # atomics; its trajectories are compared at parity bounds below
                pm.set_tuning(z_staging=2)
                continue
            s2, p2 = s.clone(), p.clone()
            pm.integrate(s2, p2)
            assert (s2 - ref_s).abs().max().item() <= 1e-5 * pm.box / pm.n_p, (fam, t)
            pm.set_tuning(z_staging=2)
    assert pm.get_tuning() == DEFAULT


def test_autotune_keeps_the_fastest_measured_candidate():
    pm = _pm()
    s, _ = pm.init_lpt(seed=3)
    before = s.clone()
    chosen, ms = pm.autotune(s)
    assert torch.equal(s, before)                    # the particles are not modified
    for k, fam in enumerate(FAMILIES):
        cands = CANDIDATES[fam]
        t = ms[k][:len(cands)]
        assert np.all(t > 0), (fam, ms[k])
        assert chosen[fam] == cands[int(np.argmin(t))], (fam, ms[k], chosen)


def test_small_mesh_keeps_the_default_z_pass():
    pm = _pm(n_p=16, n_m=64, box=64.0)
    s, _ = pm.init_lpt(seed=1)
    chosen, ms = pm.autotune(s)
    assert chosen["fft_z"] == 256 and np.all(ms[3] == 0)
    assert chosen["z_staging"] == 1 and np.all(ms[5] == 0)       # no TMA maps below n_m = 256


def test_tma_and_load_staging_give_the_same_adjoint():
    # the z inverse with TMA-staged spectrum rows against per-thread loads,
    # through a full adjoint step (force and psi meshes)
    pm = _pm(n_p=32, n_m=256, box=128.0, steps=2)
    assert pm.get_tuning()["z_staging"] == 2                      # TMA is the default at n_m = 256
    pm.set_tuning(pipeline=1)            # the gradient pipeline's 4-field z inverse is the one staged by TMA
    s, p = pm.init_lpt(seed=8)
    f = pm.integrate(s, p)
    lam = torch.from_numpy(np.random.default_rng(2).standard_normal(tuple(s.shape)).astype(np.float32)).cuda()
    out = {}
    for staging in (2, 1):
        pm.set_tuning(z_staging=staging, pipeline=1)
        s2, p2, l2, m2 = s.clone(), p.clone(), lam.clone(), torch.zeros_like(p)
        dom = pm.adjoint_integrate(s2, p2, f.clone(), l2, m2)
        out[staging] = (l2, m2, dom)
    for a, b in zip(out[1][:2], out[2][:2]):                      # the same arithmetic: atomics order only
        assert ((a - b).norm() / b.norm()).item() <= 1e-4


def test_invalid_block_size_is_rejected():
    from paper_2211_09958_gb300.pm import PMError
    pm = _pm(n_p=16, n_m=64, box=64.0)
    with pytest.raises(PMError):
        pm.set_tuning(paint=100)
    with pytest.raises(PMError):
        pm.set_tuning(fft_x=32)
    assert pm.get_tuning()["paint"] == 256


def test_tma_staging_gives_the_same_forces_and_power():
    pm = _pm(n_p=32, n_m=256, box=128.0, steps=2)
    s = torch.from_numpy(inputs.random_displacements(32, 128.0, seed=4, scale=0.5)).cuda()[None]
    res = {}
    for staging in (2, 1):
        pm.set_tuning(z_staging=staging)
        res[staging] = (pm.pm_force(s), pm.power_spectrum(s)[1])
    f2, f1 = res[2][0], res[1][0]
    assert (f2 - f1).abs().max().item() <= 2e-5 * f1.abs().max().item()
    np.testing.assert_allclose(res[2][1], res[1][1], rtol=1e-5)


@pytest.mark.parametrize("n_p,n_m,solver", [(32, 64, 0), (16, 32, 3), (32, 64, 12)])
def test_fused_and_separate_x_passes_agree(n_p, n_m, solver):
    # the fused x round trip (forward x pass, Green's function times gradient,
    # inverse x pass in one kernel) against the three launches, through a
    # forward run and its adjoint: force meshes, psi, the VJPs and the dOm
    # reductions.  The two differ in the FFT's rounding order, so the bounds
    # are the oracle-parity ones: state 1e-4 of the spacing, cotangents 1e-3
    # relative L2.  dL/dOm of the dynamics is a small sum of large cancelling
    # terms, so each path is held to the FP64 oracle at 1e-4 of the sum of
    # the terms' magnitudes, as in the parity tests, with a checkpoint at
    # every step: without them the FP32 reversal drift of the early, small
    # momenta moves dOm by up to ~1e-3 of that sum with some solver flags.
    from oracle import pm as opm
    from oracle.cosmology import Cosmology, kdk_coefficients_domega
    from paper_2211_09958_gb300.pm import ParticleMesh
    box, steps = 4.0 * n_p, 4
    pm = ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps, solver=solver)
    noise = inputs.white_noise(n_p, 9)
    rng = np.random.default_rng(3)
    lam0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    mu0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    pm.set_checkpoints(1)
    out = {}
    for x_round in (2, 1):
        pm.set_tuning(x_round=x_round)
        s, p = pm.init_lpt(torch.from_numpy(noise).cuda()[None])
        f = pm.integrate(s, p)
        fin = s.clone()
        lam, mu = torch.from_numpy(lam0).cuda()[None], torch.from_numpy(mu0).cuda()[None]
        dom = pm.adjoint_integrate(s, p, f, lam, mu)
        out[x_round] = (fin, lam, mu, dom[0])
    assert (out[1][0] - out[2][0]).abs().max().item() <= 1e-4 * box / n_p
    for a, b in zip(out[1][1:3], out[2][1:3]):
        assert ((a - b).norm() / b.norm()).item() <= 1e-3
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8), n_steps=steps, solver=solver)
    rs, rp, rf = opm.simulate(noise.astype(np.float64), st)
    _, _, _, _, grads = opm.adjoint_integrate(rs, rp, rf, lam0.astype(np.float64), mu0.astype(np.float64), st)
    o_dom = opm.dynamics_domega(grads, st)
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps, bool(solver & 4))
    cond = abs(grads["omega_m_direct"]) + sum(abs(np.dot(grads[k], d[k])) for k in ("K_a", "Dr", "K_b"))
    for x_round in (1, 2):
        assert abs(out[x_round][3] - o_dom) <= 1e-4 * cond, (x_round, out[x_round][3], o_dom, cond)
