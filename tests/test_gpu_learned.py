"""GPU parity of the learned force correction (BF16 tensor-core MLP,
include/pmgb.h pm_nn_*) against the FP64 oracle of oracle/learned.py, which
rounds to bfloat16 at the same points as the kernels.

Tolerances: both sides see the same bf16 operands, so differences come from
FP32 vs FP64 accumulation and FP32 atomics in the paint, and from the rare
bf16 rounding decisions those flip (a value within ~1e-7 relative of a bf16
rounding midpoint, probability ~1e-5 per activation).  Predictions: relative
L2 <= 1e-3; loss: relative 1e-3; gradient: relative L2 <= 5e-3, cosine >=
0.9999.
"""

import numpy as np
import pytest
import torch

from oracle import learned as olearned
from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu

SIZES = (olearned.N_IN, olearned.N_HID, olearned.N_HID, olearned.N_OUT)


def _pm(n_p, n_m, box, steps=4, om=0.3, s8=0.8):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, om, s8, steps)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _setup(pm, om=0.3, s8=0.8):
    return opm.Setup(pm.n_p, pm.n_m, pm.box, Cosmology(om, s8), n_steps=pm.n_steps)


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_param_count():
    pm = _pm(16, 32, 64.0)
    assert pm.nn_param_count() == olearned.n_params()


@pytest.mark.parametrize("n_p,n_m,box,a", [(16, 32, 64.0, 0.5), (16, 16, 40.0, 1.0), (32, 64, 128.0, 0.25)])
def test_predict_parity(n_p, n_m, box, a):
    pm = _pm(n_p, n_m, box)
    theta = inputs.mlp_params(SIZES, seed=n_m)
    pm.nn_set_params(theta)
    s = inputs.random_displacements(n_p, box, seed=5, scale=0.6)
    got = _host(pm.nn_predict(_cuda(s)[None], a))[0]
    ref = olearned.predict(s.astype(np.float64), a, theta.astype(np.float64), _setup(pm))
    assert _rel(got, ref) < 1e-3, _rel(got, ref)


def test_predict_batch_per_run_scale():
    """Each run of a batch uses its own Om in the output scale 3/2 Om h."""
    oms, s8s = np.array([0.25, 0.35]), np.array([0.8, 0.7])
    pm = _pm(16, 32, 64.0, om=oms, s8=s8s)
    theta = inputs.mlp_params(SIZES, seed=3)
    pm.nn_set_params(theta)
    s = np.stack([inputs.random_displacements(16, 64.0, seed=10 + b, scale=0.5) for b in range(2)])
    got = _host(pm.nn_predict(_cuda(s), 0.6))
    for b in range(2):
        ref = olearned.predict(s[b].astype(np.float64), 0.6, theta.astype(np.float64),
                               _setup(pm, oms[b], s8s[b]))
        assert _rel(got[b], ref) < 1e-3


@pytest.mark.parametrize("n_p,n_m,box", [(16, 32, 64.0), (16, 16, 48.0)])
def test_gradient_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    theta = inputs.mlp_params(SIZES, seed=11)
    pm.nn_set_params(theta)
    s = inputs.random_displacements(n_p, box, seed=6, scale=0.6)
    target = inputs.random_displacements(n_p, box, seed=7, scale=0.5)
    loss = pm.nn_train_step(_cuda(s)[None], _cuda(target)[None], 0.7, apply=False)
    _, grad = pm.nn_get_params()
    rl, rg = olearned.loss_and_grad(s.astype(np.float64), target.astype(np.float64), 0.7,
                                    theta.astype(np.float64), _setup(pm))
    assert abs(loss - rl) <= 1e-3 * abs(rl)
    g = grad.astype(np.float64)
    assert _rel(g, rg) < 5e-3, _rel(g, rg)
    assert g @ rg / np.linalg.norm(g) / np.linalg.norm(rg) > 0.9999
    # the sample weight scales the gradient, not the reported loss (a power
    # of two, so that the bf16 roundings scale exactly; FP32 atomics remain)
    loss4 = pm.nn_train_step(_cuda(s)[None], _cuda(target)[None], 0.7, apply=False, weight=4.0)
    _, grad4 = pm.nn_get_params()
    assert abs(loss4 - loss) <= 1e-6 * abs(loss)
    assert _rel(grad4.astype(np.float64), 4.0 * g) < 1e-4
    # every parameter block carries gradient
    k = 0
    for name, shape in olearned.param_shapes():
        size = int(np.prod(shape))
        assert _rel(g[k:k + size], rg[k:k + size]) < 1e-2, name
        k += size


def test_adam_step_matches_definition():
    """One Adam step (bias-corrected, beta 0.9 / 0.999, eps 1e-8) from zero
    moments moves each parameter by lr * g / (|g| + eps')."""
    pm = _pm(16, 32, 64.0)
    theta = inputs.mlp_params(SIZES, seed=12)
    pm.nn_set_params(theta)
    s = inputs.random_displacements(16, 64.0, seed=8, scale=0.6)
    target = inputs.random_displacements(16, 64.0, seed=9, scale=0.5)
    pm.nn_train_step(_cuda(s)[None], _cuda(target)[None], 0.7, lr=1e-3, step=1, apply=True)
    new, g = pm.nn_get_params()
    g = g.astype(np.float64)
    expect = theta - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(new - expect)) < 1e-6


def test_zero_network_leaves_integration_unchanged():
    """Zero last layer and biases: the correction adds exact zeros."""
    pm = _pm(16, 32, 64.0)
    s0, p0 = pm.init_lpt(seed=4)
    s1, p1 = s0.clone(), p0.clone()
    pm.integrate(s1, p1)
    pm.nn_set_params(olearned.init_params(1).astype(np.float32))
    pm.nn_enable(True)
    s2, p2 = s0.clone(), p0.clone()
    pm.integrate(s2, p2)
    # FP32 atomics make two plain runs differ in the last bits already
    spacing = pm.box / pm.n_p
    assert torch.max(torch.abs(s1 - s2)).item() < 1e-5 * spacing
    assert torch.max(torch.abs(p1 - p2)).item() < 1e-5 * torch.max(torch.abs(p1)).item()


def test_corrected_integration_parity():
    """pm_integrate with the correction enabled follows the oracle's KDK with
    force = PM force + network correction at each evaluation's a."""
    pm = _pm(16, 32, 64.0, steps=4)
    theta = inputs.mlp_params(SIZES, seed=13) * np.float32(0.3)
    pm.nn_set_params(theta)
    pm.nn_enable(True)
    noise = inputs.white_noise(16, seed=21)
    s, p = pm.init_lpt(_cuda(noise)[None])
    s0, p0 = _host(s)[0], _host(p)[0]
    pm.integrate(s, p)
    setup = _setup(pm)
    a_grid = setup.a_init + (setup.a_final - setup.a_init) * np.arange(pm.n_steps + 1) / pm.n_steps
    calls = [0]

    def force_fn(y):
        a = a_grid[calls[0]]
        calls[0] += 1
        return opm.force(y, setup) + olearned.predict(y, a, theta.astype(np.float64), setup)

    rs, rp, _ = opm.integrate(s0, p0, setup, force_fn)
    assert calls[0] == pm.n_steps + 1
    # A bf16 rounding decision that FP32 and FP64 accumulation take
    # differently changes one hidden activation of one cell by 2^-8 relative;
    # the particles near that cell then drift apart, so the state bound
    # (1e-4 of the spacing) holds for 99.9 % of the particles and a 10x
    # looser one for all of them.
    spacing = pm.box / pm.n_p
    ds = np.abs(_host(s)[0] - rs)
    dp = np.abs(_host(p)[0] - rp) / np.max(np.abs(rp))
    assert np.quantile(ds, 0.999) < 1e-4 * spacing and np.max(ds) < 1e-3 * spacing, np.max(ds)
    assert np.quantile(dp, 0.999) < 1e-4 and np.max(dp) < 1e-3, np.max(dp)


def test_corrected_adjoint_parity():
    """pm_adjoint_integrate with the correction on differentiates the
    corrected dynamics: cotangents of the initial state and the parameter
    gradient against the oracle's adjoint_corrected (bf16 rounding points of
    the network's backward; relative L2 1e-2, cosine 0.999)."""
    pm = _pm(16, 32, 64.0, steps=3)
    theta = inputs.mlp_params(SIZES, seed=17) * np.float32(0.3)
    pm.nn_set_params(theta)
    pm.nn_enable(True)
    s, p = pm.init_lpt(_cuda(inputs.white_noise(16, seed=23))[None])
    f = pm.integrate(s, p)
    sN, pN, fN = _host(s)[0], _host(p)[0], _host(f)[0]
    rng = np.random.default_rng(5)
    lam = rng.standard_normal(sN.shape).astype(np.float32)
    mu = (0.1 * rng.standard_normal(sN.shape)).astype(np.float32)
    lam_d, mu_d = _cuda(lam)[None], _cuda(mu)[None]
    pm.adjoint_integrate(s, p, f, lam_d, mu_d)
    _, g_theta = pm.nn_get_params()
    rs, rp, rl, rm, rg = olearned.adjoint_corrected(sN, pN, fN, lam.astype(np.float64), mu.astype(np.float64),
                                                    theta.astype(np.float64), _setup(pm))
    spacing = pm.box / pm.n_p
    assert np.max(np.abs(_host(s)[0] - rs)) < 1e-3 * spacing
    for got, ref in ((_host(lam_d)[0], rl), (_host(mu_d)[0], rm), (g_theta.astype(np.float64), rg)):
        assert _rel(got, ref) < 1e-2, _rel(got, ref)
        assert got.ravel() @ ref.ravel() / np.linalg.norm(got) / np.linalg.norm(ref) > 0.999


def test_adam_step_from_the_adjoint_gradient():
    pm = _pm(16, 32, 64.0, steps=2)
    theta = inputs.mlp_params(SIZES, seed=19) * np.float32(0.3)
    pm.nn_set_params(theta)
    pm.nn_enable(True)
    s, p = pm.init_lpt(seed=3)
    f = pm.integrate(s, p)
    lam = torch.randn_like(s)
    pm.adjoint_integrate(s, p, f, lam, torch.zeros_like(p))
    _, g = pm.nn_get_params()
    pm.nn_adam_step(1e-3, 1)
    new, _ = pm.nn_get_params()
    expect = theta - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.max(np.abs(new - expect)) < 1e-6


def test_non_pow2_mesh_refused():
    from paper_2211_09958_gb300.pm import PMError
    pm = _pm(12, 24, 48.0)
    with pytest.raises(PMError):
        pm.nn_set_params(olearned.init_params(1).astype(np.float32))


def test_training_reduces_force_error():
    """Force matching against the 4x-finer-mesh force: 60 Adam steps on one
    snapshot lower the loss below the uncorrected error |F_fine - F_coarse|^2."""
    from paper_2211_09958_gb300.pm import ParticleMesh
    coarse = ParticleMesh(32, 32, 64.0, 0.3, 0.8, 10)
    fine = ParticleMesh(32, 128, 64.0, 0.3, 0.8, 10)
    s, p = coarse.init_lpt(seed=31)
    coarse.integrate(s, p)
    # the lattice sits half a mesh cell off the nodes: same positions, shifted s
    from paper_2211_09958_gb300.learn import lattice_shift
    target = fine.pm_force(s + lattice_shift(coarse, fine)) - coarse.pm_force(s)
    base = float((target ** 2).sum(-1).mean())
    coarse.nn_set_params(olearned.init_params(2).astype(np.float32))
    first = coarse.nn_train_step(s, target, 1.0, lr=2e-3, step=1)
    assert abs(first - base) <= 1e-4 * base        # zero last layer: loss = |T|^2
    for k in range(2, 61):
        last = coarse.nn_train_step(s, target, 1.0, lr=2e-3, step=k)
    assert last < 0.8 * base, (last, base)
