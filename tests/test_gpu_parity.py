"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Inputs come from the seeded generators of ``paper_2211_09958_gb300.inputs``
and reach both sides as the same float32 values.  Tolerances (FP32 vs FP64,
non-bit-exact because floating-point atomics add in arbitrary order):
  * particle state: max |ds| <= 1e-4 of the mean inter-particle spacing
    (the target accuracy of the method's state), max |dp| <= 1e-4 of max |p| (the same relative
    bound on the momentum scale; the largest errors sit with the largest
    momenta, in collapsed regions)
  * reversal (forward then reverse, both FP32): |ds| <= 1e-4 of the spacing
    and |dp| <= 3e-4 of rms of the FINAL momenta: rounding happens at the
    scale of the late, large momenta (g_p grows ~ a^1.5, x500 from a = 1/64),
    so relative to the tiny initial momenta the same absolute error is large
  * force: max |dF| <= 2e-5 of max |F| (FP32 paint/FFT/read rounding,
    ~1e-7 per operation times the log2(n^3) FFT depth and the 8-corner sums)
  * density: 1e-5 of alpha (sums of at most a few dozen FP32 weights)
  * power spectrum: 1e-3 relative per bin (the 0.1 % target accuracy of P(k))
  * gradients: relative L2 <= 1e-3 and cosine >= 0.9999; sigma8 derivative
    within 1e-3 relative.  dL/dOm is a sum of contributions (initial
    conditions, force prefactor, each KDK factor) that are ~100x larger than
    the total and cancel, so its bound is 1e-4 of the sum of the
    contributions' magnitudes (FP32 rounding of each term), taken from the
    oracle's decomposition
  * reversal: the FP32 forward-then-reverse error is bounded by 3e-4 of the
    spacing (measured ~1e-4 after 10 steps; exact only in exact arithmetic)
"""

import numpy as np
import pytest
import torch

from oracle import lpt as olpt
from oracle import philox as ophilox
from oracle import pm as opm
from oracle.cosmology import Cosmology
from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pm(n_p, n_m, box, steps=4, om=0.3, s8=0.8, **kw):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, om, s8, steps, **kw)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _setup(pm, om=0.3, s8=0.8):
    return opm.Setup(pm.n_p, pm.n_m, pm.box, Cosmology(om, s8), n_steps=pm.n_steps)


GEOMS = [(16, 32, 64.0), (18, 36, 50.0), (20, 30, 70.0), (32, 64, 128.0), (12, 12, 40.0)]


@pytest.mark.parametrize("n_p,n_m,box", GEOMS)
def test_force_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    s = inputs.random_displacements(n_p, box, seed=n_p + n_m, scale=0.6)
    f = _host(pm.pm_force(_cuda(s)[None]))[0]
    ref = opm.force(s.astype(np.float64), _setup(pm))
    err = np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    assert err < 2e-5, err


@pytest.mark.parametrize("n_p,n_m,box", GEOMS)
def test_density_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    s = inputs.random_displacements(n_p, box, seed=3, scale=0.8)
    d = _host(pm.density(_cuda(s)[None]))[0]
    ref = opm.density(s.astype(np.float64), _setup(pm))
    assert np.max(np.abs(d - ref)) < 1e-5 * pm.cfg.n_m ** 3 / n_p ** 3 + 1e-6
    assert abs(d.sum()) < 1e-6 * d.size * (n_m / n_p) ** 3       # mass conservation


def test_density_adjoint_and_mse_parity():
    n_p, n_m, box = 16, 32, 64.0
    pm = _pm(n_p, n_m, box)
    st = _setup(pm)
    s = inputs.random_displacements(n_p, box, seed=5, scale=0.8)
    g = inputs.target_field(n_m, 9)
    ds = _host(pm.density_adjoint(_cuda(s)[None], _cuda(g)[None]))[0]
    ref = opm.density_vjp(s.astype(np.float64), g.astype(np.float64), st)
    assert np.max(np.abs(ds - ref)) < 1e-5 * np.max(np.abs(ref))
    loss, lam = pm.mse_loss(_cuda(s)[None], _cuda(g)[None])
    o_loss = opm.mse_loss(s.astype(np.float64), g.astype(np.float64), st)
    o_lam = opm.mse_loss_grad(s.astype(np.float64), g.astype(np.float64), st)
    assert abs(loss[0] - o_loss) < 1e-5 * o_loss
    assert np.max(np.abs(_host(lam)[0] - o_lam)) < 1e-4 * np.max(np.abs(o_lam))


@pytest.mark.parametrize("n_p,n_m,box", [(32, 64, 128.0), (18, 36, 50.0)])
def test_power_spectrum_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    s = inputs.random_displacements(n_p, box, seed=11, scale=1.0)
    k, pk, nmod = pm.power_spectrum(_cuda(s)[None])
    ok, opk, onm = opm.power_spectrum(s.astype(np.float64), _setup(pm))
    np.testing.assert_array_equal(nmod[0], onm)
    np.testing.assert_allclose(k[0], ok, rtol=1e-12)
    np.testing.assert_allclose(pk[0], opk, rtol=1e-3)


@pytest.mark.parametrize("n_p,n_m,box", [(32, 64, 128.0), (18, 36, 50.0), (20, 30, 70.0)])
def test_init_lpt_parity(n_p, n_m, box):
    pm = _pm(n_p, n_m, box)
    noise = inputs.white_noise(n_p, 21)
    s, p = pm.init_lpt(_cuda(noise)[None])
    rs, rp = olpt.initial_conditions(noise.astype(np.float64), _setup(pm))
    spacing = box / n_p
    assert np.max(np.abs(_host(s)[0] - rs)) < 1e-4 * spacing
    assert np.max(np.abs(_host(p)[0] - rp)) < 1e-4 * np.sqrt(np.mean(rp ** 2))


def test_device_philox_noise_matches_oracle_generator():
    n_p, n_m, box = 16, 32, 64.0
    pm = _pm(n_p, n_m, box)
    s, _ = pm.init_lpt(None, seed=77)
    rs, _ = olpt.initial_conditions(ophilox.white_noise(n_p, 77), _setup(pm))
    assert np.max(np.abs(_host(s)[0] - rs)) < 1e-4 * box / n_p


@pytest.mark.parametrize("n_p,n_m,box,steps", [(32, 64, 128.0, 10), (18, 36, 50.0, 6), (20, 30, 70.0, 5)])
def test_integrate_parity(n_p, n_m, box, steps):
    pm = _pm(n_p, n_m, box, steps)
    noise = inputs.white_noise(n_p, 0)
    s, p = pm.init_lpt(_cuda(noise)[None])
    f = pm.integrate(s, p)
    st = _setup(pm)
    rs, rp, rf = opm.simulate(noise.astype(np.float64), st)
    spacing = box / n_p
    ds = np.max(np.abs(_host(s)[0] - rs)) / spacing
    dp = np.max(np.abs(_host(p)[0] - rp)) / np.max(np.abs(rp))
    assert ds < 1e-4 and dp < 1e-4, (ds, dp)
    assert np.max(np.abs(_host(f)[0] - rf)) < 1e-3 * np.max(np.abs(rf))


def test_kdk_step_equals_merged_integrate():
    n_p, n_m, box, steps = 16, 32, 64.0, 5
    pm = _pm(n_p, n_m, box, steps)
    noise = _cuda(inputs.white_noise(n_p, 3))[None]
    s, p = pm.init_lpt(noise)
    s2, p2 = s.clone(), p.clone()
    f = pm.pm_force(s)
    for n in range(steps):
        pm.kdk_step(n, s, p, f)
    f2 = pm.integrate(s2, p2)
    assert torch.max(torch.abs(s - s2)).item() < 1e-5 * box / n_p
    assert torch.max(torch.abs(f - f2)).item() < 1e-4 * torch.max(torch.abs(f)).item()


def test_integrate_in_segments_equals_one_run():
    n_p, n_m, box, steps = 16, 32, 64.0, 6
    pm = _pm(n_p, n_m, box, steps)
    s, p = pm.init_lpt(_cuda(inputs.white_noise(n_p, 4))[None])
    s2, p2 = s.clone(), p.clone()
    pm.integrate(s, p)
    pm.integrate(s2, p2, 0, 2)
    pm.integrate(s2, p2, 2, 6)
    assert torch.max(torch.abs(s - s2)).item() < 1e-5 * box / n_p
    assert torch.max(torch.abs(p - p2)).item() < 1e-5 * torch.sqrt(torch.mean(p * p)).item()


def test_forward_then_reverse_returns_initial_state():
    n_p, n_m, box, steps = 32, 64, 128.0, 10
    pm = _pm(n_p, n_m, box, steps)
    s, p = pm.init_lpt(_cuda(inputs.white_noise(n_p, 0))[None])
    s0, p0 = s.clone(), p.clone()
    f = pm.integrate(s, p)
    p_scale = torch.sqrt(torch.mean(p * p)).item()
    lam, mu = torch.zeros_like(s), torch.zeros_like(p)
    pm.adjoint_integrate(s, p, f, lam, mu)
    ds = torch.max(torch.abs(s - s0)).item() / (box / n_p)
    dp = torch.max(torch.abs(p - p0)).item() / p_scale
    assert ds < 3e-4 and dp < 3e-4, (ds, dp)


def test_adjoint_integrate_parity():
    n_p, n_m, box, steps = 16, 32, 64.0, 4
    pm = _pm(n_p, n_m, box, steps)
    st = _setup(pm)
    noise = inputs.white_noise(n_p, 12)
    rng = np.random.default_rng(5)
    lam0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    mu0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    s, p = pm.init_lpt(_cuda(noise)[None])
    f = pm.integrate(s, p)
    lam, mu = _cuda(lam0)[None], _cuda(mu0)[None]
    dom = pm.adjoint_integrate(s, p, f, lam, mu)
    rs, rp, rf = opm.simulate(noise.astype(np.float64), st)
    _, _, olam, omu, grads = opm.adjoint_integrate(rs, rp, rf, lam0.astype(np.float64), mu0.astype(np.float64), st)
    for got, ref in ((_host(lam)[0], olam), (_host(mu)[0], omu)):
        rel = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert rel < 1e-3, rel
    o_dom = opm.dynamics_domega(grads, st)
    from oracle.cosmology import kdk_coefficients_domega
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps)
    cond = abs(grads["omega_m_direct"]) + sum(abs(np.dot(grads[k], d[k])) for k in ("K_a", "Dr", "K_b"))
    assert abs(dom[0] - o_dom) < 1e-4 * cond, (dom, o_dom, cond)


def test_init_lpt_adjoint_parity():
    n_p, n_m, box = 16, 32, 64.0
    pm = _pm(n_p, n_m, box)
    noise = inputs.white_noise(n_p, 13)
    rng = np.random.default_rng(6)
    lam = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    mu = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    dn, dcos = pm.init_lpt_adjoint(_cuda(lam)[None], _cuda(mu)[None], _cuda(noise)[None])
    gn, gom, gs8 = olpt.initial_conditions_vjp(noise.astype(np.float64), lam.astype(np.float64),
                                                mu.astype(np.float64), _setup(pm))
    got = _host(dn)[0]
    assert np.linalg.norm(got - gn) / np.linalg.norm(gn) < 1e-4
    assert abs(dcos[0, 0] - gom) < 1e-4 * abs(gom), (dcos, gom)
    assert abs(dcos[0, 1] - gs8) < 1e-4 * abs(gs8), (dcos, gs8)


@pytest.mark.parametrize("n_p,n_m,box,steps", [(32, 64, 128.0, 10), (18, 36, 50.0, 5)])
def test_loss_gradient_parity(n_p, n_m, box, steps):
    from paper_2211_09958_gb300.pm import density, simulate
    pm = _pm(n_p, n_m, box, steps)
    st = _setup(pm)
    noise = inputs.white_noise(n_p, 0)
    target = inputs.target_field(n_m, 1)
    nz = _cuda(noise)[None].requires_grad_(True)
    om = torch.tensor([0.3], dtype=torch.float64, requires_grad=True)
    s8 = torch.tensor([0.8], dtype=torch.float64, requires_grad=True)
    s, _ = simulate(pm, nz, om, s8)
    d = density(pm, s)
    loss = torch.mean((d - _cuda(target)[None]) ** 2)
    loss.backward()
    o_loss, o_gn, o_om, o_s8 = opm.loss_and_grad(noise.astype(np.float64), target.astype(np.float64), st)
    assert abs(loss.item() - o_loss) < 1e-4 * o_loss
    g = _host(nz.grad)[0].ravel()
    rel = np.linalg.norm(g - o_gn.ravel()) / np.linalg.norm(o_gn)
    cos = np.dot(g, o_gn.ravel()) / np.linalg.norm(g) / np.linalg.norm(o_gn)
    assert rel < 1e-3 and cos > 0.9999, (rel, cos)
    assert abs(s8.grad.item() - o_s8) < 1e-3 * abs(o_s8), (s8.grad, o_s8)
    assert abs(om.grad.item() - o_om) < 1e-4 * _omega_condition(noise, target, st), (om.grad, o_om)


def _omega_condition(noise, target, st):
    # sum of |contributions| to the oracle's dL/dOm
    from oracle.cosmology import kdk_coefficients_domega
    s, p, f = opm.simulate(noise.astype(np.float64), st)
    lam = opm.mse_loss_grad(s, target.astype(np.float64), st)
    _, _, lam0, mu0, g = opm.adjoint_integrate(s, p, f, lam, np.zeros_like(p), st)
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps)
    _, g_ic, _ = olpt.initial_conditions_vjp(noise.astype(np.float64), lam0, mu0, st)
    return (abs(g["omega_m_direct"]) + sum(abs(np.dot(g[k], d[k])) for k in ("K_a", "Dr", "K_b")) + abs(g_ic))


def test_batch_runs_equal_single_runs():
    n_p, n_m, box, steps = 16, 32, 64.0, 4
    om, s8 = [0.25, 0.35, 0.3], [0.7, 0.9, 0.8]
    pmb = _pm(n_p, n_m, box, steps, om=om, s8=s8)
    noise = np.stack([inputs.white_noise(n_p, 100 + b) for b in range(3)])
    s, p = pmb.init_lpt(_cuda(noise))
    pmb.integrate(s, p)
    for b in range(3):
        pm1 = _pm(n_p, n_m, box, steps, om=om[b], s8=s8[b])
        s1, p1 = pm1.init_lpt(_cuda(noise[b])[None])
        pm1.integrate(s1, p1)
        assert torch.max(torch.abs(s1[0] - s[b])).item() < 1e-5 * box / n_p


def test_errors_do_not_poison_the_context():
    from paper_2211_09958_gb300.pm import PMError
    pm = _pm(16, 32, 64.0)
    with pytest.raises(PMError):
        pm.kdk_step(99, pm.new_particles(), pm.new_particles(), pm.new_particles())
    s = torch.zeros((1, 16 ** 3, 3), device="cuda")
    f = pm.pm_force(s)
    assert torch.max(torch.abs(f)).item() < 1e-5      # uniform lattice: no force


@pytest.mark.parametrize("n", [16, 32, 64, 128, 24])
def test_mesh_fft_against_numpy(n):
    # The library's 3D real FFT (own passes for powers of two, cuFFT else)
    # against numpy's FFT in FP64: forward, and inverse of the forward.
    from paper_2211_09958_gb300 import _pmgb
    import ctypes
    pm = _pm(8, n, 40.0, om=[0.3, 0.3], s8=[0.8, 0.8])
    rng = np.random.default_rng(n)
    x = rng.standard_normal((2, n, n, n)).astype(np.float32)
    xd = _cuda(x)
    spec = torch.empty((2, n, n, n // 2 + 1, 2), dtype=torch.float32, device="cuda")
    pm._call("pm_mesh_rfft", ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(spec.data_ptr()))
    got = _host(spec)
    got = got[..., 0] + 1j * got[..., 1]
    ref = np.fft.rfftn(x.astype(np.float64), axes=(1, 2, 3))
    scale = np.sqrt(n ** 3)           # |X| ~ sqrt(n^3) for unit white noise
    assert np.max(np.abs(got - ref)) < 2e-5 * scale * np.log2(n ** 3)
    back = torch.empty_like(xd)
    pm._call("pm_mesh_irfft", ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(back.data_ptr()))
    np.testing.assert_allclose(_host(back) / n ** 3, x, atol=2e-6 * np.log2(n ** 3))


def test_graph_replay_matches_direct_launches():
    # The captured graph (first call) and its replays on the same buffers give
    # the results of individual launches, up to the ordering of float atomics.
    n_p, n_m, box, steps = 16, 32, 64.0, 5
    pm = _pm(n_p, n_m, box, steps)
    s0, p0 = pm.init_lpt(_cuda(inputs.white_noise(n_p, 8))[None])
    s, p = s0.clone(), p0.clone()
    f = pm.new_particles()
    lam0 = _cuda(np.random.default_rng(9).standard_normal((n_p ** 3, 3)))[None]
    lam, mu = lam0.clone(), torch.zeros_like(p)

    def run():
        s.copy_(s0)
        p.copy_(p0)
        pm.integrate(s, p, f=f)
        fwd = s.clone()
        lam.copy_(lam0)
        mu.zero_()
        dom = pm.adjoint_integrate(s, p, f, lam, mu)
        return fwd, lam.clone(), dom[0]

    results = [run() for _ in range(3)]          # capture, then two replays
    pm.use_graphs(False)
    ref = run()
    for fwd, l, d in results:
        assert torch.max(torch.abs(fwd - ref[0])).item() < 1e-5 * box / n_p
        # relative L2, not the largest element: a particle whose reconstructed
        # position lands on the other side of a cell face in one of the runs
        # takes the other one-sided CIC slope there, a jump of its own lam
        assert ((l - ref[1]).norm() / ref[1].norm()).item() < 1e-3
        # dL/dOm sums per-step terms about 30 times larger than itself, so the
        # order of the atomics alone moves it by ~2e-3 of its value
        assert abs(d - ref[2]) < 5e-3 * abs(ref[2])
