"""Parity against the FP64 oracle at the mesh sizes the benchmark runs (256,
512 and 1024 points per side), in every launch variant the autotuner can
pick there.  The library's 3D transform is compiled per line length, and the
variants differ in their arithmetic order, so each size and variant is
compared with the oracle itself, not with another variant:

  * pm_mesh_rfft / pm_mesh_irfft against numpy's FP64 FFT, element by
    element, at n = 256 and 512, both x-pass pencil widths and several z-pass
    block sizes; bound 2e-5 sqrt(n^3) log2(n^3) (unit white noise has
    |X(k)| ~ sqrt(n^3); FP32 rounding grows with the transform depth);
  * at n = 1024, where a full FP64 reference does not fit a test: a sum of
    three separable fields f(x) g(y) h(z) whose values are short dyadic
    fractions, so the FP32 input is exactly separable and its 3D DFT is
    exactly the sum of products of 1D DFTs (numpy, FP64).  Compared on 2^20
    random modes and on whole lines along each axis.  The inverse is checked
    on a separable Hermitian spectrum with dyadic values, whose inverse is
    exactly n^3 a(x) b(y) c(z), on 2^20 random cells;
  * the PM force at 256^3 and 512^3 meshes (32^3 and 64^3 particles) through
    both force pipelines: the potential one (default) in each z-pass block
    size, and the gradient one under each x round trip (separate launches,
    fused, fused force only), both z-inverse stagings (per-thread loads, TMA)
    and both x-pass widths; within the small-mesh force bound 2e-5 of max |F|;
  * the reverse-time adjoint at 256^3 and 512^3 meshes (two KDK steps to
    a = 0.2, random cotangents) under the same variants and both z-forward
    stagings: the state after the forward steps within 1e-4 of the spacing; lam, mu
    within 1e-3 relative L2, dL/dOm of the dynamics within 1e-4 of the sum of
    its terms' magnitudes, as in the small-mesh parity tests.
"""

import ctypes
import functools

import numpy as np
import pytest
import torch

from oracle import pm as opm
from oracle.cosmology import Cosmology, kdk_coefficients_domega
from paper_2211_09958_gb300 import inputs

pytestmark = pytest.mark.gpu


def _pm(n_p, n_m, box, steps=2, **kw):
    from paper_2211_09958_gb300.pm import ParticleMesh
    return ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps, **kw)


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def _release(pm):
    pm.close()
    torch.cuda.empty_cache()


# ------------------------------------------------------------ transforms --

@pytest.mark.parametrize("n,fft_x,fft_z", [(256, 8, 128), (256, 16, 512), (512, 8, 256), (512, 16, 128)])
def test_mesh_fft_against_numpy_at_bench_sizes(n, fft_x, fft_z):
    pm = _pm(8, n, 64.0)
    pm.set_tuning(fft_x=fft_x, fft_z=fft_z)
    rng = np.random.default_rng(n + fft_x)
    x = rng.standard_normal((1, n, n, n)).astype(np.float32)
    xd = _cuda(x)
    spec = torch.empty((1, n, n, n // 2 + 1, 2), dtype=torch.float32, device="cuda")
    pm._call("pm_mesh_rfft", ctypes.c_void_p(xd.data_ptr()), ctypes.c_void_p(spec.data_ptr()))
    got = spec.cpu().numpy()
    got = got[..., 0].astype(np.float64) + 1j * got[..., 1]
    ref = np.fft.rfftn(x[0].astype(np.float64))
    bound = 2e-5 * np.sqrt(n ** 3) * np.log2(n ** 3)
    err = np.max(np.abs(got[0] - ref))
    del got, ref
    print(f"n={n} width={fft_x} z={fft_z}: forward max err {err / np.sqrt(n ** 3):.3e} sqrt(n^3)")
    assert err < bound, err / np.sqrt(n ** 3)
    back = torch.empty_like(xd)
    pm._call("pm_mesh_irfft", ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(back.data_ptr()))
    derr = (back / n ** 3 - xd).abs().max().item()
    assert derr < 2e-6 * np.log2(n ** 3), derr
    _release(pm)


def _dyadic(rng, size, bits=4):
    # values k / 2^bits, |k| <= 2^bits: products of three stay exact in FP32
    return rng.integers(-(1 << bits), (1 << bits) + 1, size).astype(np.float64) / (1 << bits)


def test_separable_fields_at_1024():
    n, terms = 1024, 3
    pm = _pm(8, n, 1000.0)
    rng = np.random.default_rng(1024)
    f = [[_dyadic(rng, n) for _ in range(3)] for _ in range(terms)]
    # forward: x = sum_r f_r(x) g_r(y) h_r(z), built on the device in FP32 (exact)
    x = torch.zeros((1, n, n, n), dtype=torch.float32, device="cuda")
    for fx, fy, fz in f:
        a, b, c = (torch.from_numpy(v.astype(np.float32)).cuda() for v in (fx, fy, fz))
        x[0] += a[:, None, None] * b[None, :, None] * c[None, None, :]
    spec = torch.empty((1, n, n, n // 2 + 1, 2), dtype=torch.float32, device="cuda")
    pm._call("pm_mesh_rfft", ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(spec.data_ptr()))
    dft = [(np.fft.fft(fx), np.fft.fft(fy), np.fft.rfft(fz)) for fx, fy, fz in f]
    rms = float(torch.sqrt(torch.mean(x.double() ** 2)).item())
    bound = 2e-5 * rms * np.sqrt(n ** 3) * np.log2(n ** 3)
    idx = [rng.integers(0, n, 1 << 20), rng.integers(0, n, 1 << 20), rng.integers(0, n // 2 + 1, 1 << 20)]
    lines = [(np.arange(n), np.full(n, 3), np.full(n, 5)), (np.full(n, 7), np.arange(n), np.full(n, 0)),
             (np.full(n // 2 + 1, 1), np.full(n // 2 + 1, n - 2), np.arange(n // 2 + 1))]
    for kx, ky, kz in [idx] + lines:
        ref = sum(F[kx] * G[ky] * H[kz] for F, G, H in dft)
        sel = spec[0, torch.from_numpy(kx).cuda(), torch.from_numpy(ky).cuda(), torch.from_numpy(kz).cuda()]
        got = sel.cpu().numpy().astype(np.float64)
        err = np.max(np.abs(got[:, 0] + 1j * got[:, 1] - ref))
        assert err < bound, (err / (rms * np.sqrt(n ** 3)), len(kx))
    del x
    # inverse: a separable Hermitian spectrum A(kx) B(ky) C(kz) with dyadic values
    spec.zero_()
    herm = []
    for _ in range(3):
        half = _dyadic(rng, n // 2 + 1) + 1j * _dyadic(rng, n // 2 + 1)
        half[0] = half[0].real
        half[n // 2] = half[n // 2].real
        herm.append(half)
    A = np.concatenate([herm[0], np.conj(herm[0][1:n // 2][::-1])])
    B = np.concatenate([herm[1], np.conj(herm[1][1:n // 2][::-1])])
    C = herm[2]
    for k, v in ((0, A), (1, B), (2, C)):
        assert np.allclose(np.fft.ifft(v).imag if k < 2 else 0.0, 0.0)
    dev = lambda v: torch.from_numpy(np.ascontiguousarray(v)).cuda()  # noqa: E731
    Ar, Ai, Br, Bi, Cr, Ci = (dev(t.astype(np.float32)) for v in (A, B, C) for t in (v.real, v.imag))
    # (A B) C with every product exact in FP32 (dyadic values of a few bits)
    ABr = Ar[:, None] * Br[None, :] - Ai[:, None] * Bi[None, :]
    ABi = Ar[:, None] * Bi[None, :] + Ai[:, None] * Br[None, :]
    spec[0, ..., 0] = ABr[:, :, None] * Cr[None, None, :] - ABi[:, :, None] * Ci[None, None, :]
    spec[0, ..., 1] = ABr[:, :, None] * Ci[None, None, :] + ABi[:, :, None] * Cr[None, None, :]
    real = torch.empty((1, n, n, n), dtype=torch.float32, device="cuda")
    pm._call("pm_mesh_irfft", ctypes.c_void_p(spec.data_ptr()), ctypes.c_void_p(real.data_ptr()))
    a = np.fft.ifft(A).real * n
    b = np.fft.ifft(B).real * n
    c = np.fft.irfft(C, n=n) * n
    cx, cy, cz = (rng.integers(0, n, 1 << 20) for _ in range(3))
    ref = a[cx] * b[cy] * c[cz]
    got = real[0, torch.from_numpy(cx).cuda(), torch.from_numpy(cy).cuda(), torch.from_numpy(cz).cuda()]
    got = got.cpu().numpy().astype(np.float64)
    scale = np.sqrt(np.mean(np.abs(A) ** 2) * np.mean(np.abs(B) ** 2) * np.mean(np.abs(C) ** 2) * n ** 3)
    err = np.max(np.abs(got - ref))
    print(f"1024: inverse max err {err / scale:.3e} of rms")
    assert err < 2e-5 * scale * np.log2(n ** 3), err / scale
    _release(pm)


# ---------------------------------------------------------------- force --

@functools.lru_cache(maxsize=None)
def _oracle_force(n_p, n_m, box):
    s = inputs.random_displacements(n_p, box, seed=n_p + n_m, scale=0.6)
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8), n_steps=2)
    return s, opm.force(s.astype(np.float64), st)


# Launch variants per mesh: the potential pipeline (default; its z passes in
# each block size) and the gradient pipeline under each x round trip, z
# inverse staging (per-thread loads or TMA) and x-pass width.
VARIANTS = [dict(pipeline=2, fft_z=256), dict(pipeline=2, fft_z=128, z_fwd_staging=2),
            dict(pipeline=2, fft_z=512), dict(pipeline=1, x_round=1, z_staging=2, fft_x=8),
            dict(pipeline=1, x_round=2, z_staging=1, fft_x=16), dict(pipeline=1, x_round=3, z_staging=2, fft_x=16)]
MESHES = [(32, 256, 128.0), (64, 512, 256.0)]


def _vid(v):
    return "-".join(f"{k}{x}" for k, x in v.items())


@pytest.mark.parametrize("n_p,n_m,box", MESHES)
@pytest.mark.parametrize("tuning", VARIANTS, ids=_vid)
def test_force_parity_at_bench_meshes(n_p, n_m, box, tuning):
    s, ref = _oracle_force(n_p, n_m, box)
    pm = _pm(n_p, n_m, box)
    pm.set_tuning(**tuning)
    f = _host(pm.pm_force(_cuda(s)[None]))[0]
    err = np.max(np.abs(f - ref)) / np.max(np.abs(ref))
    print(f"force {n_p}/{n_m} {_vid(tuning)}: {err:.3e} of max |F|")
    assert err < 2e-5, err
    _release(pm)


# -------------------------------------------------------------- adjoint --

# Two KDK steps from the 2LPT start at a = 1/64 to a = 0.2.  With 8 or 4 mesh
# cells per particle spacing the painted density is spiky, and two steps
# across the whole history (a = 1/64 -> 1) amplify FP32-level force
# differences a thousandfold: FP64 oracle runs with the force perturbed by
# 4e-7 of max |F| then end 1e-4 of the spacing apart.  Up to a = 0.2 the same
# perturbation moves the final state by 6e-7 of the spacing, so the bounds
# below test the transforms, not the conditioning of the trajectory.
A_FINAL = 0.2


@functools.lru_cache(maxsize=None)
def _oracle_adjoint(n_p, n_m, box, steps):
    st = opm.Setup(n_p, n_m, box, Cosmology(0.3, 0.8), a_final=A_FINAL, n_steps=steps)
    noise = inputs.white_noise(n_p, n_m + 1)
    rng = np.random.default_rng(n_m)
    lam0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    mu0 = rng.standard_normal((n_p ** 3, 3)).astype(np.float32)
    rs, rp, rf = opm.simulate(noise.astype(np.float64), st)
    _, _, olam, omu, grads = opm.adjoint_integrate(rs, rp, rf, lam0.astype(np.float64), mu0.astype(np.float64), st)
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps)
    cond = abs(grads["omega_m_direct"]) + sum(abs(np.dot(grads[k], d[k])) for k in ("K_a", "Dr", "K_b"))
    return noise, lam0, mu0, rs, olam, omu, opm.dynamics_domega(grads, st), cond


@pytest.mark.parametrize("n_p,n_m,box", MESHES)
@pytest.mark.parametrize("tuning", VARIANTS, ids=_vid)
def test_adjoint_parity_at_bench_meshes(n_p, n_m, box, tuning):
    steps = 2
    noise, lam0, mu0, rs, olam, omu, o_dom, cond = _oracle_adjoint(n_p, n_m, box, steps)
    from paper_2211_09958_gb300.pm import ParticleMesh
    pm = ParticleMesh(n_p, n_m, box, 0.3, 0.8, steps, a_final=A_FINAL)
    pm.set_tuning(**tuning)
    s, p = pm.init_lpt(_cuda(noise)[None])
    f = pm.integrate(s, p)
    ds = np.max(np.abs(_host(s)[0] - rs)) / (box / n_p)
    assert ds < 1e-4, ds
    lam, mu = _cuda(lam0)[None], _cuda(mu0)[None]
    dom = pm.adjoint_integrate(s, p, f, lam, mu)
    rel = [np.linalg.norm(_host(t)[0] - r) / np.linalg.norm(r) for t, r in ((lam, olam), (mu, omu))]
    print(f"adjoint {n_p}/{n_m} {_vid(tuning)}: "
          f"state {ds:.2e}, lam {rel[0]:.2e}, mu {rel[1]:.2e}, dOm {abs(dom[0] - o_dom) / cond:.2e} of terms")
    assert max(rel) < 1e-3, rel
    assert abs(dom[0] - o_dom) < 1e-4 * cond, (dom[0], o_dom, cond)
    _release(pm)
