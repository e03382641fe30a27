"""Pins of the oracle's CIC assignment/interpolation, spectral Poisson force,
its vector-Jacobian product and the power-spectrum estimator."""

import itertools

import numpy as np
import pytest

from oracle import pm
from oracle.pm import Setup
from paper_2211_09958_gb300 import inputs


def _tent_mesh(x, n, cell):
    # Brute force: W is the product of periodic tent functions max(0, 1 - |d|/h).
    c = np.arange(n) * cell
    box = n * cell
    mesh = np.zeros((n, n, n))
    for xi in x:
        w = []
        for d in range(3):
            dist = (xi[d] - c + 0.5 * box) % box - 0.5 * box
            w.append(np.maximum(0.0, 1.0 - np.abs(dist) / cell))
        mesh += w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
    return mesh


def _special_positions(rng, n, cell, count):
    x = rng.uniform(-2 * n * cell, 3 * n * cell, (count, 3))     # outside the box too
    x[0] = [0.0, 0.0, 0.0]                                       # on a node
    x[1] = [0.5 * cell, 0.5 * cell, 0.5 * cell]                  # cell centre
    x[2] = [n * cell, 3 * cell, -cell]                           # nodes at the wrap
    x[3] = [2.0 * cell, 2.5 * cell, (n - 0.25) * cell]           # on a face
    return x


def test_cic_paint_equals_tent_definition():
    rng = np.random.default_rng(0)
    n, cell = 6, 1.7
    x = _special_positions(rng, n, cell, 40)
    np.testing.assert_allclose(pm.cic_paint(x, n, cell), _tent_mesh(x, n, cell), atol=1e-12)


def test_cic_node_and_centre():
    n, cell = 8, 1.0
    m = pm.cic_paint(np.array([[3.0, 4.0, 5.0]]), n, cell)
    assert m[3, 4, 5] == 1.0 and m.sum() == 1.0
    m = pm.cic_paint(np.array([[3.5, 4.5, 7.5]]), n, cell)
    np.testing.assert_allclose(m[3:5, 4:6, [7, 0]], np.full((2, 2, 2), 0.125), atol=1e-15)


def test_cic_mass_conservation():
    rng = np.random.default_rng(1)
    st = Setup(16, 32, 100.0)
    s = rng.normal(0, 5.0, (16 ** 3, 3))
    rho = pm.density(s, st)
    assert abs(np.sum(rho + 1.0) - 32 ** 3) < 1e-8


def test_cic_read_equals_tent_definition():
    rng = np.random.default_rng(2)
    n, cell = 6, 0.9
    mesh = rng.standard_normal((n, n, n))
    x = _special_positions(rng, n, cell, 30)
    ref = np.array([np.sum(_tent_mesh(xi[None], n, cell) * mesh) for xi in x])
    np.testing.assert_allclose(pm.cic_read(x, mesh, cell), ref, atol=1e-12)


def test_cic_read_grad_matches_finite_difference():
    rng = np.random.default_rng(3)
    n, cell = 8, 1.3
    mesh = rng.standard_normal((n, n, n))
    x = rng.uniform(0, n * cell, (50, 3))
    g = pm.cic_read_grad(x, mesh, cell)
    eps = 1e-7
    for d in range(3):
        dx = np.zeros(3)
        dx[d] = eps
        fd = (pm.cic_read(x + dx, mesh, cell) - pm.cic_read(x - dx, mesh, cell)) / (2 * eps)
        np.testing.assert_allclose(g[:, d], fd, rtol=1e-6, atol=1e-6)


@pytest.mark.parametrize("n_p,n_m,solver", [(6, 12, 0), (6, 9, 0), (6, 12, 8)])
def test_density_vjp_matches_finite_difference(n_p, n_m, solver):
    # <g, delta(s)> is piecewise linear (CIC) or smooth (TSC) in s: central
    # differences with a small step give its directional derivative, which
    # the VJP must reproduce (a missing alpha or a wrong sign fails).
    rng = np.random.default_rng(11)
    st = Setup(n_p, n_m, 2.0 * n_p, solver=solver)
    s = rng.standard_normal((n_p ** 3, 3)) * 0.4 * st.spacing
    g = rng.standard_normal((n_m, n_m, n_m))
    vjp = pm.density_vjp(s, g, st)
    eps = 1e-7
    for _ in range(3):
        v = rng.standard_normal(s.shape)
        fd = (np.sum(g * pm.density(s + eps * v, st)) - np.sum(g * pm.density(s - eps * v, st))) / (2 * eps)
        assert abs(fd - np.sum(vjp * v)) < 1e-6 * np.abs(vjp * v).sum(), (fd, np.sum(vjp * v))


@pytest.mark.parametrize("n", [4, 6, 8])
def test_force_mesh_against_direct_dft(n):
    # Green's function x gradient via explicit O(N^6) complex DFT sums on the
    # full k grid, with the same k = 0 and Nyquist (index n/2) zeroing; the
    # gradient is the 4-point central difference, here applied in real space
    # to the DFT potential (so this also pins its Fourier multiplier).
    rng = np.random.default_rng(n)
    box, om = 10.0, 0.3
    st = Setup(n, n, box, pm.Cosmology(om))
    x = rng.uniform(0, box, (3 * n, 3))
    h = box / n
    rho = st.alpha * pm.cic_paint(x, n, h) - 1.0
    idx = np.array(list(itertools.product(range(n), repeat=3)))
    nvec = np.where(idx < n // 2, idx, idx - n)                  # n in [-N/2, N/2)
    kvec = 2 * np.pi / box * nvec
    cpos = idx * h
    dft = np.exp(-1j * kvec @ cpos.T)                            # [k, c]
    rho_k = dft @ rho.ravel()
    k2 = np.sum(kvec ** 2, axis=1)
    got = pm.force_meshes(x, st)
    green = np.where(k2 > 0, -1.5 * om / np.where(k2 > 0, k2, 1.0), 0.0)
    for j in range(3):
        # potential with the Nyquist plane of axis j removed, then
        # F_j = -(8 (phi(c+e) - phi(c-e)) - (phi(c+2e) - phi(c-2e))) / (12 h)
        keep = idx[:, j] != n // 2
        phi = ((np.conj(dft).T @ (np.where(keep, green, 0.0) * rho_k)) / n ** 3).real.reshape(n, n, n)
        sh = lambda d: np.roll(phi, -d, axis=j)
        fj = -(8.0 * (sh(1) - sh(-1)) - (sh(2) - sh(-2))) / (12.0 * h)
        np.testing.assert_allclose(got[j], fj, atol=1e-12)


def _force_at(x, setup, mass_x):
    # force at x of the particles mass_x, painted with the same alpha
    rho = setup.alpha * pm.cic_paint(mass_x, setup.n_m, setup.cell) - 1.0
    mult = pm.gradient_green_multipliers(setup.n_m, setup.box, setup.cosmo.omega_m)
    meshes = [pm.irfftn(m * pm.rfftn(rho), setup.n_m) for m in mult]
    return np.stack([pm.cic_read(x, mm, setup.cell) for mm in meshes], axis=1)


def test_gravity_attracts_and_newton_third_law():
    st = Setup(4, 16, 16.0)
    a = np.array([[5.3, 7.1, 8.2]])
    b = np.array([[9.6, 8.0, 6.9]])
    f_ab = _force_at(a, st, b)          # on a due to b
    f_ba = _force_at(b, st, a)
    assert np.dot(f_ab[0], (b - a)[0]) > 0          # attractive
    np.testing.assert_allclose(f_ab, -f_ba, atol=1e-13)
    np.testing.assert_allclose(_force_at(a, st, a), 0.0, atol=1e-13)   # no self force


def test_total_force_vanishes():
    rng = np.random.default_rng(4)
    st = Setup(8, 16, 50.0)
    s = rng.normal(0, 3.0, (8 ** 3, 3))
    f = pm.force(s, st)
    assert np.max(np.abs(f.sum(0))) < 1e-10 * np.abs(f).sum()


@pytest.mark.parametrize("ratio", [1, 2, 4])
def test_plane_wave_force_converges_at_every_mesh_ratio(ratio):
    # F -> 3/2 Om s for a small longitudinal plane wave on the particle
    # lattice, with an error that falls as k^2 (halving k quarters it) at
    # every mesh-to-lattice ratio.  An exact spectral gradient i k fails
    # this for ratio >= 2 (error linear in k, +6 % at n_m = 2 n_p, k =
    # k_Nyquist / 8).
    errs = []
    for n_p in (16, 32):
        box = 8.0 * n_p
        st = Setup(n_p, ratio * n_p, box, pm.Cosmology(0.3))
        q = pm.lattice(n_p, box, ratio * n_p)
        k = 2 * np.pi / box
        s = np.zeros_like(q)
        s[:, 0] = 1e-4 * np.sin(k * q[:, 0])
        f = pm.force(s, st)[:, 0]
        errs.append(abs(f @ s[:, 0] / (s[:, 0] @ s[:, 0]) / (1.5 * 0.3) - 1.0))
    assert errs[0] < 3e-2 and errs[1] < errs[0] / 3.0, errs


def test_linear_force_prefactor():
    # A small longitudinal plane-wave displacement gives F -> 3/2 Om s as the
    # mode becomes well resolved; the CIC/mesh correction falls as (k h)^2.
    # (One particle per cell, so no lattice aliasing enters.)
    errs = []
    for n_m in (32, 64):
        st = Setup(n_m, n_m, 100.0, pm.Cosmology(0.3))
        q = pm.lattice(n_m, 100.0, n_m)
        k = 2 * np.pi / 100.0
        s = np.zeros_like(q)
        s[:, 0] = 1e-4 * np.sin(k * q[:, 0])
        f = pm.force(s, st)
        errs.append(np.max(np.abs(f[:, 0] - 1.5 * 0.3 * s[:, 0])) / np.max(np.abs(1.5 * 0.3 * s[:, 0])))
        assert np.max(np.abs(f[:, 1:])) < 1e-12
    assert errs[0] < 1e-2 and errs[1] < errs[0] / 3


def test_force_vjp_matches_finite_difference():
    rng = np.random.default_rng(5)
    st = Setup(4, 8, 10.0)
    s = rng.normal(0, 0.6, (64, 3))
    v = rng.standard_normal((64, 3))
    g = pm.force_vjp(s, v, st)
    eps = 1e-6
    for _ in range(6):
        d = rng.standard_normal((64, 3))
        fd = (np.sum(v * pm.force(s + eps * d, st)) - np.sum(v * pm.force(s - eps * d, st))) / (2 * eps)
        assert abs(fd - np.sum(g * d)) < 1e-6 * max(1.0, abs(fd))


def test_power_of_cosine_mode_closed_form():
    n, box, amp, m = 16, 40.0, 0.7, 3
    c = np.arange(n) * box / n
    delta = amp * np.cos(2 * np.pi * m / box * c)[:, None, None] * np.ones((n, n, n))
    k_mean, p, nm = pm.power_of_mesh(delta, box)
    expect = np.zeros(n // 2)
    expect[m - 1] = box ** 3 * amp ** 2 / (2 * nm[m - 1])
    np.testing.assert_allclose(p, expect, atol=1e-12 * box ** 3)


def test_power_mode_counts_brute_force():
    n, box = 12, 30.0
    _, _, nm = pm.power_of_mesh(np.zeros((n, n, n)), box)
    rng_n = np.arange(-n // 2, n // 2)
    nv = np.array(list(itertools.product(rng_n, repeat=3)))
    kk = np.sqrt(np.sum(nv ** 2, axis=1))
    b = np.floor(kk - 0.5).astype(int)
    ok = (kk > 0) & (b < n // 2)
    np.testing.assert_array_equal(nm, np.bincount(b[ok], minlength=n // 2))


def test_power_of_white_noise_is_flat():
    n, box = 32, 64.0
    rng = np.random.default_rng(6)
    ratios = []
    for _ in range(4):
        _, p, nm = pm.power_of_mesh(rng.standard_normal((n, n, n)), box)
        ratios.append(p[nm > 200] / (box ** 3 / n ** 3))
    assert abs(np.mean(ratios) - 1.0) < 0.02


def test_spectral_gradient_flag_against_direct_dft():
    # solver flag 1: F_j(k) = i k_j (3/2) Om delta / k^2 (Nyquist index of axis
    # j zeroed), checked by explicit O(N^6) DFT sums on a 6^3 mesh
    n, box, om = 6, 10.0, 0.3
    rng = np.random.default_rng(9)
    st = Setup(n, n, box, pm.Cosmology(om), solver=pm.SPECTRAL_GRADIENT)
    x = rng.uniform(0, box, (3 * n, 3))
    h = box / n
    rho = st.alpha * pm.cic_paint(x, n, h) - 1.0
    idx = np.array(list(itertools.product(range(n), repeat=3)))
    nvec = np.where(idx < n // 2, idx, idx - n)
    kvec = 2 * np.pi / box * nvec
    dft = np.exp(-1j * kvec @ (idx * h).T)
    rho_k = dft @ rho.ravel()
    k2 = np.sum(kvec ** 2, axis=1)
    got = pm.force_meshes(x, st)
    for j in range(3):
        mult = np.where((k2 > 0) & (idx[:, j] != n // 2),
                        1j * kvec[:, j] * 1.5 * om / np.where(k2 > 0, k2, 1.0), 0.0)
        fj = (np.conj(dft).T @ (mult * rho_k)) / n ** 3
        assert np.max(np.abs(fj.imag)) < 1e-12
        np.testing.assert_allclose(got[j].ravel(), fj.real, atol=1e-12)


@pytest.mark.parametrize("solver", [pm.DECONVOLVE, pm.DECONVOLVE | pm.SPECTRAL_GRADIENT])
def test_deconvolution_flattens_the_linear_response(solver):
    # One particle per cell: dividing by the paint and read CIC windows takes
    # out their (k h)^2 suppression of a long plane wave, so F -> 3/2 Om s is
    # approached much faster than without (error 5x smaller at k = k_Ny / 8
    # and falling faster than k^2).
    def err(n_p, flags):
        box = 8.0 * n_p
        st = Setup(n_p, n_p, box, pm.Cosmology(0.3), solver=flags)
        q = pm.lattice(n_p, box, n_p)
        s = np.zeros_like(q)
        s[:, 0] = 1e-4 * np.sin(2 * np.pi * q[:, 0] / box)
        f = pm.force(s, st)[:, 0]
        return abs(f @ s[:, 0] / (s[:, 0] @ s[:, 0]) / (1.5 * 0.3) - 1.0)
    plain16 = err(16, solver & ~pm.DECONVOLVE)
    dec16, dec32 = err(16, solver), err(32, solver)
    assert dec16 < plain16 / 5 and dec32 < dec16 / 5, (plain16, dec16, dec32)


# ------------------------------------------------------------------- TSC --

def _bspline2(r):
    # quadratic B-spline of unit width (the TSC kernel), r in cells
    a = np.abs(r)
    return np.where(a < 0.5, 0.75 - a * a, np.where(a < 1.5, 0.5 * (1.5 - a) ** 2, 0.0))


def _tsc_mesh(x, n, cell):
    c = np.arange(n) * cell
    box = n * cell
    mesh = np.zeros((n, n, n))
    for xi in x:
        w = [_bspline2(((xi[d] - c + 0.5 * box) % box - 0.5 * box) / cell) for d in range(3)]
        mesh += w[0][:, None, None] * w[1][None, :, None] * w[2][None, None, :]
    return mesh


def test_tsc_paint_and_read_equal_the_bspline_definition():
    rng = np.random.default_rng(10)
    n, cell = 6, 1.3
    x = _special_positions(rng, n, cell, 40)
    x[4] = [0.5 * cell, 1.5 * cell, 2.5 * cell]                 # half-node ties
    np.testing.assert_allclose(pm.cic_paint(x, n, cell, order=3), _tsc_mesh(x, n, cell), atol=1e-12)
    mesh = rng.standard_normal((n, n, n))
    ref = np.array([np.sum(_tsc_mesh(xi[None], n, cell) * mesh) for xi in x])
    np.testing.assert_allclose(pm.cic_read(x, mesh, cell, order=3), ref, atol=1e-12)


def test_tsc_mass_conservation_and_gradient():
    rng = np.random.default_rng(11)
    st = Setup(8, 16, 40.0, solver=pm.TSC)
    s = rng.normal(0, 3.0, (8 ** 3, 3))
    assert abs(np.sum(pm.density(s, st) + 1.0) - 16 ** 3) < 1e-9
    n, cell = 8, 1.1
    mesh = rng.standard_normal((n, n, n))
    x = rng.uniform(0, n * cell, (50, 3))
    g = pm.cic_read_grad(x, mesh, cell, order=3)
    eps = 1e-6
    for d in range(3):
        dx = np.zeros(3)
        dx[d] = eps
        fd = (pm.cic_read(x + dx, mesh, cell, 3) - pm.cic_read(x - dx, mesh, cell, 3)) / (2 * eps)
        np.testing.assert_allclose(g[:, d], fd, rtol=1e-6, atol=1e-6)


def test_tsc_force_vjp_matches_finite_difference():
    rng = np.random.default_rng(12)
    st = Setup(4, 8, 10.0, solver=pm.TSC)
    s = rng.normal(0, 0.6, (64, 3))
    v = rng.standard_normal((64, 3))
    g = pm.force_vjp(s, v, st)
    eps = 1e-6
    for _ in range(6):
        d = rng.standard_normal((64, 3))
        fd = (np.sum(v * pm.force(s + eps * d, st)) - np.sum(v * pm.force(s - eps * d, st))) / (2 * eps)
        assert abs(fd - np.sum(g * d)) < 1e-6 * max(1.0, abs(fd))


@pytest.mark.parametrize("ratio", [1, 2])
def test_tsc_linear_force_converges(ratio):
    # the plane-wave force F -> 3/2 Om s with an O(k^2) error, TSC at mesh
    # ratios 1 and 2
    errs = []
    for n_p in (16, 32):
        box = 8.0 * n_p
        st = Setup(n_p, ratio * n_p, box, pm.Cosmology(0.3), solver=pm.TSC)
        q = pm.lattice(n_p, box, ratio * n_p)
        s = np.zeros_like(q)
        s[:, 0] = 1e-4 * np.sin(2 * np.pi * q[:, 0] / box)
        f = pm.force(s, st)[:, 0]
        errs.append(abs(f @ s[:, 0] / (s[:, 0] @ s[:, 0]) / (1.5 * 0.3) - 1.0))
    assert errs[0] < 5e-2 and errs[1] < errs[0] / 3.0, errs


# ------------------------------------------- sampled and reduced cases ----

@pytest.mark.parametrize("n_p,n_m,box,solver", [(16, 32, 64.0, 0), (16, 16, 48.0, 0), (12, 18, 40.0, 0),
                                                (16, 32, 64.0, 8)])
def test_density_at_sampled_cells_matches_the_full_mesh(n_p, n_m, box, solver):
    st = pm.Setup(n_p, n_m, box, solver=solver)
    s = inputs.random_displacements(n_p, box, seed=31, scale=0.8).astype(np.float64)
    full = pm.density(s, st).ravel()
    cells = np.random.default_rng(3).integers(0, n_m ** 3, 40)
    got = pm.density_at(cells, s, st, np.abs(s).max())
    np.testing.assert_allclose(got, full[cells], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n_p,n_m,box", [(24, 24, 48.0), (12, 24, 48.0), (6, 6, 12.0)])
def test_density_at_reaches_far_displaced_particles(n_p, n_m, box):
    # One particle thrown several cells from its site (and, on the 6^3
    # lattice, a window wider than the lattice): the cells its CIC corners
    # land on must still see it.
    st = pm.Setup(n_p, n_m, box)
    h = st.cell
    s = inputs.random_displacements(n_p, box, seed=5, scale=0.2).astype(np.float64)
    i = (3 * n_p + 3) * n_p + 4
    s[i] = [5.9 * h, -5.9 * h, 0.3 * h]                 # corners 6 and 7 cells from the site
    cells = np.array([flat[0] for flat, _, _ in pm.cic_corners(pm.positions(s, st)[i][None], n_m, h)])
    full = pm.density(s, st).ravel()
    got = pm.density_at(cells, s, st, np.abs(s).max())
    np.testing.assert_allclose(got, full[cells], rtol=0, atol=1e-12)


@pytest.mark.parametrize("n", [8, 12])
def test_every_spectral_multiplier_gives_a_real_field(n):
    # irfftn returns a real field for any input, so a multiplier that breaks
    # Hermitian symmetry would be silently projected.  On the rfft grid the
    # symmetry M(-k) = conj M(k) constrains the n_z = 0 and n_z = n/2 planes:
    # check it there for the force multipliers (every solver variant) and the
    # 2LPT and linear-field multipliers.
    from oracle import lpt
    box = 3.0 * n
    mults = []
    for solver in (0, 1, 2, 8, 3):
        mults += pm.gradient_green_multipliers(n, box, 0.3, solver)
    s1, phi, s2 = lpt.lpt_multipliers(n, box)
    mults += s1 + phi + s2 + [lpt.linear_multiplier(Setup(n, n, box))]
    neg = (-np.arange(n)) % n
    for m in mults:
        m = np.broadcast_to(m, (n, n, n // 2 + 1))
        for z in (0, n // 2):
            plane = m[:, :, z]
            np.testing.assert_array_equal(plane[np.ix_(neg, neg)], np.conj(plane))


@pytest.mark.parametrize("n_p,n_m,solver", [(16, 32, 0), (16, 16, 0), (16, 32, 1), (16, 32, 2)])
def test_plane_wave_force_reduces_to_one_dimension(n_p, n_m, solver):
    box = 64.0
    st = pm.Setup(n_p, n_m, box, solver=solver)
    i = np.arange(n_p)
    sx = 0.4 * (box / n_p) * np.sin(2 * np.pi * 3 * (i + 0.25) / n_p) + 0.1 * (box / n_p) * np.cos(2 * np.pi * 5 * i / n_p)
    s = np.zeros((n_p, n_p, n_p, 3))
    s[..., 0] = sx[:, None, None]
    f = pm.force(s.reshape(-1, 3), st).reshape(n_p, n_p, n_p, 3)
    fx = pm.force_uniform_yz(sx, st)
    scale = np.abs(fx).max()
    assert scale > 0
    np.testing.assert_allclose(f[..., 0], np.broadcast_to(fx[:, None, None], f.shape[:3]), rtol=0, atol=1e-12 * scale)
    assert np.abs(f[..., 1:]).max() < 1e-12 * scale


def test_four_point_stencil_is_the_gradient_symbol():
    # The fused x round trip builds the adjoint's psi from one forward
    # transform: the periodic stencil S f = [8 (f(x+h) - f(x-h)) - (f(x+2h) - f(x-2h))] / 12h
    # has the Fourier symbol i D(k) of the gradient reading, so
    # -i g sum_j D_j u_j(k) = -g FFT_x(S_x u_x + i (D_y u_y + D_z u_z)).
    n, box = 64, 128.0
    h = box / n
    rng = np.random.default_rng(11)
    ux, uy, uz = (rng.standard_normal(n) + 1j * rng.standard_normal(n) for _ in range(3))
    k = 2 * np.pi / box * np.fft.fftfreq(n, 1.0 / n)
    dx = pm.gradient_operator(k, h)
    dy, dz = pm.gradient_operator(2 * np.pi / box * 5, h), pm.gradient_operator(2 * np.pi / box * -7, h)
    stencil = (8 * (np.roll(ux, -1) - np.roll(ux, 1)) - (np.roll(ux, -2) - np.roll(ux, 2))) / (12 * h)
    np.testing.assert_allclose(np.fft.fft(stencil), 1j * dx * np.fft.fft(ux), rtol=0, atol=1e-12 * np.abs(np.fft.fft(ux)).max())
    g = rng.uniform(0.5, 2.0, n)                        # any real multiplier (Green's function, windows)
    lhs = -1j * g * (dx * np.fft.fft(ux) + dy * np.fft.fft(uy) + dz * np.fft.fft(uz))
    rhs = -g * np.fft.fft(stencil + 1j * (dy * uy + dz * uz))
    np.testing.assert_allclose(rhs, lhs, rtol=0, atol=1e-12 * np.abs(lhs).max())
    assert abs(pm.gradient_operator(np.pi / h, h)) < 1e-12   # the symbol vanishes at the Nyquist index
