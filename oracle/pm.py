"""Particle-mesh force, KDK integration and its discrete adjoint, FP64
(test infrastructure only).

Paper: pmwd is a cosmological particle-mesh (PM) simulation (Summary) whose
gradients come from the adjoint method with reverse time integration
(Summary; Statement of Need) and follow the same discrete trajectory as the
forward integrator (Statement of Need: the adjoint of the discretised
equations, not a discretised continuous adjoint).  The paper prints no
equations; the readings below are the standard comoving PM ones.
[reading]

Geometry: box L, n_m^3 mesh with nodes at c h, h = L / n_m, periodic;
n_p^3 particles on the lattice q = i L / n_p + h / 2, i.e. half a mesh cell
off the nodes [reading]: the unperturbed lattice then paints an exactly
uniform mesh and small displacements sit away from the CIC kinks, so the
linear response is symmetric.  Particle state:
displacement s = x - q and momentum p = a^3 E dx/da.

  CIC weights   W(x - c) = prod_d w(u_d - c_d), u = x / h, i0 = floor(u),
                f = u - i0, w = 1 - f at i0 and f at i0 + 1.
  density       rho(c) = alpha sum_i W(x_i - c) - 1, alpha = (n_m / n_p)^3
  force         F_j(k) = i D_j(k) (3/2) Om rho(k) / k^2, zero at k = 0 and
                where n_j is the Nyquist index; F_j(c) = IDFT; F_i = sum_c W F(c)
  solver flags  SPECTRAL_GRADIENT (1): D_j = k_j instead (exact spectral
                gradient, zero at the Nyquist index); DECONVOLVE (2): the Green
                function divided by the assignment window of paint and read,
                prod_j sinc^(2 p)(k_j h / 2) (p = 2 CIC, 3 TSC); LOG_A (4):
                steps uniform in ln a; TSC (8): triangular-shaped-cloud
                assignment (quadratic B-spline over 3 nodes per axis:
                j = round(u), d = u - j, weights 1/2 (1/2 - d)^2, 3/4 - d^2,
                1/2 (1/2 + d)^2 at j - 1, j, j + 1) in paint and read
  gradient      D_j(k) = (8 sin(k_j h) - sin(2 k_j h)) / (6 h), the 4-point
                central difference in Fourier space [reading]: it vanishes
                smoothly at the Nyquist frequency.  With a mesh finer than the
                particle lattice (n_m > n_p) the perturbed lattice puts
                density at the lattice harmonics near the mesh Nyquist; the
                exact spectral gradient i k_j jumps there and makes the
                linear force on a long plane wave too strong by an amount
                linear in k (+6 % at n_m = 2 n_p, k = k_Nyquist(particles)/8),
                while D_j keeps the error O(k^2) at every mesh ratio
  step n        p <- p + K_a F(s);  s <- s + Dr p;  p <- p + K_b F(s)

Every routine below is written as the definition it implements; FFTs are
library calls (scipy.fft), everything else is plain numpy.
"""

import itertools
from dataclasses import dataclass, field

import numpy as np
import scipy.fft as sfft

from .cosmology import Cosmology, kdk_coefficients, kdk_coefficients_domega

_WORKERS = -1   # scipy.fft threads: all host cores


@dataclass(frozen=True)
class Setup:
    n_p: int
    n_m: int
    box: float
    cosmo: Cosmology = field(default_factory=Cosmology)
    a_init: float = 1.0 / 64
    a_final: float = 1.0
    n_steps: int = 10
    solver: int = 0                   # bit mask of the solver flags below

    @property
    def order(self):
        """Assignment order: 2 (CIC) or 3 (TSC, solver flag 8)."""
        return 3 if self.solver & 8 else 2

    @property
    def cell(self):
        return self.box / self.n_m

    @property
    def spacing(self):
        return self.box / self.n_p

    @property
    def alpha(self):
        return (self.n_m / self.n_p) ** 3


# ------------------------------------------------------------ geometry ----

def lattice(n_p, box, n_m):
    """Lagrangian positions q = i L / n_p + h / 2, lattice order (x slowest,
    z fastest)."""
    g = np.arange(n_p, dtype=np.float64) * (box / n_p) + 0.5 * box / n_m
    qx, qy, qz = np.meshgrid(g, g, g, indexing="ij")
    return np.stack([qx.ravel(), qy.ravel(), qz.ravel()], axis=1)


def positions(s, setup):
    return lattice(setup.n_p, setup.box, setup.n_m) + s


def rfft_wavenumbers(n, box):
    """k_x, k_y, k_z broadcastable over an (n, n, n//2+1) rfft grid and the
    Nyquist masks of each axis (index n//2 on every axis)."""
    kf = 2.0 * np.pi / box
    full = np.fft.fftfreq(n, 1.0 / n)
    half = np.arange(n // 2 + 1, dtype=np.float64)
    kx = (kf * full)[:, None, None]
    ky = (kf * full)[None, :, None]
    kz = (kf * half)[None, None, :]
    ix = np.arange(n)
    iz = np.arange(n // 2 + 1)
    nyq = ((ix == n // 2)[:, None, None], (ix == n // 2)[None, :, None],
           (iz == n // 2)[None, None, :])
    return (kx, ky, kz), nyq


def rfftn(a):
    return sfft.rfftn(a, workers=_WORKERS)


def irfftn(a, n):
    return sfft.irfftn(a, s=(n, n, n), workers=_WORKERS)


# ---------------------------------------------------------------- CIC ----

def _axis_weights(u, order, cell):
    """First node, then per node k = 0 .. order-1: weight and d weight / dx,
    per axis (arrays shaped like u)."""
    if order == 2:                    # CIC, floor convention
        base = np.floor(u)
        f = u - base
        return base.astype(np.int64), [(1.0 - f, -np.ones_like(f) / cell), (f, np.ones_like(f) / cell)]
    j = np.floor(u + 0.5)             # TSC: nearest node j, d in [-1/2, 1/2)
    d = u - j
    return (j - 1).astype(np.int64), [(0.5 * (0.5 - d) ** 2, -(0.5 - d) / cell),
                                      (0.75 - d * d, -2.0 * d / cell),
                                      (0.5 * (0.5 + d) ** 2, (0.5 + d) / cell)]


def cic_corners(x, n_m, cell, order=2):
    """For each of the order^3 corners: flat mesh index, weight W and dW/dx
    (N,3).  CIC (order 2) dW/dx uses the one-sided slopes -1/h, +1/h of the
    floor convention; TSC (order 3) weights are C^1."""
    u = x / cell
    base, ax = _axis_weights(u, order, cell)
    out = []
    for off in itertools.product(range(order), repeat=3):
        idx = (base + np.array(off)) % n_m
        flat = (idx[:, 0] * n_m + idx[:, 1]) * n_m + idx[:, 2]
        w1 = np.stack([ax[off[d]][0][:, d] for d in range(3)], axis=1)
        dw1 = [ax[off[d]][1][:, d] for d in range(3)]
        w = w1[:, 0] * w1[:, 1] * w1[:, 2]
        grad = np.stack([dw1[0] * w1[:, 1] * w1[:, 2],
                         w1[:, 0] * dw1[1] * w1[:, 2],
                         w1[:, 0] * w1[:, 1] * dw1[2]], axis=1)
        out.append((flat, w, grad))
    return out


def cic_paint(x, n_m, cell, weights=None, order=2):
    """sum_i weights_i W(x_i - c) on the n_m^3 mesh (CIC, or TSC for order 3)."""
    mesh = np.zeros(n_m ** 3)
    wts = np.ones(len(x)) if weights is None else weights
    for flat, w, _ in cic_corners(x, n_m, cell, order):
        mesh += np.bincount(flat, weights=w * wts, minlength=n_m ** 3)
    return mesh.reshape(n_m, n_m, n_m)


def cic_read(x, mesh, cell, order=2):
    """sum_c W(x_i - c) mesh(c) per particle."""
    n_m = mesh.shape[0]
    flatmesh = mesh.ravel()
    val = np.zeros(len(x))
    for flat, w, _ in cic_corners(x, n_m, cell, order):
        val += w * flatmesh[flat]
    return val


def cic_read_grad(x, mesh, cell, order=2):
    """sum_c dW(x_i - c)/dx_i mesh(c) per particle, (N, 3)."""
    n_m = mesh.shape[0]
    flatmesh = mesh.ravel()
    val = np.zeros((len(x), 3))
    for flat, _, grad in cic_corners(x, n_m, cell, order):
        val += grad * flatmesh[flat][:, None]
    return val


def density(s, setup):
    """CIC density contrast alpha sum W - 1 of the particles at s."""
    return setup.alpha * cic_paint(positions(s, setup), setup.n_m, setup.cell, order=setup.order) - 1.0


# -------------------------------------------------------------- force ----

SPECTRAL_GRADIENT, DECONVOLVE, LOG_A, TSC = 1, 2, 4, 8


def gradient_operator(k, h):
    """Fourier multiplier of the 4-point central difference d/dx on a mesh of
    spacing h (times i): (8 sin(k h) - sin(2 k h)) / (6 h)."""
    return (8.0 * np.sin(k * h) - np.sin(2.0 * k * h)) / (6.0 * h)


def cic_window(k, h, order=2):
    """Fourier transform of one assignment along one axis, sinc^order(k h / 2)
    (CIC order 2, TSC order 3)."""
    return np.sinc(k * h / (2.0 * np.pi)) ** order


def gradient_green_multipliers(n, box, omega_m, solver=0):
    order = 3 if solver & TSC else 2
    """i D_j (3/2) Om / k^2 on the rfft grid (D_j the 4-point difference
    gradient, or k_j with SPECTRAL_GRADIENT; k^2 exact; divided by the paint
    and read CIC windows with DECONVOLVE), zero at k = 0 and where n_j is the
    Nyquist index (so each inverse transform is exactly real) [reading]."""
    (kx, ky, kz), nyq = rfft_wavenumbers(n, box)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    k2s = np.where(k2 > 0, k2, 1.0)
    h = box / n
    if solver & DECONVOLVE:
        k2s = k2s * (cic_window(kx, h, order) * cic_window(ky, h, order) * cic_window(kz, h, order)) ** 2
    out = []
    for kj, mj in zip((kx, ky, kz), nyq):
        dj = kj if solver & SPECTRAL_GRADIENT else gradient_operator(kj, h)
        m = 1j * dj * (1.5 * omega_m) / k2s
        m = np.where((k2 > 0) & ~mj, m, 0.0)
        out.append(m)
    return out


def force_meshes(x, setup):
    rho = setup.alpha * cic_paint(x, setup.n_m, setup.cell, order=setup.order) - 1.0
    rho_k = rfftn(rho)
    mult = gradient_green_multipliers(setup.n_m, setup.box, setup.cosmo.omega_m, setup.solver)
    return [irfftn(m * rho_k, setup.n_m) for m in mult]


def force(s, setup):
    """PM force per particle, (N, 3), in lattice order."""
    x = positions(s, setup)
    meshes = force_meshes(x, setup)
    return np.stack([cic_read(x, m, setup.cell, setup.order) for m in meshes], axis=1)


def force_vjp(s, v, setup):
    """J(s)^T v for F(s) above (exact vector-Jacobian product):
    term A differentiates the interpolation weights, term B the painted
    density through the (real, odd) Green-gradient convolution whose adjoint
    multiplies by the conjugate multiplier."""
    x = positions(s, setup)
    meshes = force_meshes(x, setup)
    term_a = np.zeros((len(x), 3))
    for j in range(3):
        term_a += cic_read_grad(x, meshes[j], setup.cell, setup.order) * v[:, j:j + 1]
    mult = gradient_green_multipliers(setup.n_m, setup.box, setup.cosmo.omega_m, setup.solver)
    psi_k = 0.0
    for j in range(3):
        u_j = cic_paint(x, setup.n_m, setup.cell, v[:, j], setup.order)
        psi_k = psi_k + np.conj(mult[j]) * rfftn(u_j)
    psi = irfftn(psi_k, setup.n_m)
    term_b = setup.alpha * cic_read_grad(x, psi, setup.cell, setup.order)
    return term_a + term_b


# ------------------------------------------- sampled and reduced cases ----
# For meshes too large to run whole (the 512^3 / 1024^3 workload): values at
# chosen cells, and a state whose 3D PM force reduces exactly to 1D.

def lattice_sites(idx, n_p, box, n_m):
    """Lagrangian positions of the given flat lattice indices (the rule of
    `lattice`), (len(idx), 3)."""
    idx = np.asarray(idx, dtype=np.int64)
    ijk = np.stack([idx // (n_p * n_p), (idx // n_p) % n_p, idx % n_p], axis=1)
    return ijk * (box / n_p) + 0.5 * box / n_m


def density_at(cells, s, setup, s_max):
    """delta at the given flat mesh cells, each summed one by one over every
    lattice site whose particle can reach it: with |s| <= s_max per axis the
    CIC corners of site i along an axis lie within 2 + s_max / h nodes of
    i n_m / n_p + 1/2, so a window of sites around the cell covers them all."""
    n_p, n_m, h = setup.n_p, setup.n_m, setup.cell
    r = n_m / n_p
    half = int(np.ceil((2.0 + s_max / h) / r)) + 1
    win = np.arange(-half, half + 1)
    out = np.empty(len(cells))
    for j, c in enumerate(np.asarray(cells, dtype=np.int64)):
        cxyz = (c // (n_m * n_m), (c // n_m) % n_m, c % n_m)
        # each site once, also when the window is wider than the lattice
        ax = [np.unique((int(round((cxyz[d] - 0.5) / r)) + win) % n_p) for d in range(3)]
        ii = ((ax[0][:, None, None] * n_p + ax[1][None, :, None]) * n_p + ax[2][None, None, :]).ravel()
        x = lattice_sites(ii, n_p, setup.box, n_m) + s[ii]
        acc = 0.0
        for flat, w, _ in cic_corners(x, n_m, h, setup.order):
            acc += w[flat == c].sum()
        out[j] = setup.alpha * acc - 1.0
    return out


def force_uniform_yz(sx, setup):
    """PM force on a state uniform in y and z: every particle of lattice
    plane i_x has s = (sx[i_x], 0, 0).  With the half-cell lattice offset and
    n_m / n_p = 1 or 2, every y and every z node then receives the same CIC
    weight from each row of particles (n_p / n_m), so the density and the
    force depend on x alone, F_y = F_z = 0 (D(0) = 0), and the 3D definition
    above is exactly its 1D restriction:
        rho_1(c) = (n_m / n_p) sum_i w(u_i - c) - 1
        F(k) = i D(k) (3/2) Om rho_1(k) / k^2 (zero at k = 0 and Nyquist)
        F_i = sum_c w(u_i - c) F(c)
    (3D DFT normalisation: the y and z sums give n_m^2 forward and 1 / n_m^2
    back).  Returns F_x per lattice plane, (n_p,).  CIC only."""
    n_p, n_m, h = setup.n_p, setup.n_m, setup.cell
    if setup.order != 2 or n_m not in (n_p, 2 * n_p):
        raise ValueError("the 1D reduction holds for CIC with n_m = n_p or 2 n_p")
    x = np.arange(n_p) * (setup.box / n_p) + 0.5 * h + np.asarray(sx, dtype=np.float64)
    base, ax = _axis_weights(x / h, 2, h)
    rho = np.zeros(n_m)
    for k, (w, _) in enumerate(ax):
        rho += np.bincount((base + k) % n_m, weights=w, minlength=n_m)
    rho = (n_m / n_p) * rho - 1.0
    kx = 2.0 * np.pi / setup.box * np.arange(n_m // 2 + 1)
    k2 = np.where(kx > 0, kx * kx, 1.0)
    if setup.solver & DECONVOLVE:
        k2 = k2 * cic_window(kx, h) ** 2
    d = kx if setup.solver & SPECTRAL_GRADIENT else gradient_operator(kx, h)
    mult = np.where((kx > 0) & (np.arange(n_m // 2 + 1) != n_m // 2), 1j * d * 1.5 * setup.cosmo.omega_m / k2, 0.0)
    fmesh = sfft.irfft(mult * sfft.rfft(rho), n=n_m)
    out = np.zeros(n_p)
    for k, (w, _) in enumerate(ax):
        out += w * fmesh[(base + k) % n_m]
    return out


# ---------------------------------------------------------------- KDK ----

def coefficients(setup):
    return kdk_coefficients(setup.cosmo, setup.a_init, setup.a_final, setup.n_steps, bool(setup.solver & LOG_A))


def integrate(s, p, setup, force_fn=None, steps=None):
    """Forward KDK from a_init; returns (s, p, F(s)) after ``steps`` steps
    (default: all).  ``force_fn`` defaults to the PM force."""
    fn = force_fn or (lambda y: force(y, setup))
    c = coefficients(setup)
    s, p = s.copy(), p.copy()
    f = fn(s)
    for n in range(setup.n_steps if steps is None else steps):
        p = p + c["K_a"][n] * f
        s = s + c["Dr"][n] * p
        f = fn(s)
        p = p + c["K_b"][n] * f
    return s, p, f


def reverse_integrate(s, p, f, setup, steps=None):
    """Reverse time integration: undo the KDK steps from the last one back,
    recomputing forces instead of reading a stored history."""
    c = coefficients(setup)
    s, p = s.copy(), p.copy()
    n_steps = setup.n_steps if steps is None else steps
    for n in reversed(range(n_steps)):
        p = p - c["K_b"][n] * f
        s = s - c["Dr"][n] * p
        f = force(s, setup)
        p = p - c["K_a"][n] * f
    return s, p, f


def adjoint_integrate(s, p, f, lam, mu, setup):
    """Discrete adjoint of ``integrate`` run backward in time along the
    reconstructed trajectory.  (s, p, f) is the final state and F(s);
    (lam, mu) the cotangents of the final s and p.  Returns the initial state,
    the cotangents of the initial s and p, and the cotangents of the
    coefficients (K_a, Dr, K_b per step) and of Om through the force
    prefactor."""
    c = coefficients(setup)
    om = setup.cosmo.omega_m
    n_steps = setup.n_steps
    g_ka, g_dr, g_kb = np.zeros(n_steps), np.zeros(n_steps), np.zeros(n_steps)
    g_om_direct = 0.0
    s, p, lam, mu = s.copy(), p.copy(), lam.copy(), mu.copy()
    for n in reversed(range(n_steps)):
        # p_{n+1} = p_half + K_b F(s_{n+1})
        g_kb[n] = np.sum(mu * f)
        g_om_direct += c["K_b"][n] * g_kb[n] / om
        lam = lam + c["K_b"][n] * force_vjp(s, mu, setup)
        p_half = p - c["K_b"][n] * f
        # s_{n+1} = s_n + Dr p_half
        g_dr[n] = np.sum(lam * p_half)
        mu = mu + c["Dr"][n] * lam
        s = s - c["Dr"][n] * p_half
        f = force(s, setup)
        # p_half = p_n + K_a F(s_n)
        g_ka[n] = np.sum(mu * f)
        g_om_direct += c["K_a"][n] * g_ka[n] / om
        lam = lam + c["K_a"][n] * force_vjp(s, mu, setup)
        p = p_half - c["K_a"][n] * f
    grads = {"K_a": g_ka, "Dr": g_dr, "K_b": g_kb, "omega_m_direct": g_om_direct}
    return s, p, lam, mu, grads


def dynamics_domega(grads, setup):
    """Total d/dOm of the dynamics part: chain through the coefficient tables
    plus the direct force prefactor."""
    d = kdk_coefficients_domega(setup.cosmo, setup.a_init, setup.a_final, setup.n_steps, bool(setup.solver & LOG_A))
    return (np.dot(grads["K_a"], d["K_a"]) + np.dot(grads["Dr"], d["Dr"])
            + np.dot(grads["K_b"], d["K_b"]) + grads["omega_m_direct"])


# --------------------------------------------------------------- loss ----

def mse_loss(s, target, setup):
    """L = n_m^-3 sum_c (delta(c) - target(c))^2 of the final CIC density."""
    d = density(s, setup) - target
    return float(np.mean(d * d))


def mse_loss_grad(s, target, setup):
    """dL/ds: the CIC-weight-gradient read of 2 (delta - target) / n_m^3."""
    x = positions(s, setup)
    g_mesh = 2.0 * (density(s, setup) - target) / setup.n_m ** 3
    return setup.alpha * cic_read_grad(x, g_mesh, setup.cell, setup.order)


def density_vjp(s, g_mesh, setup):
    """Cotangent of s for a cotangent g_mesh of ``density(s)``."""
    return setup.alpha * cic_read_grad(positions(s, setup), g_mesh, setup.cell, setup.order)


# ----------------------------------------------------- power spectrum ----

def power_of_mesh(delta, box):
    """Binned power of a real n^3 mesh: bins b = 0 .. n/2-1 with edges
    (b + 1/2) k_F .. (b + 3/2) k_F over the full k space (rfft entries with
    0 < n_z < n/2 count twice), k = 0 excluded, no shot-noise or window
    correction [reading].  P_b = V / n^6 <|delta_k|^2>.  Returns
    (k_mean, P, n_modes)."""
    n = delta.shape[0]
    dk = rfftn(delta)
    (kx, ky, kz), _ = rfft_wavenumbers(n, box)
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    kf = 2.0 * np.pi / box
    iz = np.arange(n // 2 + 1)
    wz = np.where((iz == 0) | (iz == n // 2), 1.0, 2.0)[None, None, :]
    w = np.broadcast_to(wz, dk.shape).ravel()
    kk = np.broadcast_to(kmag, dk.shape).ravel()
    pw = (np.abs(dk) ** 2).ravel()
    nb = n // 2
    b = np.floor(kk / kf - 0.5).astype(np.int64)
    ok = (kk > 0) & (b >= 0) & (b < nb)
    n_modes = np.bincount(b[ok], weights=w[ok], minlength=nb)
    ksum = np.bincount(b[ok], weights=(w * kk)[ok], minlength=nb)
    psum = np.bincount(b[ok], weights=(w * pw)[ok], minlength=nb)
    vol = box ** 3
    safe = np.where(n_modes > 0, n_modes, 1.0)
    return ksum / safe, vol / n ** 6 * psum / safe, n_modes


def power_spectrum(s, setup):
    return power_of_mesh(density(s, setup), setup.box)


# ------------------------------------------------------------ pipeline ----

def simulate(noise, setup):
    """White noise -> 2LPT at a_init -> KDK to a_final: (s, p, F)."""
    from .lpt import initial_conditions
    s0, p0 = initial_conditions(noise, setup)
    return integrate(s0, p0, setup)


def loss_and_grad(noise, target, setup):
    """MSE of the final density against ``target`` and its gradient with
    respect to the white noise, Om and sigma8, by the adjoint method."""
    from .lpt import initial_conditions_vjp
    s, p, f = simulate(noise, setup)
    loss = mse_loss(s, target, setup)
    lam = mse_loss_grad(s, target, setup)
    _, _, lam0, mu0, grads = adjoint_integrate(s, p, f, lam, np.zeros_like(p), setup)
    g_noise, g_om_ic, g_s8 = initial_conditions_vjp(noise, lam0, mu0, setup)
    return loss, g_noise, g_om_ic + dynamics_domega(grads, setup), g_s8
