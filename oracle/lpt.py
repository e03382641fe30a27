"""Linear field and 2LPT initial conditions, and their adjoint (FP64, test
infrastructure only).

The paper treats the initial conditions of the cosmic density field as
parameters to be inferred together with the physical parameters (Statement of
Need) and differentiates with respect to cosmological parameters (Summary).
It gives no formulas; readings:

* delta_L(k) = omega(k) sqrt(P(|k|) / V_c), V_c = (L / n_p)^3, omega the
  unnormalised DFT of unit white noise on the n_p^3 lattice, delta_L(0) = 0
  [reading].
* 2LPT (Scoccimarro convention, D2 ~ -3/7 D1^2):                 [reading]
    phi1(k) = -delta_L / k^2,  s1 = -grad phi1,
    S = sum_{i<j} phi1_ii phi1_jj - phi1_ij^2  (real space),
    phi2(k) = -S(k) / k^2,     s2 = +grad phi2,
    s = D1 s1 + D2 s2,  p = a^3 E (D1' s1 + D2' s2)  at a_init.
  Odd derivatives along an axis at its Nyquist index, and mixed second
  derivatives with either axis at Nyquist, are set to zero so that every
  inverse transform is exactly real.                               [reading]
"""

import numpy as np

from .cosmology import FD_OMEGA, linear_power, lpt_growth, lpt_growth_domega
from .pm import irfftn, rfft_wavenumbers, rfftn

_PAIRS = ((0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2))


def _apply(mult, field, n):
    return irfftn(mult * rfftn(field), n)


def _adjoint_apply(mult, field, n):
    return irfftn(np.conj(mult) * rfftn(field), n)


def linear_multiplier(setup, cosmo=None):
    """sqrt(P(|k|) / V_c) on the rfft grid of the particle lattice."""
    cosmo = cosmo or setup.cosmo
    n = setup.n_p
    (kx, ky, kz), _ = rfft_wavenumbers(n, setup.box)
    kmag = np.sqrt(kx ** 2 + ky ** 2 + kz ** 2)
    vc = setup.spacing ** 3
    return np.sqrt(linear_power(kmag, cosmo) / vc)


def lpt_multipliers(n, box):
    """Multipliers for s1_j (i k_j / k^2), phi1_ij (k_i k_j / k^2) and
    s2_j (-i k_j / k^2), with the Nyquist zeroing of the module docstring."""
    (kx, ky, kz), nyq = rfft_wavenumbers(n, box)
    ks = (kx, ky, kz)
    k2 = kx ** 2 + ky ** 2 + kz ** 2
    nz = k2 > 0
    k2s = np.where(nz, k2, 1.0)
    s1 = [np.where(nz & ~nyq[j], 1j * ks[j] / k2s, 0.0) for j in range(3)]
    phi = []
    for i, j in _PAIRS:
        m = ks[i] * ks[j] / k2s
        keep = nz if i == j else nz & ~nyq[i] & ~nyq[j]
        phi.append(np.where(keep, m, 0.0))
    s2 = [-m for m in s1]
    return s1, phi, s2


def linear_field(noise, setup):
    return _apply(linear_multiplier(setup), noise, setup.n_p)


def lpt_fields(delta_l, setup):
    """First- and second-order displacement fields, each (N, 3) in lattice
    order, plus the six phi1_ij fields (for the adjoint)."""
    n = setup.n_p
    m_s1, m_phi, m_s2 = lpt_multipliers(n, setup.box)
    dk = rfftn(delta_l)
    s1 = [irfftn(m * dk, n) for m in m_s1]
    phi = [irfftn(m * dk, n) for m in m_phi]
    src = (phi[0] * phi[1] + phi[0] * phi[2] + phi[1] * phi[2]
           - phi[3] ** 2 - phi[4] ** 2 - phi[5] ** 2)
    sk = rfftn(src)
    s2 = [irfftn(m * sk, n) for m in m_s2]
    flat = lambda fs: np.stack([f.ravel() for f in fs], axis=1)
    return flat(s1), flat(s2), phi


def initial_conditions(noise, setup):
    """(s, p) at a_init from the white noise, lattice order."""
    delta_l = linear_field(noise, setup)
    s1, s2, _ = lpt_fields(delta_l, setup)
    d1, d2, g1, g2 = lpt_growth(setup.cosmo, setup.a_init)
    return d1 * s1 + d2 * s2, g1 * s1 + g2 * s2


def initial_conditions_vjp(noise, lam, mu, setup):
    """Adjoint of ``initial_conditions``: cotangents (lam, mu) of (s, p) ->
    (d/dnoise, d/dOm, d/dsigma8).  Each linear spectral map x -> IDFT(M DFT x)
    with Hermitian M has the adjoint y -> IDFT(conj(M) DFT y)."""
    n = setup.n_p
    cosmo = setup.cosmo
    shape = (n, n, n)
    m_lin = linear_multiplier(setup)
    delta_l = _apply(m_lin, noise, n)
    s1, s2, phi = lpt_fields(delta_l, setup)
    d1, d2, g1, g2 = lpt_growth(cosmo, setup.a_init)
    # s = d1 s1 + d2 s2, p = g1 s1 + g2 s2
    gs1 = d1 * lam + g1 * mu
    gs2 = d2 * lam + g2 * mu
    g_growth = np.array([np.sum(lam * s1), np.sum(lam * s2),
                         np.sum(mu * s1), np.sum(mu * s2)])
    m_s1, m_phi, m_s2 = lpt_multipliers(n, setup.box)
    # s2_j = IDFT(m_s2_j DFT S)
    g_src = sum(_adjoint_apply(m_s2[j], gs2[:, j].reshape(shape), n) for j in range(3))
    # S = phi_xx phi_yy + phi_xx phi_zz + phi_yy phi_zz - phi_xy^2 - phi_xz^2 - phi_yz^2
    g_phi = [g_src * (phi[1] + phi[2]), g_src * (phi[0] + phi[2]), g_src * (phi[0] + phi[1]),
             -2.0 * g_src * phi[3], -2.0 * g_src * phi[4], -2.0 * g_src * phi[5]]
    g_dl = sum(_adjoint_apply(m_s1[j], gs1[:, j].reshape(shape), n) for j in range(3))
    g_dl = g_dl + sum(_adjoint_apply(m_phi[q], g_phi[q], n) for q in range(6))
    g_noise = _adjoint_apply(m_lin, g_dl, n)
    g_sigma8 = np.sum(g_dl * delta_l) / cosmo.sigma8
    dm_lin = (linear_multiplier(setup, cosmo.with_omega_m(cosmo.omega_m + FD_OMEGA))
              - linear_multiplier(setup, cosmo.with_omega_m(cosmo.omega_m - FD_OMEGA))) / (2 * FD_OMEGA)
    g_om = np.sum(g_dl * _apply(dm_lin, noise, n))
    g_om += np.dot(g_growth, lpt_growth_domega(cosmo, setup.a_init))
    return g_noise, g_om, g_sigma8
