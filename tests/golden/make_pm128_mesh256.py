"""Write the FP64 oracle's results for the 128^3-particle, 256^3-mesh
gradient workload (256 Mpc/h, 63 KDK steps from 2LPT at a = 1/64, MSE of the
final CIC density against a seeded N(0, 1) target) to
``pm128_mesh256.npz`` beside this script.

The full run takes the oracle over an hour on a few host cores, too long for
a test, so this script runs it once and stores what the GPU test compares
with: the state after 10 steps and at a = 1 on a fixed sample of particles,
the loss, its gradients with respect to Omega_m and sigma8 (with the
magnitudes of the terms of dL/dOm), the cotangents (lam, mu) of the initial
state and the white-noise gradient on fixed samples.  Only ``oracle/`` and the
seeded input generators are called.

    python tests/golden/make_pm128_mesh256.py
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import lpt as olpt  # noqa: E402
from oracle import pm as opm  # noqa: E402
from oracle.cosmology import Cosmology, kdk_coefficients_domega  # noqa: E402
from paper_2211_09958_gb300 import inputs  # noqa: E402

N_P, N_M, BOX, STEPS = 128, 256, 256.0, 63
IC_SEED, TARGET_SEED = 1234, 1235
N_SAMPLE_PART, N_SAMPLE_NOISE, SAMPLE_SEED = 8192, 32768, 4242
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "pm128_mesh256.npz")


def main():
    t0 = time.time()
    st = opm.Setup(N_P, N_M, BOX, Cosmology(0.3, 0.8, 0.7, 0.96), a_init=1.0 / 64, a_final=1.0, n_steps=STEPS)
    noise = inputs.white_noise(N_P, IC_SEED).astype(np.float64)
    target = inputs.target_field(N_M, TARGET_SEED).astype(np.float64)
    rng = np.random.Generator(np.random.PCG64(SAMPLE_SEED))
    part = np.sort(rng.choice(N_P ** 3, N_SAMPLE_PART, replace=False))
    cells = np.sort(rng.choice(N_P ** 3, N_SAMPLE_NOISE, replace=False))

    s0, p0 = olpt.initial_conditions(noise, st)
    s10, p10, _ = opm.integrate(s0, p0, st, steps=10)
    print(f"10 steps: {time.time() - t0:.0f} s", flush=True)
    s, p, f = opm.integrate(s0, p0, st)
    print(f"63 steps: {time.time() - t0:.0f} s", flush=True)
    loss = opm.mse_loss(s, target, st)
    lam = opm.mse_loss_grad(s, target, st)
    _, _, lam0, mu0, grads = opm.adjoint_integrate(s, p, f, lam, np.zeros_like(p), st)
    print(f"adjoint: {time.time() - t0:.0f} s", flush=True)
    g_noise, g_om_ic, g_s8 = olpt.initial_conditions_vjp(noise, lam0, mu0, st)
    g_om_dyn = opm.dynamics_domega(grads, st)
    d = kdk_coefficients_domega(st.cosmo, st.a_init, st.a_final, st.n_steps)
    om_terms = (abs(grads["omega_m_direct"]) + sum(abs(np.dot(grads[k], d[k])) for k in ("K_a", "Dr", "K_b"))
                + abs(g_om_ic))
    np.savez_compressed(
        OUT, part=part, cells=cells,
        s10=s10[part].astype(np.float32), p10=p10[part].astype(np.float32),
        p10_max=np.abs(p10).max(),
        s63=s[part].astype(np.float32), p63=p[part].astype(np.float32),
        p63_max=np.abs(p).max(), p63_rms=np.sqrt(np.mean(p * p)),
        loss=loss, g_om=g_om_ic + g_om_dyn, g_om_dyn=g_om_dyn, g_om_ic=g_om_ic, g_om_terms=om_terms, g_s8=g_s8,
        lam0=lam0[part].astype(np.float32), mu0=mu0[part].astype(np.float32),
        g_noise=g_noise.ravel()[cells].astype(np.float32))
    print(f"wrote {OUT} in {time.time() - t0:.0f} s: loss {loss:.8g}, dL/dOm {g_om_ic + g_om_dyn:.8g}, "
          f"dL/ds8 {g_s8:.8g}")


if __name__ == "__main__":
    main()
