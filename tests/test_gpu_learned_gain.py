"""What the trained correction gains over plain PM (learned force
correction, include/pmgb.h pm_nn_*; training in paper_2211_09958_gb300/learn.py).

Workload (small version of the 128^3 / 128^3 / 40-step one): 64^3 particles
on a 64^3 mesh in a 128 Mpc/h box, 20 KDK steps from a = 1/64; reference PM
on a 4x finer mesh (256^3) with 4x the steps; the network trained on 16
seeded reference runs, evaluated on 4 other seeds by the P(k) of the final
density, all measured on the reference mesh, up to half the coarse mesh's
Nyquist frequency.  Plain PM there is ~29 % low; the correction must take
at least half of that error away, and no bin may get worse than plain PM.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_trained_correction_beats_plain_pm():
    from paper_2211_09958_gb300 import learn
    st = learn.LearnedSetup(n_p=64, n_m=64, box=128.0, n_steps=20, group=4)
    theta, log = learn.train(st, list(range(100, 116)), epochs=3, lr=1e-3, lr_final=1e-4)
    # the weighted force-matching loss falls on every snapshot after a = a_init
    nb = st.n_steps + 1
    last = np.array(log.losses[-nb:])
    assert np.all(np.isfinite(last)) and np.mean(last) < 1.0
    ev = learn.evaluate(st, theta, [1000, 1001, 1002, 1003])
    plain, corr = ev["plain"]["max_abs_rel_err"], ev["corrected"]["max_abs_rel_err"]
    assert plain > 0.1, plain                      # the coarse mesh is visibly wrong
    assert corr < 0.5 * plain, (corr, plain)
    sel = ev["k"] <= ev["k_cut"]
    assert np.all(np.abs(ev["corrected"]["rel_err"][sel]) <= np.abs(ev["plain"]["rel_err"][sel]) + 5e-3)


def test_trajectory_training_lowers_the_density_loss():
    """Fine-tuning through the trajectory (final-density MSE against the
    reference, gradient by the corrected reverse-time adjoint) lowers its
    loss on the training runs."""
    from paper_2211_09958_gb300 import learn
    st = learn.LearnedSetup(n_p=64, n_m=64, box=128.0, n_steps=10, group=4)
    theta, _ = learn.train(st, list(range(100, 108)), epochs=2, lr=1e-3, lr_final=1e-4)
    _, losses = learn.train_trajectory(st, list(range(100, 108)), theta, steps=40, lr=6e-4, lr_final=6e-5)
    assert np.all(np.isfinite(losses))
    assert np.mean(losses[-6:]) < 0.9 * np.mean(losses[:6]), (losses[:6], losses[-6:])
