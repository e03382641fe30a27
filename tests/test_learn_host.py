"""Host helpers of the learned-correction training (paper_2211_09958_gb300/learn.py),
pinned against the oracle's definitions.  No GPU."""

from types import SimpleNamespace

import numpy as np

from oracle import learned as olearned
from oracle import pm as opm
from paper_2211_09958_gb300 import inputs, learn


def test_lattice_shift_keeps_positions_between_meshes():
    # the same particle positions as displacements of two contexts whose
    # lattices sit half a (different) mesh cell off the nodes
    n_p, box = 8, 32.0
    src, dst = SimpleNamespace(box=box, n_m=32), SimpleNamespace(box=box, n_m=8)
    s = inputs.random_displacements(n_p, box, seed=3, scale=0.4).astype(np.float64)
    x_src = opm.lattice(n_p, box, src.n_m) + s
    x_dst = opm.lattice(n_p, box, dst.n_m) + s + learn.lattice_shift(src, dst)
    np.testing.assert_allclose(x_src, x_dst, rtol=0, atol=1e-12)
    assert learn.lattice_shift(src, src) == 0.0
    assert learn.lattice_shift(src, dst) == -learn.lattice_shift(dst, src)


def test_a_grid_is_uniform_in_a():
    pm = SimpleNamespace(cfg=SimpleNamespace(a_init=1.0 / 64, a_final=1.0), n_steps=40)
    a = learn.a_grid(pm)
    assert a.shape == (41,) and a[0] == 1.0 / 64 and abs(a[-1] - 1.0) < 1e-15
    np.testing.assert_allclose(np.diff(a), (1.0 - 1.0 / 64) / 40, rtol=1e-12)


def test_untrained_network_adds_nothing():
    theta = learn._init_theta(olearned.n_params(), seed=5)
    assert theta.dtype == np.float32 and theta.size == olearned.n_params()
    p = olearned.unflatten(theta)
    assert not np.any(p["W3"]) and not np.any(p["b1"]) and not np.any(p["b2"]) and not np.any(p["b3"])
    assert np.all(np.abs(p["W1"]).sum(axis=0) > 0) and np.all(np.abs(p["W2"]).sum(axis=0) > 0)
    setup = opm.Setup(8, 8, 32.0)
    s = inputs.random_displacements(8, 32.0, seed=6, scale=0.5).astype(np.float64)
    dF = olearned.predict(s, 0.5, theta, setup)
    assert not np.any(dF)                               # exactly zero: zero output layer and bias
