"""The growth-function emulator (include/pmgb.h pm_growth_emulate, solver
flag PM_SOLVER_GROWTH_EMULATOR) against the FP64 oracle's growth ODE solve,
on the host (no GPU).

  * D1, D2, dD1/da, dD2/da at 300 random (a, Omega_m) over the emulator's
    domain, a in [1e-3, 1] (log-uniform), Omega_m in [0.1, 0.6]: within
    1e-9 relative of the oracle's ODE solve (DOP853, rtol 1e-13); the oracle
    pins that solve against the EdS closed form and the Heath integral;
  * the Omega_m derivatives against central differences of the oracle's
    solve (step 1e-5): within 1e-6 relative (the accuracy of the differences);
  * the KDK, d/dOm and 2LPT tables pm_create computes with the emulator flag
    against the same tables from the ODE solve, for the workloads' time grids
    and the batched workload's Omega_m range;
  * out-of-range inputs are rejected (PM_ERANGE), also by pm_create.
"""

import ctypes
import os

import numpy as np
import pytest

from oracle import cosmology as C
from paper_2211_09958_gb300 import _pmgb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_pmgb.library_path()):
        import __graft_entry__
        __graft_entry__.build()
    return _pmgb.load()


def _emulate(lib, om, a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    out = np.zeros((len(a), 8))
    rc = lib.pm_growth_emulate(om, len(a), a.ctypes.data_as(_pmgb._c_double_p), out.ctypes.data_as(_pmgb._c_double_p))
    return rc, out


def test_emulator_matches_the_oracle_growth_solve(lib):
    rng = np.random.default_rng(11)
    worst = 0.0
    for om in rng.uniform(0.1, 0.6, 12):
        a = np.sort(np.exp(rng.uniform(np.log(1e-3), 0.0, 25)))
        rc, out = _emulate(lib, om, a)
        assert rc == 0
        g = C.growth(a, om)
        for col, key in ((0, "D1"), (1, "D2"), (2, "dD1"), (3, "dD2")):
            err = np.max(np.abs(out[:, col] - g[key]) / np.abs(g[key]))
            worst = max(worst, err)
            assert err < 1e-9, (om, key, err)
    print(f"emulator vs oracle growth solve: worst relative error {worst:.2e}")


def test_emulator_omega_derivatives_match_central_differences(lib):
    rng = np.random.default_rng(12)
    eps = 1e-5
    for om in rng.uniform(0.15, 0.55, 5):
        a = np.sort(np.exp(rng.uniform(np.log(2e-3), 0.0, 10)))
        rc, out = _emulate(lib, om, a)
        assert rc == 0
        up, dn = C.growth(a, om + eps), C.growth(a, om - eps)
        for col, key in ((4, "D1"), (5, "D2"), (6, "dD1"), (7, "dD2")):
            fd = (up[key] - dn[key]) / (2 * eps)
            scale = np.maximum(np.abs(fd), 1e-3 * np.abs(up[key]) / 0.3)
            err = np.max(np.abs(out[:, col] - fd) / scale)
            assert err < 1e-6, (om, key, err)


@pytest.mark.parametrize("steps,a_init,oms", [(10, 1 / 64, [0.3]), (100, 1 / 64, [0.3]),
                                              (20, 1 / 64, [0.2, 0.27, 0.33, 0.4]), (40, 0.02, [0.25])])
def test_tables_with_the_emulator_match_the_ode_tables(lib, steps, a_init, oms):
    out = {}
    for solver in (0, _pmgb.SOLVER_GROWTH_EMULATOR):
        cfg = _pmgb.make_config(32, 64, 128.0, oms, [0.8] * len(oms), steps, a_init=a_init, solver=solver)
        kdk = np.zeros((len(oms), steps, 3))
        dkdk = np.zeros_like(kdk)
        lpt = np.zeros((len(oms), 4))
        amp = np.zeros((len(oms), 2))
        rc = lib.pm_host_coefficients(ctypes.byref(cfg), *(x.ctypes.data_as(_pmgb._c_double_p)
                                                           for x in (kdk, dkdk, lpt, amp)))
        assert rc == 0
        out[solver] = (kdk, dkdk, lpt, amp)
    ode, emu = out[0], out[_pmgb.SOLVER_GROWTH_EMULATOR]
    assert np.max(np.abs(emu[0] - ode[0]) / np.abs(ode[0])) < 1e-8      # K_a, Dr, K_b
    assert np.max(np.abs(emu[2] - ode[2]) / np.abs(ode[2])) < 1e-8      # D1, D2, g1, g2 at a_init
    # d/dOm by central differences of either table (step 1e-5): the
    # differences carry ~1e-11 / 1e-5 of rounding
    assert np.max(np.abs(emu[1] - ode[1])) < 1e-5 * np.max(np.abs(ode[1]))
    np.testing.assert_array_equal(emu[3], ode[3])                         # P(k) amplitude: no growth involved


def test_out_of_range_is_rejected(lib):
    assert _emulate(lib, 0.05, [0.5])[0] == -5
    assert _emulate(lib, 0.3, [5e-4])[0] == -5
    assert _emulate(lib, 0.3, [1.5])[0] == -5
    assert lib.pm_growth_emulate(0.3, -1, None, None) == -1
    assert lib.pm_growth_emulate(0.3, 0, None, None) == 0
    cfg = _pmgb.make_config(32, 64, 128.0, [0.7], [0.8], 4, solver=_pmgb.SOLVER_GROWTH_EMULATOR)
    out = ctypes.c_void_p()
    assert lib.pm_create(ctypes.byref(cfg), ctypes.byref(out)) == -5
    cfg = _pmgb.make_config(32, 64, 128.0, [0.3], [0.8], 4, a_init=1e-4, solver=_pmgb.SOLVER_GROWTH_EMULATOR)
    assert lib.pm_create(ctypes.byref(cfg), ctypes.byref(out)) == -5
