"""Host-side checks of libpmgb.so that need no GPU: every symbol declared in
include/pmgb.h is exported, config validation errors come back as codes,
and the library's own FP64 coefficient tables (independent C++ code) agree
with the oracle's."""

import ctypes
import os
import re

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


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "pmgb.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pm_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in _pmgb._SIGNATURES, n


@pytest.mark.parametrize("field,value", [("n_p", 3), ("n_p", 15), ("n_p", 8192), ("n_m", 2), ("n_m", 8194),
                                         ("n_batch", 0), ("n_steps", 0), ("box", -1.0), ("box", float("nan")),
                                         ("a_init", 2.0), ("a_final", 0.01), ("h", 0.0), ("solver", 32)])
def test_create_rejects_bad_config(lib, field, value):
    cfg = _pmgb.make_config(8, 16, 32.0, 0.3, 0.8, 4)
    setattr(cfg, field, value)
    out = ctypes.c_void_p()
    rc = lib.pm_create(ctypes.byref(cfg), ctypes.byref(out))
    assert rc == -1 and not out.value
    assert lib.pm_last_error(None)


def test_create_rejects_too_many_particles_before_allocating(lib):
    # 4096^3 particles x 3 floats x 6 runs exceeds the 2^40 element limit
    cfg = _pmgb.make_config(4096, 64, 1000.0, [0.3] * 6, [0.8] * 6, 4)
    out = ctypes.c_void_p()
    assert lib.pm_create(ctypes.byref(cfg), ctypes.byref(out)) == _pmgb.PM_ERANGE and not out.value
    assert b"too many particles" in lib.pm_last_error(None)


def test_null_arguments_are_rejected(lib):
    out = ctypes.c_void_p()
    assert lib.pm_create(None, ctypes.byref(out)) == _pmgb.PM_EINVAL and not out.value
    cfg = _pmgb.make_config(8, 16, 32.0, 0.3, 0.8, 4)
    assert lib.pm_create(ctypes.byref(cfg), None) == _pmgb.PM_EINVAL
    assert lib.pm_destroy(None) == _pmgb.PM_OK                   # destroying nothing is harmless
    assert lib.pm_set_tuning(None, None) == _pmgb.PM_EINVAL
    assert lib.pm_set_checkpoints(None, 1, None) == _pmgb.PM_EINVAL


def test_create_rejects_bad_cosmology(lib):
    cfg = _pmgb.make_config(8, 16, 32.0, 1.5, 0.8, 4)
    out = ctypes.c_void_p()
    assert lib.pm_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    assert b"omega_m" in lib.pm_last_error(None)


@pytest.mark.parametrize("om,s8,steps", [(0.3, 0.8, 10), (0.22, 0.65, 63), (0.38, 0.95, 3)])
def test_host_tables_match_oracle(lib, om, s8, steps):
    cfg = _pmgb.make_config(32, 64, 128.0, [om, 0.3], [s8, 0.8], steps)
    kdk, dkdk, lpt, amp = _pmgb.host_coefficients(cfg)
    cosmo = C.Cosmology(om, s8)
    ref = C.kdk_coefficients(cosmo, 1 / 64, 1.0, steps)
    dref = C.kdk_coefficients_domega(cosmo, 1 / 64, 1.0, steps)
    for j, k in enumerate(("K_a", "Dr", "K_b")):
        np.testing.assert_allclose(kdk[0, :, j], ref[k], rtol=1e-9)
        np.testing.assert_allclose(dkdk[0, :, j], dref[k], rtol=2e-6, atol=1e-9)
    np.testing.assert_allclose(lpt[0], C.lpt_growth(cosmo, 1 / 64), rtol=1e-9)
    np.testing.assert_allclose(amp[0, 0], C.power_amplitude(cosmo), rtol=1e-10)
    e = 1e-4
    dlna = (np.log(C.power_amplitude(cosmo.with_omega_m(om + e))) - np.log(C.power_amplitude(cosmo.with_omega_m(om - e)))) / (2 * e)
    np.testing.assert_allclose(amp[0, 1], dlna, rtol=1e-6)


@pytest.mark.parametrize("steps", [5, 40])
def test_log_a_tables_match_oracle(lib, steps):
    cfg = _pmgb.make_config(32, 64, 128.0, [0.3], [0.8], steps, solver=_pmgb.SOLVER_LOG_A)
    kdk, dkdk, _, _ = _pmgb.host_coefficients(cfg)
    cosmo = C.Cosmology(0.3, 0.8)
    ref = C.kdk_coefficients(cosmo, 1 / 64, 1.0, steps, log_a=True)
    dref = C.kdk_coefficients_domega(cosmo, 1 / 64, 1.0, steps, log_a=True)
    for j, k in enumerate(("K_a", "Dr", "K_b")):
        np.testing.assert_allclose(kdk[0, :, j], ref[k], rtol=1e-9)
        np.testing.assert_allclose(dkdk[0, :, j], dref[k], rtol=2e-6, atol=1e-9)
    plain, _, _, _ = _pmgb.host_coefficients(_pmgb.make_config(32, 64, 128.0, [0.3], [0.8], steps))
    assert not np.allclose(plain, kdk)                  # the flag reaches the tables


def test_unknown_solver_flag_is_rejected(lib):
    cfg = _pmgb.make_config(32, 64, 128.0, [0.3], [0.8], 4, solver=32)
    out = ctypes.c_void_p()
    assert lib.pm_create(ctypes.byref(cfg), ctypes.byref(out)) == -1
    assert b"solver" in lib.pm_last_error(None)


def test_noalloc_rejects_bad_arguments_before_any_device_work(lib):
    # every rejection of the allocation-free loss returns before the entry
    # point touches a device, so fake (never dereferenced) pointers serve
    s, t = ctypes.c_void_p(0x10000), ctypes.c_void_p(0x20000)
    loss_ok, loss_odd = ctypes.c_void_p(0x30000), ctypes.c_void_p(0x30004)
    f = lib.pm_mse_loss_noalloc
    assert f(8, 16, 65, 32.0, s, t, loss_ok, None, None) == -5          # more runs than loss slots
    assert f(64, 256, 1, 64.0, s, t, loss_ok, None, None) == -5         # 256^3 cells exceed the scratch
    assert f(8, 16, 1, 32.0, s, t, loss_odd, None, None) == -1          # loss not 8-byte aligned
    assert f(8, 16, 1, 32.0, s, None, loss_ok, None, None) == -1        # NULL target
    assert f(8, 16, 1, 32.0, None, t, loss_ok, None, None) == -1        # NULL displacements
    assert f(8, 16, 1, 32.0, s, t, None, None, None) == -1              # NULL loss
    assert f(1 << 21, 16, 1, 32.0, s, t, loss_ok, None, None) == -1     # n_p beyond pm_create's 4096
    assert f(7, 16, 1, 32.0, s, t, loss_ok, None, None) == -1           # odd n_p
    assert f(8, 16, 1, 0.0, s, t, loss_ok, None, None) == -1            # box <= 0
