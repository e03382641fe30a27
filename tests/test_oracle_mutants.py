"""Mutation check of the oracle's pins (slow: collected by pytest, run only
with ``--runslow``; about 30 s per mutant, 30 minutes in all).

Each entry plants one plausible mistake in the oracle -- a dropped term, a
wrong sign, index, exponent or prefactor -- in a temporary copy of the
repository, runs the oracle's pin tests (tests/test_oracle_*.py, CPU only)
there and reports whether at least one of them failed.  A mutant that
survives marks a piece of the oracle that nothing pins.  The working tree is
never modified.

    python -m pytest tests/test_oracle_mutants.py --runslow -q   # every mutant
    python tests/test_oracle_mutants.py "D sign"                 # named ones, by hand

Expected survivor: "out scale", the output scale of the learned correction,
which is part of the network's design rather than of the method.
"""

import os
import shutil
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTANTS = [
    ("oracle/pm.py", "+ 0.5 * box / n_m\n    qx", "+ 0.0 * box / n_m\n    qx", "lattice offset"),
    ("oracle/pm.py", "(1.0 - f, -np.ones_like(f) / cell)", "(1.0 - f, np.ones_like(f) / cell)", "cic dw sign"),
    ("oracle/pm.py", "(0.75 - d * d, -2.0 * d / cell)", "(0.75 - d * d, -1.0 * d / cell)", "tsc dw"),
    ("oracle/pm.py", "(0.75 - d * d,", "(0.70 - d * d,", "tsc w"),
    ("oracle/pm.py", "return (8.0 * np.sin(k * h)", "return (7.0 * np.sin(k * h)", "D 8"),
    ("oracle/pm.py", "- np.sin(2.0 * k * h)) / (6.0 * h)", "+ np.sin(2.0 * k * h)) / (6.0 * h)", "D sign"),
    ("oracle/pm.py", "/ (2.0 * np.pi)) ** order", "/ (2.0 * np.pi)) ** (order + 1)", "window order"),
    ("oracle/pm.py", "m = 1j * dj * (1.5 * omega_m) / k2s", "m = -1j * dj * (1.5 * omega_m) / k2s", "mult sign"),
    ("oracle/pm.py", "m = 1j * dj * (1.5 * omega_m) / k2s", "m = 1j * dj * (1.4 * omega_m) / k2s", "mult 1.5"),
    ("oracle/pm.py", "m = np.where((k2 > 0) & ~mj, m, 0.0)", "m = np.where((k2 > 0), m, 0.0)", "nyq mask"),
    ("oracle/pm.py", "psi_k = psi_k + np.conj(mult[j])", "psi_k = psi_k + (mult[j])", "vjp conj"),
    ("oracle/pm.py", "term_b = setup.alpha * cic_read_grad", "term_b = cic_read_grad", "vjp alpha"),
    ("oracle/pm.py", "half = int(np.ceil((2.0 + s_max / h) / r)) + 1", "half = int(np.ceil((0.0 + s_max / h) / r))", "density_at window"),
    ("oracle/pm.py", "k2 = k2 * cic_window(kx, h) ** 2", "k2 = k2 * cic_window(kx, h)", "1d deconv"),
    ("oracle/pm.py", "rho = (n_m / n_p) * rho - 1.0", "rho = (n_m / n_p) ** 2 * rho - 1.0", "1d alpha"),
    ("oracle/pm.py", "        p = p + c[\"K_b\"][n] * f\n    return s, p, f", "        p = p + c[\"K_a\"][n] * f\n    return s, p, f", "fwd Kb"),
    ("oracle/pm.py", "        g_dr[n] = np.sum(lam * p_half)", "        g_dr[n] = np.sum(lam * p)", "g_dr"),
    ("oracle/pm.py", "        g_om_direct += c[\"K_a\"][n] * g_ka[n] / om", "        g_om_direct += 0.0", "g_om ka"),
    ("oracle/pm.py", "        mu = mu + c[\"Dr\"][n] * lam", "        mu = mu - c[\"Dr\"][n] * lam", "mu update"),
    ("oracle/pm.py", "g_mesh = 2.0 * (density(s, setup) - target)", "g_mesh = 1.0 * (density(s, setup) - target)", "mse grad 2"),
    ("oracle/pm.py", "wz = np.where((iz == 0) | (iz == n // 2), 1.0, 2.0)", "wz = np.where((iz == 0), 1.0, 2.0)", "pk nyq weight"),
    ("oracle/pm.py", "b = np.floor(kk / kf - 0.5)", "b = np.floor(kk / kf - 1.0)", "pk bins"),
    ("oracle/pm.py", "return ksum / safe, vol / n ** 6 * psum / safe", "return ksum / safe, vol / n ** 3 * psum / safe", "pk norm"),
    ("oracle/lpt.py", "s1 = [np.where(nz & ~nyq[j], 1j * ks[j] / k2s, 0.0)", "s1 = [np.where(nz & ~nyq[j], -1j * ks[j] / k2s, 0.0)", "s1 sign"),
    ("oracle/lpt.py", "    s2 = [-m for m in s1]", "    s2 = [m for m in s1]", "s2 sign"),
    ("oracle/lpt.py", "- phi[3] ** 2 - phi[4] ** 2 - phi[5] ** 2)", "- phi[3] ** 2 - phi[4] ** 2 - phi[4] ** 2)", "src index"),
    ("oracle/lpt.py", "keep = nz if i == j else nz & ~nyq[i] & ~nyq[j]", "keep = nz", "phi nyq"),
    ("oracle/lpt.py", "    vc = setup.spacing ** 3", "    vc = setup.spacing ** 2", "vc"),
    ("oracle/lpt.py", "-2.0 * g_src * phi[3]", "-1.0 * g_src * phi[3]", "adj phi3"),
    ("oracle/lpt.py", "g_sigma8 = np.sum(g_dl * delta_l) / cosmo.sigma8", "g_sigma8 = 2 * np.sum(g_dl * delta_l) / cosmo.sigma8", "g_s8"),
    ("oracle/lpt.py", "g_om += np.dot(g_growth, lpt_growth_domega(cosmo, setup.a_init))", "g_om += 0.0", "g_om growth"),
    ("oracle/cosmology.py", "    damp = 3.0 / a + _dlne_da(a, om)", "    damp = 2.0 / a + _dlne_da(a, om)", "damp"),
    ("oracle/cosmology.py", "acc2 = -damp * v2 + src * (d2 - d1 * d1)", "acc2 = -damp * v2 + src * (d2 + d1 * d1)", "D2 src"),
    ("oracle/cosmology.py", "g[\"gp2\"] = a ** 3 * e * g[\"dD2\"]", "g[\"gp2\"] = a ** 2 * e * g[\"dD2\"]", "gp2"),
    ("oracle/cosmology.py", "return a, np.sqrt(a[:-1] * a[1:])", "return a, 0.5 * (a[:-1] + a[1:])", "log mid"),
    ("oracle/cosmology.py", "k_a = (gp_h - gp_a[:-1]) / gf_a[:-1]", "k_a = (gp_h - gp_a[:-1]) / gf_a[1:]", "k_a"),
    ("oracle/cosmology.py", "drift = (d1_a[1:] - d1_a[:-1]) / gp_h", "drift = (d1_a[1:] - d1_a[:-1]) / gp_a[1:]", "drift"),
    ("oracle/cosmology.py", "(1.0 / 280.0 + x2 * (-1.0 / 15120.0 + x2 / 1330560.0))", "(1.0 / 280.0)", "tophat series m3"),
    ("oracle/pm.py", "ax = [np.unique((int(round((cxyz[d] - 0.5) / r)) + win) % n_p)", "ax = [((int(round((cxyz[d] - 0.5) / r)) + win) % n_p)", "density_at unique"),
    ("oracle/learned.py", "f[:, q] = np.roll(d, shift=(-ox, -oy, -oz)", "f[:, q] = np.roll(d, shift=(ox, oy, oz)", "feat roll"),
    ("oracle/learned.py", "    f[:, 27] = a\n", "    f[:, 27] = 0.0\n", "feat a"),
    ("oracle/learned.py", "d = np.arcsinh(rho - 1.0)", "d = np.arcsinh(rho)", "feat asinh"),
    ("oracle/learned.py", "h2 = r(np.maximum(z2, 0.0))", "h2 = r(z2)", "relu2"),
    ("oracle/learned.py", "rounded = (u + 0x7FFF + ((u >> 16) & 1))", "rounded = (u + 0x8000)", "bf16 rne"),
    ("oracle/learned.py", "pm.cic_paint(xpos, n, setup.cell, 2.0 * d[:, j] / npart, setup.order)", "pm.cic_paint(xpos, n, setup.cell, 1.0 * d[:, j] / npart, setup.order)", "lg 2"),
    ("oracle/learned.py", "g_d += np.roll(gx[:, q].reshape(n, n, n), shift=(ox, oy, oz)", "g_d += np.roll(gx[:, q].reshape(n, n, n), shift=(-ox, -oy, -oz)", "vjp roll"),
    ("oracle/learned.py", "g_rho = g_d / np.sqrt(1.0 + (rho - 1.0) ** 2)", "g_rho = g_d", "vjp asinh"),
    ("oracle/learned.py", "g_paint = setup.alpha * pm.cic_read_grad(xpos, g_rho, h, order)", "g_paint = pm.cic_read_grad(xpos, g_rho, h, order)", "vjp alpha nn"),
    ("oracle/learned.py", "        gl, gt = vjp(s, mu, a[n + 1], c[\"K_b\"][n])", "        gl, gt = vjp(s, mu, a[n], c[\"K_b\"][n])", "adj a index"),
    ("oracle/pm.py", "qx, qy, qz = np.meshgrid(g, g, g, indexing=\"ij\")", "qx, qy, qz = np.meshgrid(g, g, g, indexing=\"xy\")", "lattice order"),
    ("oracle/pm.py", "ksum = np.bincount(b[ok], weights=(w * kk)[ok], minlength=nb)", "ksum = np.bincount(b[ok], weights=(kk)[ok], minlength=nb)", "pk kmean"),
    ("oracle/pm.py", "return float(np.mean(d * d))", "return float(np.sum(d * d))", "mse mean"),
    ("oracle/pm.py", "    kz = (kf * half)[None, None, :]", "    kz = (kf * half * 1.0000001)[None, None, :]", "kz"),
    ("oracle/pm.py", "nyq = ((ix == n // 2)[:, None, None], (ix == n // 2)[None, :, None],", "nyq = ((ix == n // 2 + 1)[:, None, None], (ix == n // 2)[None, :, None],", "nyq x index"),
    ("oracle/pm.py", "        p = p - c[\"K_a\"][n] * f\n    return s, p, f", "        p = p - c[\"K_b\"][n] * f\n    return s, p, f", "rev Ka"),
    ("oracle/pm.py", "        g_kb[n] = np.sum(mu * f)", "        g_kb[n] = np.sum(mu * p)", "g_kb"),
    ("oracle/pm.py", "    return setup.alpha * cic_read_grad(positions(s, setup), g_mesh, setup.cell, setup.order)", "    return cic_read_grad(positions(s, setup), g_mesh, setup.cell, setup.order)", "density_vjp alpha"),
    ("oracle/lpt.py", "g_om = np.sum(g_dl * _apply(dm_lin, noise, n))", "g_om = 0.0", "g_om lin"),
    ("oracle/lpt.py", "g_src * (phi[1] + phi[2]), g_src * (phi[0] + phi[2])", "g_src * (phi[1] + phi[2]), g_src * (phi[0] + phi[1])", "adj phi1"),
    ("oracle/cosmology.py", "    return np.sqrt(om * a ** -3 + (1.0 - om))", "    return np.sqrt(om * a ** -3 + (1.0 - om) * 1.001)", "E"),
    ("oracle/cosmology.py", "    src = 1.5 * om / (a ** 5 * e2)", "    src = 1.5 * om / (a ** 5 * e2) * 1.001", "growth src"),
    ("oracle/cosmology.py", "    g[\"gf\"] = 1.5 * om * g[\"D1\"]", "    g[\"gf\"] = 1.5 * om * g[\"D1\"] * 1.001", "gf"),
    ("oracle/learned.py", "return 1.5 * setup.cosmo.omega_m * setup.cell", "return 1.5 * setup.cosmo.omega_m",
     "out scale"),
]
EXPECTED_SURVIVORS = {"out scale"}

PIN_TESTS = ["tests/test_oracle_pm.py", "tests/test_oracle_lpt.py", "tests/test_oracle_integrate.py",
             "tests/test_oracle_cosmology.py", "tests/test_oracle_learned.py", "tests/test_oracle_philox.py"]


def _copy_repo(dst):
    skip = shutil.ignore_patterns(".git", "_work", "gpurun_out", "_lib", "_build", "__pycache__", "baseline",
                                  "*.so", "*.o")
    shutil.copytree(ROOT, dst, ignore=skip)


def _pins_fail(repo, path, old, new):
    """Plant one mistake in the copy at ``repo``, run the pin tests there and
    restore the file; returns (True if a pin failed, the last output line),
    or (None, message) when the original text is not found exactly once."""
    target = os.path.join(repo, path)
    text = open(target).read()
    if text.count(old) != 1:
        return None, f"the original text occurs {text.count(old)} times"
    xdist = ["-n", "8"] if _have_xdist() else []
    open(target, "w").write(text.replace(old, new))
    try:
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *xdist,
                            *PIN_TESTS], cwd=repo, capture_output=True, text=True, timeout=1800)
    finally:
        open(target, "w").write(text)
    return r.returncode != 0, (r.stdout.strip().splitlines() or [""])[-1]


def run(names=()):
    survivors = []
    with tempfile.TemporaryDirectory() as tmp:
        repo = os.path.join(tmp, "repo")
        _copy_repo(repo)
        for path, old, new, label in MUTANTS:
            if names and label not in names:
                continue
            killed, tail = _pins_fail(repo, path, old, new)
            print(f"{'killed   ' if killed else 'SURVIVED '} {label}: {tail}", flush=True)
            if not killed:
                survivors.append(label)
    unexpected = sorted(set(survivors) - EXPECTED_SURVIVORS)
    print("survivors:", survivors, "unexpected:", unexpected)
    return 1 if unexpected else 0


def _have_xdist():
    try:
        import xdist  # noqa: F401
        return True
    except ImportError:
        return False


@pytest.fixture(scope="module")
def repo_copy(tmp_path_factory):
    repo = str(tmp_path_factory.mktemp("mutants") / "repo")
    _copy_repo(repo)
    return repo


@pytest.mark.slow
@pytest.mark.parametrize("path,old,new,label", MUTANTS, ids=[m[3] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(repo_copy, path, old, new, label):
    killed, tail = _pins_fail(repo_copy, path, old, new)
    assert killed is not None, tail
    if label in EXPECTED_SURVIVORS:
        pytest.skip(f"{label} is part of the network's design, which nothing in the method fixes")
    assert killed, f"{label} survived: {tail}"


if __name__ == "__main__":
    sys.exit(run(tuple(sys.argv[1:])))
