"""PyTorch front end of the GB300 particle-mesh library.

``ParticleMesh`` owns one library context (include/pmgb.h) and exposes its
calls under the same names; torch supplies device memory and the current
CUDA stream only.  ``simulate`` and ``density`` are ``torch.autograd``
functions: the backward of ``simulate`` is the library's reverse-time adjoint
(pmwd's adjoint method with reverse time integration, paper Summary and
Statement of Need), so no trajectory is stored.
"""

import ctypes

import numpy as np
import torch

from . import _pmgb


class PMError(RuntimeError):
    pass


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class ParticleMesh:
    """A batch of n_batch PM simulations sharing (n_p, n_m, box, steps)."""

    def __init__(self, n_p, n_m, box, omega_m=0.3, sigma8=0.8, n_steps=10, a_init=1.0 / 64, a_final=1.0,
                 h=0.7, n_s=0.96, device=None, solver=0):
        if not torch.cuda.is_available():
            raise PMError("ParticleMesh needs a CUDA device (there is no CPU path)")
        self._lib = _pmgb.load()
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None else
                                   torch.device(device).index or 0)
        self.cfg = _pmgb.make_config(n_p, n_m, box, omega_m, sigma8, n_steps, a_init, a_final, h, n_s, solver)
        self.n_p, self.n_m, self.box, self.n_steps = n_p, n_m, float(box), n_steps
        self.n_batch = self.cfg.n_batch
        self.omega_m = np.array(self.cfg._keep[0])
        self.sigma8 = np.array(self.cfg._keep[1])
        self._ctx = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self._lib.pm_create(ctypes.byref(self.cfg), ctypes.byref(self._ctx))
        if rc != _pmgb.PM_OK:
            raise PMError(f"pm_create: {_pmgb.ERRORS.get(rc, rc)}: {self._lib.pm_last_error(None).decode()}")
        tuning = self.get_tuning()
        self._x_round_default = tuning["x_round"]          # 2, or 3 on meshes of 512 and more
        self._pipeline_default = tuning["pipeline"]        # 2, or 1 with the spectral-gradient flag
        self._deposit_default = tuning["deposit"]          # 1: the atomic scatter

    # ------------------------------------------------------------ helpers --
    @property
    def n_part(self):
        return self.n_p ** 3

    def _call(self, name, *args):
        stream = torch.cuda.current_stream(self.device).cuda_stream
        rc = self._lib.pm_set_stream(self._ctx, ctypes.c_void_p(stream))
        if rc == _pmgb.PM_OK:
            rc = getattr(self._lib, name)(self._ctx, *args)
        if rc != _pmgb.PM_OK:
            raise PMError(f"{name}: {_pmgb.ERRORS.get(rc, rc)}: {self._lib.pm_last_error(self._ctx).decode()}")

    def _particles(self, t, name):
        if t is None:
            raise PMError(f"{name} is required")
        want = (self.n_batch, self.n_part, 3)
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != want:
            raise PMError(f"{name} must be a contiguous float32 CUDA tensor of shape {want}, got "
                          f"{tuple(t.shape)} {t.dtype} {t.device}")
        return t

    def _mesh(self, t, name):
        want = (self.n_batch, self.n_m, self.n_m, self.n_m)
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != want:
            raise PMError(f"{name} must be a contiguous float32 CUDA tensor of shape {want}")
        return t

    def _lattice(self, t, name):
        want = (self.n_batch, self.n_p, self.n_p, self.n_p)
        if t.dtype != torch.float32 or not t.is_cuda or not t.is_contiguous() or tuple(t.shape) != want:
            raise PMError(f"{name} must be a contiguous float32 CUDA tensor of shape {want}")
        return t

    def new_particles(self):
        return torch.empty((self.n_batch, self.n_part, 3), dtype=torch.float32, device=self.device)

    # ------------------------------------------------------------- C ABI --
    def set_cosmology(self, omega_m, sigma8):
        om = np.ascontiguousarray(np.broadcast_to(np.asarray(omega_m, np.float64), (self.n_batch,)))
        s8 = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma8, np.float64), (self.n_batch,)))
        if np.array_equal(om, self.omega_m) and np.array_equal(s8, self.sigma8):
            return
        self._call("pm_set_cosmology", _pmgb._dptr(om), _pmgb._dptr(s8))
        self.omega_m, self.sigma8 = om, s8

    def coefficients(self):
        out = np.zeros((self.n_batch, self.n_steps, 3))
        dout = np.zeros_like(out)
        self._call("pm_get_coefficients", _pmgb._dptr(out), _pmgb._dptr(dout))
        return out, dout

    def init_lpt(self, noise=None, seed=0):
        s, p = self.new_particles(), self.new_particles()
        if noise is not None:
            self._lattice(noise, "noise")
        self._call("pm_init_lpt", _ptr(noise), ctypes.c_uint64(seed), _ptr(s), _ptr(p))
        return s, p

    def init_lpt_adjoint(self, lam, mu, noise=None, seed=0, want_noise_grad=True):
        self._particles(lam, "lam")
        self._particles(mu, "mu")
        if noise is not None:
            self._lattice(noise, "noise")
        dnoise = torch.empty((self.n_batch, self.n_p, self.n_p, self.n_p), dtype=torch.float32,
                             device=self.device) if want_noise_grad else None
        dcos = np.zeros((self.n_batch, 2))
        self._call("pm_init_lpt_adjoint", _ptr(noise), ctypes.c_uint64(seed), _ptr(lam), _ptr(mu), _ptr(dnoise),
                   _pmgb._dptr(dcos))
        return dnoise, dcos

    def pm_force(self, s):
        self._particles(s, "s")
        f = self.new_particles()
        self._call("pm_force", _ptr(s), _ptr(f))
        return f

    def kdk_step(self, step, s, p, f):
        for t, n in ((s, "s"), (p, "p"), (f, "f")):
            self._particles(t, n)
        self._call("pm_kdk_step", int(step), _ptr(s), _ptr(p), _ptr(f))

    def integrate(self, s, p, step_begin=0, step_end=None, f=None):
        """In place: (s, p) at a[step_begin] -> a[step_end]; returns F(s)."""
        self._particles(s, "s")
        self._particles(p, "p")
        f = self.new_particles() if f is None else self._particles(f, "f")
        end = self.n_steps if step_end is None else step_end
        self._call("pm_integrate", int(step_begin), int(end), _ptr(s), _ptr(p), _ptr(f))
        return f

    def adjoint_integrate(self, s, p, f, lam, mu, step_begin=0, step_end=None, mu_zero=False):
        """In place, backward in time; returns dL/dOm of the dynamics."""
        for t, n in ((s, "s"), (p, "p"), (f, "f"), (lam, "lam"), (mu, "mu")):
            self._particles(t, n)
        end = self.n_steps if step_end is None else step_end
        dom = np.zeros(self.n_batch)
        self._call("pm_adjoint_integrate", int(step_begin), int(end), _ptr(s), _ptr(p), _ptr(f), _ptr(lam),
                   _ptr(mu), _pmgb._dptr(dom), _pmgb.PM_ADJ_MU_ZERO if mu_zero else 0)
        return dom

    def set_checkpoints(self, every):
        """Sparse checkpoints against FP32 reversal drift: integrate() keeps
        s_m and p_{m+1/2} at every `every`-th step in a device buffer that
        this object owns, and adjoint_integrate() restores them.  0 turns
        them off and frees the buffer.  Returns the buffer (or None)."""
        n = int(self._lib.pm_checkpoint_floats(self._ctx, int(every)))
        if n < 0:
            raise PMError("every must be >= 0")
        buf = torch.empty(n, dtype=torch.float32, device=self.device) if n > 0 else None
        self._call("pm_set_checkpoints", int(every), None if buf is None else _ptr(buf))
        self._ck_buf = buf
        return buf

    def density(self, s):
        self._particles(s, "s")
        d = torch.empty((self.n_batch, self.n_m, self.n_m, self.n_m), dtype=torch.float32, device=self.device)
        self._call("pm_density", _ptr(s), _ptr(d))
        return d

    def density_adjoint(self, s, ddelta):
        self._particles(s, "s")
        self._mesh(ddelta, "ddelta")
        ds = self.new_particles()
        self._call("pm_density_adjoint", _ptr(s), _ptr(ddelta), _ptr(ds))
        return ds

    def mse_loss(self, s, target, want_grad=True):
        self._particles(s, "s")
        self._mesh(target, "target")
        loss = np.zeros(self.n_batch)
        g = self.new_particles() if want_grad else None
        self._call("pm_mse_loss", _ptr(s), _ptr(target), _pmgb._dptr(loss), _ptr(g))
        return loss, g

    def power_spectrum(self, s):
        self._particles(s, "s")
        nb = self.n_m // 2
        k = np.zeros((self.n_batch, nb))
        pk = np.zeros_like(k)
        nm = np.zeros_like(k)
        self._call("pm_power_spectrum", _ptr(s), _pmgb._dptr(k), _pmgb._dptr(pk), _pmgb._dptr(nm))
        return k, pk, nm

    # ------------------------------------------- learned force correction --
    def nn_param_count(self):
        return int(self._lib.pm_nn_param_count())

    def nn_set_params(self, theta):
        """Upload the flat FP32 parameter vector (host) and reset Adam."""
        th = np.ascontiguousarray(np.asarray(theta, dtype=np.float32))
        if th.shape != (self.nn_param_count(),):
            raise PMError(f"theta must have {self.nn_param_count()} values, got {th.shape}")
        self._call("pm_nn_set_params", th.ctypes.data_as(ctypes.c_void_p))

    def nn_get_params(self):
        """(theta, last gradient) as float32 host arrays."""
        th = np.zeros(self.nn_param_count(), np.float32)
        g = np.zeros_like(th)
        self._call("pm_nn_get_params", th.ctypes.data_as(ctypes.c_void_p), g.ctypes.data_as(ctypes.c_void_p))
        return th, g

    def nn_enable(self, enable=True):
        """Add the network's correction to every force of pm_integrate / pm_kdk_step."""
        self._call("pm_nn_enable", int(bool(enable)))

    def nn_adam_step(self, lr, step):
        """One Adam step with the parameter gradient in the context (left by
        adjoint_integrate with the correction on, or by nn_train_step)."""
        self._call("pm_nn_adam_step", ctypes.c_double(lr), ctypes.c_int64(step))

    def nn_predict(self, s, a):
        self._particles(s, "s")
        df = self.new_particles()
        self._call("pm_nn_predict", _ptr(s), ctypes.c_double(a), _ptr(df))
        return df

    def nn_train_step(self, s, target, a, lr=1e-3, step=1, apply=True, weight=1.0):
        """Force-matching loss at (s, a) against target (returned unweighted);
        the gradient of weight * loss, then one Adam step when apply."""
        self._particles(s, "s")
        self._particles(target, "target")
        loss = ctypes.c_double(0.0)
        self._call("pm_nn_train_step", _ptr(s), _ptr(target), ctypes.c_double(a), ctypes.c_double(weight),
                   ctypes.c_double(lr),
                   ctypes.c_int64(step), int(bool(apply)), ctypes.byref(loss))
        return loss.value

    # ------------------------------------------------------- autotuner --
    TUNE_FAMILIES = ("paint", "read", "spectral", "fft_z", "fft_x", "z_staging", "z_fwd_staging", "x_round",
                     "pipeline", "deposit")

    def autotune(self, s):
        """Pick the fastest launch shape per kernel family on particles s;
        returns (chosen {family: value}, times [family][candidate] ms; the
        block-size families try 128, 256, 512 threads, fft_x widths 8, 16,
        z_staging 1 (loads) and 2 (TMA), z_fwd_staging 1 (strided loads) and
        2 (coalesced, staged), x_round 1 (x pass, spectral multiply and
        inverse x pass as three launches), 2 (one fused kernel) and 3 (fused
        for the force, three launches for the adjoint), pipeline 1 (force
        components as inverse transforms) and 2 (one inverse transform of
        the potential, then the 4-point difference on the real mesh),
        deposit 1 (zeroing and the atomic scatter) and 2 (particles binned
        by tile, each cell written once by the block that owns it))."""
        self._particles(s, "s")
        ms = np.zeros((len(self.TUNE_FAMILIES), 3), np.float32)
        self._call("pm_autotune", _ptr(s), ms.ctypes.data_as(ctypes.c_void_p))
        return self.get_tuning(), ms

    def get_tuning(self):
        t = np.zeros(len(self.TUNE_FAMILIES), np.int32)
        self._call("pm_get_tuning", t.ctypes.data_as(ctypes.c_void_p))
        return dict(zip(self.TUNE_FAMILIES, (int(v) for v in t)))

    def set_tuning(self, paint=256, read=256, spectral=256, fft_z=256, fft_x=8, z_staging=None, z_fwd_staging=1,
                   x_round=None, pipeline=None, deposit=None):
        """Fix the launch shapes; a family not named takes the context's
        default (z_staging keeps its current value, x_round and pipeline the
        defaults the context was created with, and so does deposit)."""
        if z_staging is None:
            z_staging = self.get_tuning()["z_staging"]
        if x_round is None:
            x_round = self._x_round_default
        if pipeline is None:
            pipeline = self._pipeline_default
        if deposit is None:
            deposit = self._deposit_default
        t = np.array([paint, read, spectral, fft_z, fft_x, z_staging, z_fwd_staging, x_round, pipeline, deposit],
                     np.int32)
        self._call("pm_set_tuning", t.ctypes.data_as(ctypes.c_void_p))

    def use_graphs(self, enable=True):
        """Replay pm_integrate / pm_adjoint_integrate from captured CUDA graphs."""
        self._call("pm_use_graphs", int(bool(enable)))

    def launch_count(self):
        return int(self._lib.pm_launch_count(self._ctx))

    def close(self):
        if self._ctx:
            self._lib.pm_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------ autograd ----

class _Simulate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, noise, omega_m, sigma8, pm):
        ctx.set_materialize_grads(False)
        pm.set_cosmology(omega_m.detach().cpu().numpy(), sigma8.detach().cpu().numpy())
        noise = noise.detach().contiguous()
        s, p = pm.init_lpt(noise)
        f = pm.integrate(s, p)
        ctx.pm = pm
        ctx.cosmo = (pm.omega_m.copy(), pm.sigma8.copy())
        ctx.cosmo_dev = (omega_m.device, sigma8.device)
        ctx.cosmo_dtype = (omega_m.dtype, sigma8.dtype)
        ctx.save_for_backward(noise, s, p, f)
        return s, p

    @staticmethod
    def backward(ctx, gs, gp):
        pm = ctx.pm
        noise, s, p, f = ctx.saved_tensors
        pm.set_cosmology(*ctx.cosmo)
        s, p = s.clone(), p.clone()
        lam = gs.contiguous().clone() if gs is not None else torch.zeros_like(s)
        mu = gp.contiguous().clone() if gp is not None else torch.zeros_like(p)
        dom = pm.adjoint_integrate(s, p, f, lam, mu, mu_zero=gp is None)
        dnoise, dcos = pm.init_lpt_adjoint(lam, mu, noise, want_noise_grad=ctx.needs_input_grad[0])
        g_om = torch.as_tensor(dom + dcos[:, 0], dtype=ctx.cosmo_dtype[0], device=ctx.cosmo_dev[0]) \
            if ctx.needs_input_grad[1] else None
        g_s8 = torch.as_tensor(dcos[:, 1], dtype=ctx.cosmo_dtype[1], device=ctx.cosmo_dev[1]) \
            if ctx.needs_input_grad[2] else None
        return dnoise, g_om, g_s8, None


class _Density(torch.autograd.Function):
    @staticmethod
    def forward(ctx, s, pm):
        ctx.pm = pm
        ctx.save_for_backward(s)
        return pm.density(s.detach().contiguous())

    @staticmethod
    def backward(ctx, gd):
        (s,) = ctx.saved_tensors
        return ctx.pm.density_adjoint(s, gd.contiguous()), None


def simulate(pm, noise, omega_m, sigma8):
    """Differentiable forward run: white noise (n_batch, n_p, n_p, n_p) and
    per-simulation Omega_m, sigma8 (float64 tensors of n_batch values) ->
    final displacement and momentum (n_batch, n_p^3, 3)."""
    return _Simulate.apply(noise, omega_m, sigma8, pm)


def density(pm, s):
    """Differentiable CIC density contrast (n_batch, n_m, n_m, n_m)."""
    return _Density.apply(s, pm)
