"""Training data, training loop and evaluation of the learned force
correction (include/pmgb.h pm_nn_*), all on the GPU through the library.

The paper names a learned optimisation of the PM gravity solver as work
built on pmwd (Statement of Need) without describing it.  Here the network
corrects the coarse-mesh PM force towards a reference PM run on a finer mesh
with more time steps:

  data       for each seed, the reference (mesh_factor x finer mesh,
             step_factor x more steps) is integrated from the same 2LPT start;
             at every coarse step time a_n its particles give one training
             sample (s, T = F_fine(s) - F_coarse(s), a_n)
  loss       force matching, mean over particles of |dF(s) - T|^2
             (pm_nn_train_step), Adam
  evaluate   the P(k) of the final density of the corrected coarse run
             against the reference, next to the plain coarse run and plain PM
             at 2x the coarse mesh, all measured on one mesh

Displacements are relative to a lattice offset by half a mesh cell, so the
same positions have different displacements in contexts with different
meshes: ``lattice_shift`` converts between them.
"""

import math
import time
from dataclasses import dataclass, field

import numpy as np
import torch

from .pm import ParticleMesh


def lattice_shift(src, dst):
    """Add to a displacement of context ``src`` to express the same positions
    in context ``dst`` (lattice q = i L / n_p + h / 2, h = L / n_m)."""
    return 0.5 * (src.box / src.n_m - dst.box / dst.n_m)


@dataclass
class LearnedSetup:
    n_p: int = 128
    n_m: int = 128
    box: float = 256.0
    n_steps: int = 40
    mesh_factor: int = 4
    step_factor: int = 4
    omega_m: float = 0.3
    sigma8: float = 0.8
    group: int = 4            # runs simulated together (context batch)

    def coarse(self, n_m=None, n_batch=None):
        b = self.group if n_batch is None else n_batch
        return ParticleMesh(self.n_p, self.n_m if n_m is None else n_m, self.box, [self.omega_m] * b,
                            [self.sigma8] * b, self.n_steps)

    def fine(self, n_batch=None):
        b = self.group if n_batch is None else n_batch
        return ParticleMesh(self.n_p, self.n_m * self.mesh_factor, self.box, [self.omega_m] * b,
                            [self.sigma8] * b, self.n_steps * self.step_factor)


def a_grid(pm):
    return pm.cfg.a_init + (pm.cfg.a_final - pm.cfg.a_init) * np.arange(pm.n_steps + 1) / pm.n_steps


def snapshots(setup, fine, coarse, seed):
    """Samples of ``fine.n_batch`` reference runs with seeds seed .. seed + B - 1:
    S, T of shape (n_steps + 1, B, n_p^3, 3) in the coarse context's
    displacements, and the scale factors a_n."""
    r = setup.step_factor
    n = coarse.n_steps
    shift = lattice_shift(fine, coarse)
    S = torch.empty((n + 1,) + tuple(coarse.new_particles().shape), dtype=torch.float32, device=coarse.device)
    T = torch.empty_like(S)
    s, p = fine.init_lpt(seed=seed)
    f = fine.pm_force(s)
    for k in range(n + 1):
        if k > 0:
            f = fine.integrate(s, p, r * (k - 1), r * k)
        torch.add(s, shift, out=S[k])
        torch.sub(f, coarse.pm_force(S[k]), out=T[k])
    return S, T, a_grid(coarse)


@dataclass
class TrainLog:
    losses: list = field(default_factory=list)      # per Adam step, relative to the sample's |T|^2
    samples: list = field(default_factory=list)     # snapshot index of each step
    base: list = field(default_factory=list)        # |T|^2 of each sample
    seconds_data: float = 0.0
    seconds_train: float = 0.0


def _init_theta(count, seed):
    """He-normal hidden layers, zero output layer and biases: the untrained
    network adds nothing to the PM force."""
    sizes = (32, 128, 128, 3)
    rng = np.random.Generator(np.random.PCG64(seed))
    out = []
    for li, (fi, fo) in enumerate(zip(sizes[:-1], sizes[1:])):
        w = rng.standard_normal(fi * fo) * math.sqrt(2.0 / fi) if li < len(sizes) - 2 else np.zeros(fi * fo)
        out += [w, np.zeros(fo)]
    theta = np.concatenate(out).astype(np.float32)
    if theta.size != count:
        raise ValueError(f"network has {count} parameters, initialiser made {theta.size}")
    return theta


def train(setup, seeds, epochs=3, lr=1e-3, lr_final=1e-4, init_seed=0, theta=None, log=None, weighted=True):
    """Train the correction on the reference runs of ``seeds`` (consumed
    ``setup.group`` at a time, each group's samples visited ``epochs`` times
    in a seeded random order, learning rate decaying geometrically from lr to
    lr_final; with ``weighted`` each sample's loss counts relative to its
    |T|^2); returns (theta, log)."""
    log = log or TrainLog()
    coarse, fine = setup.coarse(), setup.fine()
    if theta is None:
        theta = _init_theta(coarse.nn_param_count(), init_seed)
    coarse.nn_set_params(theta)
    groups = [seeds[i:i + setup.group] for i in range(0, len(seeds), setup.group)]
    total = len(groups) * epochs * (setup.n_steps + 1)
    rng = np.random.Generator(np.random.PCG64(init_seed + 7))
    step = 0
    for g in groups:
        if len(g) != setup.group or list(g) != list(range(g[0], g[0] + setup.group)):
            raise ValueError("seeds must come in consecutive groups of setup.group")
        t0 = time.perf_counter()
        S, T, a = snapshots(setup, fine, coarse, g[0])
        log.base += [float((T[k] ** 2).sum(-1).mean()) for k in range(len(a))]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        # each sample's loss relative to its own |T|^2, so that early times
        # (forces ~1e-5 of the late ones) weigh as much as late ones
        scale = [1.0 / max(b, 1e-30) for b in log.base[-len(a):]]
        for _ in range(epochs):
            for k in rng.permutation(len(a)):
                step += 1
                rate = lr * (lr_final / lr) ** ((step - 1) / max(total - 1, 1))
                log.losses.append(coarse.nn_train_step(S[k], T[k], float(a[k]), lr=rate, step=step,
                                                       weight=scale[k] if weighted else 1.0) * scale[k])
                log.samples.append(int(k))
        t2 = time.perf_counter()
        log.seconds_data += t1 - t0
        log.seconds_train += t2 - t1
        del S, T
    theta, _ = coarse.nn_get_params()
    coarse.close()
    fine.close()
    return theta, log


def _timed_integrate(pm, s, p):
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    pm.integrate(s, p)
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1) / 1e3


def evaluate(setup, theta, seeds):
    """P(k) errors of the final density against the reference for ``seeds``
    (one group): plain coarse, corrected coarse and plain PM at 2x the coarse
    mesh, all on the reference mesh; throughput of each run in
    particle-steps/s (warm second run, CUDA events)."""
    if len(seeds) != setup.group:
        raise ValueError("evaluate takes one group of seeds")
    fine = setup.fine()
    s_ref, p_ref = fine.init_lpt(seed=seeds[0])
    fine.integrate(s_ref, p_ref)
    k, pk_ref, _ = fine.power_spectrum(s_ref)
    runs = {}
    for name, n_m, nn in (("plain", setup.n_m, False), ("corrected", setup.n_m, True),
                          ("plain_2x", 2 * setup.n_m, False)):
        pm = setup.coarse(n_m=n_m)
        if nn:
            pm.nn_set_params(theta)
            pm.nn_enable(True)
        secs = None
        for _ in range(2):
            s, p = pm.init_lpt(seed=seeds[0])
            secs = _timed_integrate(pm, s, p)
        _, pk, _ = fine.power_spectrum(s + lattice_shift(pm, fine))
        runs[name] = {"pk": pk, "seconds": secs,
                      "particle_steps_per_s": pm.n_batch * pm.n_part * pm.n_steps / secs}
        pm.close()
    k_cut = 0.5 * math.pi * setup.n_m / setup.box       # half the coarse mesh's Nyquist
    sel = k[0] <= k_cut
    out = {"k": k[0], "pk_ref": pk_ref, "k_cut": k_cut}
    for name, r in runs.items():
        rel = r["pk"] / pk_ref - 1.0                       # per run and bin
        mean_rel = rel.mean(0)
        out[name] = {"max_abs_rel_err": float(np.max(np.abs(mean_rel[sel]))),
                     "rel_err": mean_rel, "seconds": r["seconds"],
                     "particle_steps_per_s": r["particle_steps_per_s"]}
    fine.close()
    return out


def reference_densities(setup, seeds, measure):
    """Final CIC density contrasts of the reference runs for ``seeds`` (one
    group), painted on the mesh of the context ``measure``."""
    fine = setup.fine()
    s, p = fine.init_lpt(seed=seeds[0])
    fine.integrate(s, p)
    d = measure.density(s + lattice_shift(fine, measure))
    fine.close()
    return d


def train_trajectory(setup, seeds, theta, steps=100, lr=3e-4, lr_final=3e-5, log=None):
    """Fine-tune the correction through the trajectory: each Adam step runs
    the corrected coarse simulations of one group of seeds (cycling through
    ``seeds``), takes the mean squared difference between their final density
    contrast and the reference's (painted on the coarse mesh), and
    differentiates it with the reverse-time adjoint of the corrected
    dynamics.  Returns (theta, losses)."""
    import numpy as np
    groups = [seeds[i:i + setup.group] for i in range(0, len(seeds), setup.group)]
    pm = setup.coarse()
    pm.nn_set_params(theta)
    pm.nn_enable(True)
    targets = [reference_densities(setup, g, pm) for g in groups]
    losses = []
    for step in range(1, steps + 1):
        k = (step - 1) % len(groups)
        s, p = pm.init_lpt(seed=groups[k][0])
        f = pm.integrate(s, p)
        loss, lam = pm.mse_loss(s, targets[k])
        losses.append(float(np.mean(loss)))
        pm.adjoint_integrate(s, p, f, lam, torch.zeros_like(p), mu_zero=True)
        rate = lr * (lr_final / lr) ** ((step - 1) / max(steps - 1, 1))
        pm.nn_adam_step(rate, step)
    theta, _ = pm.nn_get_params()
    pm.close()
    if log is not None:
        log.losses += losses
    return theta, losses
