"""Benchmark of the differentiable PM hot path on GB300.

One bench step = the whole hot path over one synthetic realisation of the
workload: 2LPT initial conditions from white noise, forward KDK integration
over all time steps, MSE loss of the final CIC density against a target
field, the reverse-time adjoint back to a_init, and the adjoint of the
initial conditions (gradients w.r.t. the white noise, Omega_m and sigma8).
Metric: particle-steps/s = n_batch * n_p^3 * n_steps / time, forward +
adjoint together (also reported separately).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--sim-steps S]

--workload learned_pm128_mesh128 trains the learned force correction on
reference runs first (untimed), reports its P(k) gain, then times the
corrected forward integration.

With N > 1 (under torchrun) every rank runs an independent replica (the
path does not shard; no data-path collective), value = all ranks' work /
max time.  --impl reference times the FP64 CPU oracle instead.
"""

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2211_09958_gb300.configs import WORKLOADS  # noqa: E402

METRIC = "particle-steps/s (fwd+adjoint) at 512³"
LEARNED_WORKLOAD = "learned_pm128_mesh128"
LEARNED_METRIC = "particle-steps/s (learned-correction PM forward) at 128³ on a 128³ mesh"
UNIT = "particle-steps/s"
DEFAULT_WORKLOAD = "pm512_mesh1024"
ORACLE_SAMPLE = dict(n_p=64, n_m=128, box=125.0, n_steps=1)


# --------------------------------------------------------------- helpers --

def _dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"pm_bench_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# Algorithmic HBM bytes per launch of each library kernel (FP32 state,
# (N, 3) particle arrays; mesh bytes counted on the unpadded n_m^3 grid,
# complex modes on the n_m^2 (n_m/2+1) rfft grid).
def algorithmic_bytes(kind, npart, ncell, nmodes, pot_read=False):
    """pot_read: the CIC reads take the potential (and psi) meshes, one (two)
    float per cell, instead of the float4 force mesh (the library does with
    its default force pipeline, CIC and no learned correction)."""
    fmesh = 4 if pot_read else 12                         # mesh bytes per cell of a force read
    per = {
        "paint_density": 12 * npart + 4 * ncell,
        "paint_adj": 24 * npart + 16 * ncell,                # s, mu in; 4 fields out
        "read_force": 24 * npart + fmesh * ncell,
        "read_kick_drift": 48 * npart + fmesh * ncell,       # s, p in and out; phi or 3 force fields in
        "read_half_kick": 48 * npart + fmesh * ncell,        # s, p in; p, F out
        "read_adj": (48 + 48) * npart + (8 if pot_read else 16) * ncell,   # s, p, lam, mu in and out (fused drift)
        "read_grad": 24 * npart + 4 * ncell,
        "pre_rev_drift": 72 * npart,
        "pre_kick_drift": 60 * npart,
        "spectral_force": (8 + 24) * nmodes,
        "spectral_adj": (32 + 32) * nmodes,
        "grad_stencil_1": (4 + 16) * ncell,                  # phi in; (F, 0) float4 out
        "grad_stencil_2": (8 + 16) * ncell,                  # (phi, psi) in; (F, psi) out
        "vjp_source": (16 + 8) * ncell,                      # (rho, u) float4 in; (rho, v) out
        # binned deposit: binning (s in, tile and rank out; then the CSR
        # scatter), the tile-owned paint (the paint's own bytes: particles in,
        # every cell out once) and the halo pass (33 of 256 cells' halo lines
        # in; the 31 x = 0 / y = 0 lines of 256 read and written)
        "bin_count": 20 * npart,
        "bin_scan_sums": 4 * (ncell // 4096),
        "bin_scan": 12 * (ncell // 4096),
        "bin_scatter": 12 * npart,
        "deposit_density": 12 * npart + 4 * ncell,
        "deposit_adj": 24 * npart + 16 * ncell,
        "deposit_halo_1": (33 * 4 + 31 * 8) * ncell // 256,
        "deposit_halo_4": (33 * 16 + 31 * 32) * ncell // 256,
    }
    # own FFT passes: kind "fft_<axis>_<dir>_<fields>"
    if kind.startswith("fft_"):
        _, axis, direction, nf = kind.split("_")
        nf = int(nf)
        if axis == "z" and direction == "fwd":
            return nf * (4 * ncell + 8 * nmodes)          # real fields in, half spectra out
        if axis == "z":
            return nf * 8 * nmodes + (16 if nf >= 3 else 4 * nf) * ncell   # spectra in, real mesh out
        if direction == "round":                          # fused x pass: density in, 3 fields out; 4 in, 4 out
            return (8 + 24) * nmodes if nf == 1 else 64 * nmodes
        if direction == "pot":                            # potential x pass: 1 in, 1 out; 2 in, 2 out; 4 in, 2 out
            return {1: 16, 2: 32, 4: 48}[nf] * nmodes
        return nf * 16 * nmodes                             # pencil pass: read + write
    return per.get(kind)


def _source_digest():
    """Digest of the library sources that hold device code (kernels and the
    headers they include), comments and blank lines left out: a DRAM traffic
    capture stays valid while the code in them is unchanged.  Host-only
    orchestration files do not enter."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2211_09958_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh", ".cpp", ".h")):
            with open(os.path.join(csrc, f), "rb") as fh:
                text = fh.read()
            if b"__global__" in text or b"__device__" in text:
                code = re.sub(rb"/\*.*?\*/", b"", text, flags=re.S)
                code = re.sub(rb"//[^\n]*", b"", code)
                h.update(b"\n".join(line.rstrip() for line in code.splitlines() if line.strip()))
    return h.hexdigest()[:16]


def _ncu_traffic(kind, workload):
    """DRAM bytes per launch from the committed ncu capture, if it was taken
    on the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as fh:
        d = json.load(fh)
    if d.get("source_digest") != _source_digest():
        return None
    direct = d.get("direct", {}).get(workload, {}).get(kind)
    if direct:                                  # captured on this workload itself
        return float(direct["dram_bytes_per_launch"])
    ent = d.get("kernels", {}).get(kind)
    if not ent:
        return None
    scale = ent.get("scale_to", {}).get(workload)
    return ent["dram_bytes_per_launch"] * (scale if scale else 1.0) if (scale or ent.get("workload") == workload) else None


TRAFFIC_WORKLOAD = "pm128_mesh256"
TRAFFIC_COMMAND = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum "
                   "--clock-control none --kernel-name-base demangled -k regex:<kernel> -c 3 --csv "
                   "python bench.py --workload pm128_mesh256 --sim-steps 2 --steps 1 --warmup 1 "
                   "--no-cpu-baseline --no-autotune [--tuning deposit=2 for the binned-deposit kernels]")


def _kernel_kind(name, grid, n):
    """Launch kind of a library kernel from its ncu name (template arguments
    printed plain or with C-style casts) and grid."""
    m = re.search(r"(k_\w+)<([^>]*)>", name)
    if not m:
        m = re.search(r"(k_bin_count|k_bin_scatter)\b", name)
        return {"k_bin_count": "bin_count", "k_bin_scatter": "bin_scatter"}.get(m.group(1)) if m else None
    k = m.group(1)
    args = [re.sub(r"^\((int|bool)\)", "", a.strip()) for a in m.group(2).split(",")]
    zc = ((n // 2 + 1) + 7) // 8 * 8
    if k == "k_paint":
        return {"0": "paint_density", "2": "paint_adj"}.get(args[0])
    if k == "k_read":
        return {"0": "read_force", "1": "read_kick_drift", "2": "read_half_kick", "3": "read_adj",
                "4": "read_grad"}.get(args[0])
    if k == "k_deposit":
        return {"1": "deposit_density", "4": "deposit_adj"}.get(args[0])
    if k == "k_deposit_halo":
        return f"deposit_halo_{args[0]}"
    if k in ("k_fft_z_fwd", "k_fft_z_inv"):
        return f"fft_z_{k[-3:]}_{args[1]}"
    if k == "k_fft_xpot":
        return f"fft_x_pot_{args[1]}"
    if k in ("k_vjp_source", "k_vjp_source_x"):
        return "vjp_source"
    if k == "k_fft_pencil":
        blocks = int(grid.strip("()").split(",")[0])
        return f"fft_y_{'inv' if args[1] in ('1', 'true') else 'fwd'}_{blocks // (zc // 8 * n)}"
    return None


def traffic_digest(paths, out_path=None):
    """profiles/traffic.json from ncu CSV captures (TRAFFIC_COMMAND, one
    kernel per capture) on the 128^3 / 256^3 workload: mean DRAM bytes per
    launch of each kind, with the ratio to its algorithmic bytes and the
    factor that scales it to the other workloads."""
    import csv
    import collections
    launches = collections.OrderedDict()
    for path in paths:
        with open(path) as fh:
            rows = list(csv.reader(line for line in fh if line.startswith('"')))
        if not rows:
            continue
        hdr = rows[0]
        ki, mi, vi, gi, ii = (hdr.index(c) for c in ("Kernel Name", "Metric Name", "Metric Value", "Grid Size", "ID"))
        for r in rows[1:]:
            d = launches.setdefault((path, r[ii]), {"name": r[ki], "grid": r[gi]})
            d[r[mi]] = float(r[vi].replace(",", ""))
    src = WORKLOADS[TRAFFIC_WORKLOAD]

    def sizes(w):
        return (w.n_batch * w.n_p ** 3, w.n_batch * w.n_m ** 3, w.n_batch * w.n_m ** 2 * (w.n_m // 2 + 1))

    per = collections.defaultdict(list)
    for d in launches.values():
        kd = _kernel_kind(d["name"], d["grid"], src.n_m)
        if kd:
            per[kd].append(d.get("dram__bytes_read.sum", 0.0) + d.get("dram__bytes_write.sum", 0.0))
    if per.get("fft_x_pot_1") and not per.get("fft_x_pot_2"):  # two 1-field round trips per launch of its kind
        per["fft_x_pot_2"] = [2 * v for v in per["fft_x_pot_1"]]
    out = {"source_digest": _source_digest(), "command": TRAFFIC_COMMAND,
           "note": "mean DRAM bytes (read + write) per launch on the 128^3 / 256^3 workload, one capture per kernel; "
                   "scale_to multiplies by the ratio of algorithmic bytes per launch (the kernels' traffic grows in "
                   "proportion to particles, cells and modes); at 256^3 one mesh field fits in L2, so the scaled "
                   "figures are lower bounds for 1024^3",
           "kernels": {}, "direct": {}}
    for kd, vals in sorted(per.items()):
        ab = algorithmic_bytes(kd, *sizes(src))
        ent = {"dram_bytes_per_launch": sum(vals) / len(vals), "launches": len(vals), "workload": src.name}
        if ab:
            ent["algorithmic_bytes_per_launch"] = ab
            ent["ratio"] = round(ent["dram_bytes_per_launch"] / ab, 3)
            ent["scale_to"] = {w.name: algorithmic_bytes(kd, *sizes(w)) / ab for w in WORKLOADS.values()
                               if w.name != src.name and not getattr(w, "learned", False)}
        out["kernels"][kd] = ent
    with open(out_path or os.path.join(ROOT, "profiles", "traffic.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    return out


def replica_throughput(dist, world, work, steps, times_ms, device="cpu"):
    """Whole-job throughput of `world` independent replicas: each rank did
    `work` units per step for `steps` steps; the job took the slowest rank's
    time.  times_ms: this rank's timings (ms) -> (max over ranks of each,
    world * work * steps / max time for each)."""
    import torch
    t = list(times_ms)
    if dist is not None:
        buf = torch.tensor(t, dtype=torch.float64, device=device)
        dist.all_reduce(buf, op=dist.ReduceOp.MAX)
        t = [float(v) for v in buf]
    return t, [world * work * steps / (v / 1e3) for v in t]


def timed_steps(pm, stream, steps, step, barrier, profile=False, split=False):
    """Run `steps` bench steps between barriers, each bracketed by CUDA events
    on `stream`.  Without `profile` the library runs as a user calls it
    (integration loops replayed from its CUDA graphs); with `profile` it
    brackets every launch with its own event pair, which needs eager
    launches, and the per-kind table {kind: (launches, ms)} is returned.
    step(ev) runs one step; with `split` it records `ev` between the forward
    and the adjoint part.  -> (step_ms, forward_ms or None, launches, table)"""
    import ctypes
    import torch
    lib = pm._lib
    if profile:
        lib.pm_profile(pm._ctx, 1)
        lib.pm_profile_read(pm._ctx, None, None, 0)       # drop older records
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    barrier()
    launches0 = pm.launch_count()
    for k in range(steps):
        ev[k][0].record(stream)
        step(ev[k][1] if split else None)
        ev[k][2].record(stream)
    barrier()
    launches = pm.launch_count() - launches0
    table = None
    if profile:
        nk = lib.pm_profile_kinds(pm._ctx)
        counts = (ctypes.c_int64 * nk)()
        kms = (ctypes.c_double * nk)()
        lib.pm_profile_read(pm._ctx, counts, kms, nk)
        lib.pm_profile(pm._ctx, 0)
        table = {lib.pm_profile_name(pm._ctx, i).decode(): (int(counts[i]), float(kms[i])) for i in range(nk)}
    step_ms = [a.elapsed_time(c) for a, _, c in ev]
    fwd_ms = [a.elapsed_time(b) for a, b, _ in ev] if split else None
    return step_ms, fwd_ms, launches, table


PROFILED_NOTE = ("a second pass of the same steps with an event pair around every launch (eager launches, "
                 "no CUDA graphs); source of `kernels` and of the roofline's per-launch time")


# ----------------------------------------------------------------- oracle --

def oracle_sample(seed=0):
    """Time the FP64 oracle on a bounded sample: one KDK step forward and
    its adjoint step for 64^3 particles on a 128^3 mesh in a 125 Mpc/h box
    (the 512^3 / 1024^3 / 1 Gpc/h workload's recipe and resolution at 1/512
    of the particles)."""
    from oracle import pm as opm
    from oracle.cosmology import Cosmology
    from paper_2211_09958_gb300 import inputs

    smp = ORACLE_SAMPLE
    st = opm.Setup(smp["n_p"], smp["n_m"], smp["box"], Cosmology(0.3, 0.8), n_steps=smp["n_steps"])
    s0 = inputs.random_displacements(st.n_p, st.box, seed, scale=0.5).astype(np.float64)
    p0 = 0.01 * s0
    target = inputs.target_field(st.n_m, seed + 1).astype(np.float64)
    t0 = time.perf_counter()
    s, p, f = opm.integrate(s0, p0, st)
    t1 = time.perf_counter()
    lam = opm.mse_loss_grad(s, target, st)
    opm.adjoint_integrate(s, p, f, lam, np.zeros_like(p), st)
    t2 = time.perf_counter()
    work = st.n_p ** 3 * st.n_steps
    return {"value": work / (t2 - t0), "fwd_s": t1 - t0, "adj_s": t2 - t1, "seconds": t2 - t0}


LEARNED_SAMPLE = dict(n_p=64, n_m=64, box=128.0)
LEARNED_SAMPLE_TEXT = ("FP64 oracle (numpy + scipy.fft), one corrected force evaluation (PM force + per-cell MLP "
                       "correction, bf16 rounding points) for 64^3 particles on a 64^3 mesh, 128 Mpc/h (the "
                       "learned workload's resolution at 1/8 of its particles); particle-steps/s of that sample")


def oracle_learned_sample(seed=0):
    """Time the FP64 oracle's corrected force (PM force + network
    correction) on a bounded sample of the learned workload's resolution."""
    from oracle import learned as olearned
    from oracle import pm as opm
    from oracle.cosmology import Cosmology
    from paper_2211_09958_gb300 import inputs

    smp = LEARNED_SAMPLE
    st = opm.Setup(smp["n_p"], smp["n_m"], smp["box"], Cosmology(0.3, 0.8))
    s = inputs.random_displacements(st.n_p, st.box, seed, scale=0.5).astype(np.float64)
    theta = inputs.mlp_params((32, 128, 128, 3), seed=seed).astype(np.float64)
    t0 = time.perf_counter()
    opm.force(s, st) + olearned.predict(s, 0.5, theta, st)
    dt = time.perf_counter() - t0
    return {"value": st.n_p ** 3 / dt, "seconds": dt}


def _cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


SAMPLE_TEXT = ("FP64 oracle (numpy + scipy.fft), one forward KDK step plus its adjoint step, "
               "64^3 particles on a 128^3 mesh, 125 Mpc/h (the 512^3 workload's recipe and resolution "
               "at 1/512 of its particles), 2LPT excluded; particle-steps/s of that sample")


def run_reference(args):
    rank, _, world = _dist_env()
    if world > 1 and rank != 0:
        return 0
    w = WORKLOADS[args.workload]
    learned = w.name == LEARNED_WORKLOAD
    sample_fn = oracle_learned_sample if learned else oracle_sample
    for _ in range(args.warmup):
        sample_fn()
    times, vals = [], []
    for k in range(args.steps):
        r = sample_fn(seed=k)
        times.append(r["seconds"])
        vals.append(r["value"])
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": LEARNED_METRIC if learned else METRIC, "value": value, "unit": UNIT,
        "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(times)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w.name, "sample": LEARNED_SAMPLE if learned else ORACLE_SAMPLE},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _cores(), "kind": "oracle",
                         "sample": LEARNED_SAMPLE_TEXT if learned else SAMPLE_TEXT},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------------- ours --

def run_ours(args):
    rank, local_rank, world = _dist_env()
    w = WORKLOADS[args.workload]
    n_steps = args.sim_steps or w.n_steps

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        runs = [oracle_sample(seed=k) for k in range(2)]      # before any GPU call
        cpu = {"value": float(np.mean([r["value"] for r in runs]))}

    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")

    from paper_2211_09958_gb300 import _pmgb
    from paper_2211_09958_gb300.pm import ParticleMesh

    if w.n_batch > 1:
        from paper_2211_09958_gb300.inputs import batch_cosmologies
        om, s8 = batch_cosmologies(w.n_batch)
    else:
        om, s8 = w.omega_m, w.sigma8
    pm = ParticleMesh(w.n_p, w.n_m, w.box, om, s8, n_steps, w.a_init, w.a_final, w.h, w.n_s)
    dev = pm.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.ic_seed + 7919 * rank)
    noise = torch.randn((pm.n_batch, w.n_p, w.n_p, w.n_p), generator=gen, device=dev, dtype=torch.float32)
    target = torch.randn((pm.n_batch, w.n_m, w.n_m, w.n_m), generator=gen, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()

    def hot_path(nz, tg, ev=None):
        s, p = pm.init_lpt(nz)
        f = pm.integrate(s, p)
        if ev is not None:
            ev.record(stream)
        loss, lam = pm.mse_loss(s, tg)
        mu = torch.zeros_like(p)
        dom = pm.adjoint_integrate(s, p, f, lam, mu, mu_zero=True)
        dn, dcos = pm.init_lpt_adjoint(lam, mu, nz)
        return dn, loss, dom, dcos

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    tuning = pm.get_tuning()
    if args.tuning:                                       # fixed launch shapes (e.g. those a plain run picked)
        pm.set_tuning(**{**tuning, **args.tuning})
        tuning = pm.get_tuning()
    elif not args.no_autotune:                            # untimed: the library's own launch-shape tuner
        s_t, _ = pm.init_lpt(noise)
        tuning, _ = pm.autotune(s_t)
        del s_t
    for _ in range(args.warmup):
        hot_path(noise, target)
    barrier()

    # device-resident timing: the production pass gives the value, a second
    # pass with per-launch events gives the kernel table and the roofline
    def step(ev):
        hot_path(noise, target, ev)

    with ClockSampler(torch.cuda.current_device()) as clocks:
        step_ms, fwd_ms, launches, _ = timed_steps(pm, stream, args.steps, step, barrier, split=True)
        prof_ms, _, _, kernels = timed_steps(pm, stream, args.steps, step, barrier, profile=True)
    total_ms = float(sum(step_ms))
    prof_total = float(sum(prof_ms))

    # end to end: pinned host inputs in, gradient out, every step
    h_noise = noise.cpu().pin_memory()
    h_target = target.cpu().pin_memory()
    h_grad = torch.empty_like(h_noise).pin_memory()
    hot_path(h_noise.to(dev, non_blocking=True), h_target.to(dev, non_blocking=True))
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        dn, loss, dom, dcos = hot_path(h_noise.to(dev, non_blocking=True), h_target.to(dev, non_blocking=True))
        h_grad.copy_(dn, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    h2d = h_noise.numel() * 4 + h_target.numel() * 4
    d2h = h_grad.numel() * 4 + 8 * pm.n_batch * 4        # dnoise + loss, dOm (dyn, IC), dsigma8

    work = pm.n_batch * w.n_p ** 3 * n_steps            # particle-steps per rank per bench step
    (t_max, e2e_max), (value, e2e_value) = replica_throughput(dist, world, work, args.steps, (total_ms, e2e_ms), dev)

    if rank == 0:
        hbm, peak_src = _peaks()
        npart, ncell, nmodes = pm.n_batch * w.n_p ** 3, pm.n_batch * w.n_m ** 3, pm.n_batch * w.n_m ** 2 * (w.n_m // 2 + 1)
        pot_read = tuning.get("pipeline") == 2 and (w.n_m & (w.n_m - 1)) == 0
        table = {}
        for kind, (cnt, ms) in kernels.items():
            ab = algorithmic_bytes(kind, npart, ncell, nmodes, pot_read)
            ent = {"launches": cnt, "total_ms": round(ms, 3), "share": round(ms / prof_total, 4)}
            if ab is not None and cnt:
                ent["gbs"] = round(ab / (ms / cnt / 1e3) / 1e9, 1)
                ent["frac"] = round(ent["gbs"] / hbm, 3)
            table[kind] = ent
        mine = {k: v for k, v in table.items() if "gbs" in v}
        dom_kind = max(mine, key=lambda k: mine[k]["total_ms"])
        dk = mine[dom_kind]
        cnt, ms = kernels[dom_kind]
        traffic = _ncu_traffic(dom_kind, w.name)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "n_p": w.n_p, "n_m": w.n_m, "box_mpc_h": w.box, "n_steps": n_steps,
                       "n_batch": pm.n_batch, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (each mesh field > 129 MB)" if pm.n_batch * w.n_m ** 3 * 4 > 129e6
                       else "working set per pass < L2; not flushed", "tuning": tuning},
            "forward": {"value": world * work * args.steps / (sum(fwd_ms) / 1e3), "unit": UNIT,
                        "ms_per_step": float(np.mean(fwd_ms))},
            "adjoint": {"value": world * work * args.steps / ((total_ms - sum(fwd_ms)) / 1e3), "unit": UNIT,
                        "ms_per_step": float(np.mean(step_ms) - np.mean(fwd_ms))},
            "roofline": {"bound": "hbm", "kernel": dom_kind, "achieved": dk["gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": dk["frac"], "peak_source": peak_src,
                         "algorithmic_bytes_per_launch": algorithmic_bytes(dom_kind, npart, ncell, nmodes, pot_read),
                         "traffic": traffic},
            "kernels": table,
            "profiled": {"ms_per_step": prof_total / args.steps, "pass": PROFILED_NOTE},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)},
            "cpu_baseline": None if cpu is None else {
                "value": cpu["value"], "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": SAMPLE_TEXT},
        }
        print(json.dumps(line))
    pm.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_learned(args):
    """The learned-correction workload: train the network on reference runs
    (untimed), evaluate its P(k) gain, then time the corrected forward
    integration of a batch of 4 runs (2LPT + 40 corrected KDK steps)."""
    rank, local_rank, world = _dist_env()
    w = WORKLOADS[args.workload]
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = {"value": float(np.mean([oracle_learned_sample(seed=k)["value"] for k in range(2)]))}
    import torch
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2211_09958_gb300 import learn

    st = learn.LearnedSetup(n_p=w.n_p, n_m=w.n_m, box=w.box, n_steps=w.n_steps, group=4)
    t0 = time.perf_counter()
    seeds = list(range(100 + 1000 * rank, 100 + 1000 * rank + args.learn_runs))
    theta, log = learn.train(st, seeds, epochs=args.learn_epochs, lr=1e-3, lr_final=1e-4)
    train_s = time.perf_counter() - t0
    ev = learn.evaluate(st, theta, [90000 + 4 * rank + j for j in range(4)])

    pm = st.coarse()
    pm.nn_set_params(theta)
    pm.nn_enable(True)
    dev = pm.device
    gen = torch.Generator(device=dev)
    gen.manual_seed(w.ic_seed + 7919 * rank)
    noise = torch.randn((pm.n_batch, w.n_p, w.n_p, w.n_p), generator=gen, device=dev, dtype=torch.float32)
    stream = torch.cuda.current_stream()
    tuning = pm.get_tuning()
    if args.tuning:
        pm.set_tuning(**{**tuning, **args.tuning})
        tuning = pm.get_tuning()
    elif not args.no_autotune:
        s_t, _ = pm.init_lpt(noise)
        tuning, _ = pm.autotune(s_t)
        del s_t

    def hot_path(nz):
        s, p = pm.init_lpt(nz)
        pm.integrate(s, p)
        return s

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        hot_path(noise)
    barrier()
    with ClockSampler(torch.cuda.current_device()) as clocks:
        step_ms, _, launches, _ = timed_steps(pm, stream, args.steps, lambda ev: hot_path(noise), barrier)
        prof_ms, _, _, kernels = timed_steps(pm, stream, args.steps, lambda ev: hot_path(noise), barrier,
                                             profile=True)
    total_ms = float(sum(step_ms))
    prof_total = float(sum(prof_ms))

    # end to end: noise from pinned host memory in, final displacements out
    h_noise = noise.cpu().pin_memory()
    h_s = torch.empty((pm.n_batch, pm.n_part, 3), dtype=torch.float32).pin_memory()
    hot_path(h_noise.to(dev, non_blocking=True))
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        h_s.copy_(hot_path(h_noise.to(dev, non_blocking=True)), non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)

    work = pm.n_batch * w.n_p ** 3 * w.n_steps
    (t_max, e2e_max), (value, _) = replica_throughput(dist, world, work, args.steps, (total_ms, e2e_ms), dev)
    if rank == 0:
        d = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        peak = float(d.get("bf16_tflops_sustained", 1700.0))
        cells = pm.n_batch * w.n_m ** 3
        flops = 2.0 * (32 * 128 + 128 * 128 + 128 * 3) * cells     # algorithmic MLP flops per evaluation
        cnt, ms = kernels.get("nn_fwd_tc", (0, 0.0))
        achieved = flops / (ms / cnt / 1e3) / 1e12 if cnt else None
        table = {k: {"launches": c, "total_ms": round(m, 3), "share": round(m / prof_total, 4)}
                 for k, (c, m) in kernels.items()}
        line = {
            "metric": LEARNED_METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
            "config": {"workload": w.name, "n_p": w.n_p, "n_m": w.n_m, "box_mpc_h": w.box, "n_steps": w.n_steps,
                       "n_batch": pm.n_batch, "parallelism": "replicas" if world > 1 else "single",
                       "l2": "mesh and particle working set > L2 per step (4 x 128^3 x 16 B meshes)",
                       "tuning": tuning},
            "roofline": {"bound": "tensor", "kernel": "nn_fwd_tc", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                         "peak_source": "measured (bf16, sustained)",
                         "algorithmic_flops_per_launch": flops, "traffic": _ncu_traffic("nn_fwd_tc", w.name)},
            "learned": {
                "train_runs": args.learn_runs, "epochs": args.learn_epochs, "train_seconds": round(train_s, 1),
                "k_cut_h_per_mpc": ev["k_cut"],
                "pk_max_abs_rel_err": {k: ev[k]["max_abs_rel_err"] for k in ("plain", "corrected", "plain_2x")},
                "particle_steps_per_s": {k: ev[k]["particle_steps_per_s"] for k in ("plain", "corrected", "plain_2x")},
                "reference": "PM on a 4x finer mesh with 4x the steps, same 2LPT start",
            },
            "kernels": table,
            "profiled": {"ms_per_step": prof_total / args.steps, "pass": PROFILED_NOTE},
            "gpu_launches": int(launches),
            "clocks": clocks.summary(),
            "e2e": {"value": world * work * args.steps / (e2e_max / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": int(h_noise.numel() * 4), "d2h_bytes_per_step": int(h_s.numel() * 4)},
            "cpu_baseline": None if cpu is None else {
                "value": cpu["value"], "unit": UNIT, "cores": _cores(), "kind": "oracle", "sample": LEARNED_SAMPLE_TEXT},
        }
        print(json.dumps(line))
    pm.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_paint_stress(args):
    """Paint and read kernels on a clustered state (half of the particles in
    1 % of the volume) against the 2LPT state of the same workload: the last
    KDK step and its adjoint, per-launch event timing, K repetitions after W
    warm-up ones.  Prints one JSON line (a kernel measurement, not a bench
    line)."""
    import torch
    from paper_2211_09958_gb300 import inputs
    from paper_2211_09958_gb300.pm import ParticleMesh

    w = WORKLOADS[args.workload]
    t0 = time.time()
    s_cl = torch.from_numpy(inputs.clustered_displacements(w.n_p, w.box, seed=w.ic_seed)).cuda()[None]
    gen_s = time.time() - t0
    pm = ParticleMesh(w.n_p, w.n_m, w.box, w.omega_m, w.sigma8, w.n_steps, w.a_init, w.a_final, w.h, w.n_s)
    gen = torch.Generator(device=pm.device)
    gen.manual_seed(w.ic_seed)
    noise = torch.randn((1, w.n_p, w.n_p, w.n_p), generator=gen, device=pm.device, dtype=torch.float32)
    s_lpt, p_lpt = pm.init_lpt(noise)
    if not args.no_autotune:
        pm.autotune(s_lpt)
    stream = torch.cuda.current_stream()
    last = w.n_steps - 1
    kinds = ("paint_density", "paint_adj", "read_kick_drift", "read_half_kick", "read_adj")
    out = {}
    for name, s0 in (("uniform", s_lpt), ("clustered", s_cl)):
        p0 = p_lpt
        s, p, f = s0.clone(), p0.clone(), pm.new_particles()
        lam, mu = torch.randn_like(s), torch.randn_like(p)

        def step(ev):
            s.copy_(s0)
            p.copy_(p0)
            pm.integrate(s, p, last, w.n_steps, f)
            pm.adjoint_integrate(s, p, f, lam, mu, last, w.n_steps)

        for _ in range(args.warmup):
            step(None)
        _, _, _, table = timed_steps(pm, stream, args.steps, step, torch.cuda.synchronize, profile=True)
        out[name] = {k: table[k] for k in kinds if k in table}
    res = {}
    for k in kinds:
        if k in out["uniform"] and k in out["clustered"]:
            (cu, mu_), (cc, mc) = out["uniform"][k], out["clustered"][k]
            res[k] = {"uniform_ms_per_launch": round(mu_ / cu, 4), "clustered_ms_per_launch": round(mc / cc, 4),
                      "clustered_over_uniform": round((mc / cc) / (mu_ / cu), 3), "launches": cc}
    print(json.dumps({"measurement": "paint/read kernels on a clustered state (1/2 of the particles in 1 % of "
                                     "the volume) vs the 2LPT state", "workload": w.name, "steps": args.steps,
                      "warmup": args.warmup, "tuning": pm.get_tuning(), "host_generation_s": round(gen_s, 1),
                      "kernels": res}))
    pm.close()
    return 0


def _tuning_arg(text):
    """'family=value,...' -> {family: int}."""
    out = {}
    for item in text.split(","):
        k, _, v = item.partition("=")
        out[k.strip()] = int(v)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD, choices=sorted(WORKLOADS))
    ap.add_argument("--sim-steps", type=int, default=0, help="override the number of KDK steps")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--tuning", type=_tuning_arg, default=None,
                    help="fixed launch shapes instead of the autotuner, e.g. paint=512,read=128,x_round=3")
    ap.add_argument("--learn-runs", type=int, default=32, help="reference runs the correction trains on")
    ap.add_argument("--learn-epochs", type=int, default=3)
    ap.add_argument("--paint-stress", action="store_true",
                    help="time the paint and read kernels on a clustered state instead of the bench step")
    ap.add_argument("--traffic-from", nargs="+", metavar="CSV",
                    help="write profiles/traffic.json from ncu DRAM-byte captures (no GPU work)")
    args = ap.parse_args()
    if args.traffic_from:
        d = traffic_digest(args.traffic_from)
        print(json.dumps({k: v.get("ratio") for k, v in d["kernels"].items()}))
        return 0
    if args.paint_stress:
        return run_paint_stress(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == LEARNED_WORKLOAD:
        return run_learned(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
