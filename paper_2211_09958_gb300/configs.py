"""Named workloads (sizes, cosmology, seeds) of the PM hot path.

Each is fully synthetic: Gaussian white-noise initial conditions from a seed,
BBKS linear power, 2LPT at a = 1/64, growth-matched KDK to a = 1.
"""

from dataclasses import dataclass, field


@dataclass(frozen=True)
class Workload:
    name: str
    n_p: int
    n_m: int
    box: float
    n_steps: int
    n_batch: int = 1
    omega_m: float = 0.3
    sigma8: float = 0.8
    h: float = 0.7
    n_s: float = 0.96
    a_init: float = 1.0 / 64
    a_final: float = 1.0
    ic_seed: int = 0
    target_seed: int = 1
    notes: str = ""

    @property
    def particles(self):
        return self.n_batch * self.n_p ** 3


WORKLOADS = {
    w.name: w
    for w in (
        Workload("pm32_mesh64", 32, 64, 128.0, 10, ic_seed=0, target_seed=1,
                 notes="32^3 particles, 64^3 mesh, 128 Mpc/h, 10 steps"),
        Workload("pm128_mesh256", 128, 256, 256.0, 63, ic_seed=1234, target_seed=1235,
                 notes="128^3 particles, 256^3 mesh, 256 Mpc/h, 63 steps; MSE-density gradient"),
        Workload("pm512_mesh1024", 512, 1024, 1000.0, 100, ic_seed=2022, target_seed=2023,
                 notes="512^3 particles, 1024^3 mesh, 1 Gpc/h, 100 steps; forward + adjoint"),
        Workload("learned_pm128_mesh128", 128, 128, 256.0, 40, ic_seed=0, target_seed=1,
                 notes="coarse run of the learned-correction workload (box is a reading)"),
        Workload("batch32_pm64_mesh128", 64, 128, 128.0, 20, n_batch=32, ic_seed=5000, target_seed=6000,
                 notes="32 runs, Omega_m ~ U[0.2,0.4], sigma8 ~ U[0.6,1.0] (seed 99), seeds 5000+i"),
    )
}
