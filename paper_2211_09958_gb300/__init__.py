"""GB300-native differentiable particle-mesh N-body core (pmwd hot path).

The compute runs in ``_lib/libpmgb.so`` (hand-written sm_103a CUDA kernels
plus cuFFT) behind the C ABI of ``include/pmgb.h``; this package is its thin
Python binding.  Importing the package does not load the library; the first
``ParticleMesh`` does, and fails loudly if it is missing.
"""

from .configs import WORKLOADS, Workload  # noqa: F401


def __getattr__(name):
    if name in ("ParticleMesh", "simulate", "density", "PMError"):
        from . import pm
        return getattr(pm, name)
    raise AttributeError(name)
