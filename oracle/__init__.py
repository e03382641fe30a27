"""FP64 CPU oracle for the differentiable particle-mesh (PM) method of pmwd
(arXiv:2211.09958).

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code with the CUDA library under
``paper_2211_09958_gb300/``; the only thing both sides consume in common are
seeded input arrays made by ``paper_2211_09958_gb300.inputs``, which holds
none of the method's arithmetic.

The paper (a software summary) states the method in prose only: a
differentiable cosmological particle-mesh simulation (Summary), gradients by
the adjoint method with reverse time integration to recover the forward
history instead of storing it (Summary; Statement of Need), and the
discretize-then-optimize choice, i.e. gradients that run backward along the
same discrete trajectory as the forward integrator (Statement of Need).  It
prints no equations, so every formula here is a reading of that prose in the
standard comoving PM form; each reading is marked ``[reading]`` where it is
made.

Modules
-------
cosmology  growth functions, BBKS linear power, sigma8 normalisation, KDK
           coefficients and their Omega_m derivatives
philox     counter-based white noise (Philox4x32-10 + Box-Muller)
lpt        linear field and 2LPT initial conditions, and their adjoint
pm         CIC mass assignment / interpolation, spectral Poisson force,
           kick-drift-kick integration, reverse integration, the discrete
           adjoint, the density-MSE loss and the power-spectrum estimator

Parity status: every function is pinned by ``tests/test_oracle_*.py``
against closed forms, brute-force definitions, finite differences,
invariants or, for the Philox4x32-10 round function, the generator's
published known-answer vectors (bit for bit).  ``tests/test_oracle_mutants.py``
plants plausible mistakes one at a time and checks that each fails a pin.
Parity unpinned: the learned correction's architecture (features, layer
sizes, output scale), which is a design choice, not part of the method;
its arithmetic is pinned by finite differences.
"""

from .cosmology import Cosmology, growth, kdk_coefficients, linear_power  # noqa: F401
from . import philox, lpt, pm  # noqa: F401
