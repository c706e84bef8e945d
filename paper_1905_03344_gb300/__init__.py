"""GB300-native hot path of one SPH timestep (SPH-EXA mini-app, arXiv 1905.03344).

Neighbour discovery into CSR lists, density and equation of state, momentum
and energy with artificial viscosity, Courant time-step and leapfrog /
Adams-Bashforth update, for one or many square patches, as hand-written CUDA
for sm_103a behind the C ABI in include/sph.h.

  * ``binding``  -- the Python binding of the C ABI (``SPH`` and ``sph_*``)
  * ``inputs``   -- seeded synthetic square-patch inputs (numpy)
  * ``build``    -- compiles libsph_gb300.so in-tree with nvcc
"""
from . import inputs  # noqa: F401
from .binding import SPH, SphError, FIELDS, PHASES  # noqa: F401
