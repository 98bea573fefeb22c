"""FP64 CPU oracle of the channel-flow tribocharging hot path.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check of the package
entry point and the CPU-baseline leg of the benchmark may import or run this
package.  The CUDA library never calls it and shares no code with it: this
package holds its own grid arithmetic, its own Poisson solver (numpy FFT in x,
z plus a plain Thomas sweep in y), its own interpolation, drag, integrator and
charging formulas, all in FP64 numpy, written to be checked against the paper
by eye.

Modules
  constants  -- Table 1 material constants and model switches
  grid       -- cells, locate, wall-extended lattice, trilinear gather
  poisson    -- deposition, FV Poisson operator and solver, E = -grad(phi)
  particles  -- drag, exponential integrator, wall impacts, condenser charge,
                the coupled step, statistics
  adjoint    -- parameter gradients of the mean charge (reference values)
Every function names the passage of the paper it follows.  Readings of
passages that are silent or garbled are listed in the docstrings as
"reading:".
"""
from .constants import Params, TABLE1  # noqa: F401
from .grid import Grid, locate, trilinear  # noqa: F401
from .poisson import deposit, poisson, efield, fv_apply, dense_poisson  # noqa: F401
from .particles import (  # noqa: F401
    State, relaxation_time, push, wrap, wall_impacts, condenser_wall, step, run, momentum_source,
    ystats, particle_mass, coulomb_near, pp_charge, pp_collisions,
)
