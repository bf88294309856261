"""FP64 CPU oracle for the k-space pseudospectral time step.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may call it.  It shares no code, table or helper with the CUDA
library; both sides receive the same seeded inputs from the input generators
and compute everything else on their own.

The oracle follows the paper (Jaros, Rendell, Treeby, "Full-wave nonlinear
ultrasound simulation on distributed clusters with applications in HIFU"):

* Sec. 2.2, Eqs. 4a-4d  -- staggered spectral gradients and the k-space
  corrected leapfrog updates of velocity and split density,
* Eq. 5                 -- wavenumber grid,
* kappa = sinc(c_ref k dt / 2) (Sec. 2.2, text after Eq. 5),
* Eq. 6                 -- nonlinear pressure-density relation,
* Eq. 8 (with Eq. 3)    -- discrete power-law absorption / dispersion term,

in that order, in float64, using whole-grid complex FFTs (numpy/scipy) as the
only library primitive.  Every reading where the paper is silent is listed in
``kspace.py``'s module docstring.

Pinned by ``tests/test_oracle_*.py`` (closed forms, invariants, physics).  The
adjoint functions in ``adjoint.py`` are pinned by a dot-product test and by
finite differences of the forward oracle.
"""

from .kspace import (  # noqa: F401
    Grid, Simulation, wavenumbers, kappa, apply_operator, pml_profile,
    NONLINEAR, ABSORBING, P_MAX, P_RMS, I_AVG, P_MIN, P_SERIES, U_SERIES, ADDITIVE_MASS, FORCE_X, FORCE_Y, FORCE_Z,
    DIRICHLET_P,
    OP_GRAD_FWD, OP_DIV_BWD, OP_ABS_TAU, OP_ABS_ETA,
)
from . import adjoint  # noqa: F401,E402
