"""GB300-native data-driven GMRES for 2D FDFD Maxwell solves.

The compute path is the CUDA library libddgmres.so (C ABI in include/ddgmres.h);
`binding` is its thin ctypes binding with the same function names, and
`inputs` draws the seeded synthetic problems.  Importing the package loads
nothing; the first binding call loads the library and raises if it is missing.
"""
from . import inputs  # noqa: F401
from .binding import (  # noqa: F401
    Context, DdgError, Operator, augmented_gmres_solve, augmented_gmres_solve_batched, gmres_solve_noalloc,
    ddg_context_create, fdfd_apply, fdfd_solve_host, fdfd_apply_c64, fdfd_operator, fdfd_source, gmres_solve,
    gmres_solve_batched, gmres_solve_queue, gmres_solve_queue_trajectories, gmres_solve_trajectories, load, make_grid, pca_fit, Predictor, predictor_create,
)
