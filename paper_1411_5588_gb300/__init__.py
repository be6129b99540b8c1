"""GB300-native Ising-film Monte Carlo (arXiv:1411.5588 hot path).

The checkerboard Metropolis sweep of the Eq. 1 film with the Eq. 11 boundary
and its int64 observable sums run in hand-written CUDA kernels for sm_103a
behind the C ABI of ``include/ising.h``; this package is the ctypes binding
(``binding``) and the in-tree build (``build``).
"""
from .binding import (  # noqa: F401
    EBUSY, ECUDA, EINVAL, ENOMEM, ENOTFOUND, ETIMEOUT, INIT_ALL_UP, INIT_RANDOM, INIT_SLAB_Y, MAX_LANES, OK, SHAPE_AUTO,
    SHAPE_CLUSTER, SHAPE_GRID_1, SHAPE_GRID_2, SHAPE_GRID_Q, SHAPE_RESIDENT, X_FREE, X_PBC, Y_APBC, Y_GAPBC, Y_PBC, Batch, Film, IsingError,
    Server, check, check_counters, gauss_legendre, lib, make_jobs, series_energy, series_mean, ti_beta_trapezoid,
    ti_surface_field, ti_temperature_trapezoid)
