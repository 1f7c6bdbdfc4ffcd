"""GB300-native SPH neighbour-sum path of Bonsai-SPH (arXiv 1909.07439).

The computation lives in the CUDA library ``lib/libsph.so`` (C ABI declared
in ``include/sph.h``); this package builds it (``build``), binds it with the
same function names (``native``), holds device state in torch tensors
(``state``) and draws seeded synthetic inputs (``inputs``).
"""
from . import inputs  # noqa: F401
from .native import (NativeLibraryMissing, SphError, load, sph_batch_evaluate,  # noqa: F401
                     sph_batch_step, sph_build_tree, sph_conserved, sph_conserved_noalloc,
                     sph_density_bwd, sph_force_bwd, sph_rollout,
                     sph_create, sph_density, sph_destroy, sph_force, sph_get_stats,
                     sph_get_timing, sph_get_tree, sph_last_error, sph_neighbours, sph_params,
                     sph_params_default, sph_set_timing, sph_state, sph_step, sph_step_host,
                     sph_sync, sph_test_lookback_timeout, sph_timestep)
from .state import DeviceState  # noqa: F401
