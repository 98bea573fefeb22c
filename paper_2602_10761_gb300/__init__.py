"""GB300 (sm_103a) library for the data-parallel hot path of point-particle
triboelectric charging in a turbulent channel (Wilms & Grosshans).

The compute path is the CUDA library libtribo.so (C ABI in include/tribo.h);
this package is its binding.  There is no CPU fallback: calls fail loudly when
the library is not built or no GPU is present.
"""
from ._abi import (  # noqa: F401
    TRIBO_FP64, TRIBO_MIXED, TRIBO_DRAG_STOKES, TRIBO_DRAG_SCHILLER_NAUMANN, TRIBO_DRAG_OFF,
    TRIBO_IMPACT_SPEED, TRIBO_IMPACT_NORMAL, TRIBO_DEV_ESCAPED, TRIBO_DEV_NONFINITE,
    TRIBO_DEV_OUTSIDE, TRIBO_DEV_TIMEOUT, TriboError, load, library_path, exported_names,
)
from .api import (  # noqa: F401
    Params, Particles, Channel, tribo_init, tribo_set_fluid, tribo_set_params, tribo_step,
    tribo_poisson, tribo_poisson_noalloc, tribo_stats, tribo_reset_stats, tribo_sync, tribo_error_bits,
    tribo_clear_error, tribo_test_pipeline_wait, tribo_launch_count, tribo_destroy, tribo_timing_enable, tribo_timing_read,
    tribo_phase_name, tribo_set_modes, tribo_eval_modes, tribo_adjoint, mean_charge, Batch, tribo_set_ssm,
    SSMParams, tribo_set_momentum_source, tribo_set_adjoint_memory, tribo_transfer_bytes,
)
