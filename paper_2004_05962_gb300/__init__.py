"""GB300-native (sm_103a) cubic B-spline interpolation of FFD control grids.

The C ABI is ``include/bsi.h``; ``bsi`` is its Python binding (same names),
``autograd.field`` the differentiable wrapper, ``synth`` the seeded workload
generators and ``model`` the traffic / operation-count models.
"""
from .bsi import (  # noqa: F401
    BsiError,
    BsiLibraryMissing,
    bsi_adjoint_workspace_bytes,
    bsi_batched_adjoint_workspace_bytes,
    bsi_check_device_status,
    bsi_field_adjoint,
    bsi_field_adjoint_batched,
    bsi_field_forward,
    bsi_field_forward_batched,
    bsi_field_adjoint_rational,
    bsi_field_forward_rational,
    bsi_rational_adjoint_workspace_bytes,
    bsi_field_forward_variant,
    bsi_field_adjoint_noalloc,
    bsi_get_tile_config,
    bsi_probe_fill,
    bsi_resample_backward,
    bsi_resample_backward_workspace_bytes,
    bsi_resample_forward,
    bsi_scalar_forward,
    bsi_selfcheck_ranges,
    bsi_selftest_lost_copy,
    bsi_set_tile_configs,
    bsi_tile_configs,
    grid_shape,
    rational_grid_shape,
    library,
)
from .autograd import BSIField, BSIFieldRational, BSIResample, field, field_rational, resample  # noqa: F401
