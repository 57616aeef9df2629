"""GB300-native (sm_103a) CCPR time-domain adjoint gradient for density-based topology
optimisation of dispersive nanophotonic structures (arXiv 2305.00234).

The compute path is the CUDA library ``libfdtdccpr.so`` (C-ABI: include/fdtd_ccpr.h); this
package only marshals arguments to it.  There is no CPU fallback.
"""
from ._native import (FdtdError, fdtd_adjoint, fdtd_cancel, fdtd_create_grid, fdtd_destroy,  # noqa: F401
                      fdtd_filter_project, fdtd_filter_project_grad, fdtd_footprint_bytes, fdtd_forward,
                      fdtd_get_dft, fdtd_get_field, fdtd_get_gradient_constants, fdtd_gradient_static,
                      fdtd_inject_wait_timeout,
                      fdtd_get_index_map, fdtd_get_info, fdtd_get_timings, fdtd_gradient,
                      fdtd_gradient_norm, fdtd_last_error, fdtd_reset_timings, fdtd_set_density,
                      fdtd_set_materials, fdtd_set_profiling, load_library)
from .problem import Batch, Problem, box_shape, problem  # noqa: F401


def __getattr__(name):
    # torch is only needed for the autograd wrapper; import it on first use
    if name in ("FdtdGrad", "FilterProject", "objective", "checkpoint_bytes"):
        from . import grad
        return getattr(grad, name)
    raise AttributeError(name)
