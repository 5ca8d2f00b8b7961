"""GB300 (sm_103a) implementation of the Scatman's Multi-Slice Fourier Transform.

The computation lives in ``libscatman.so`` (CUDA kernels behind the C ABI of
include/scatman.h); this package is its thin Python binding.  Importing it does
not load the library; the first call does, and fails loudly if the library has
not been built (``paper_2202_03411_gb300.build.build()``).
"""
from . import _lib, types
from .api import (Handle, ScatmanError, scatman_acquire, scatman_acquire_batch, scatman_backward, scatman_contraction_flops,
                  scatman_create, scatman_destroy,
                  scatman_device_bytes, scatman_elem_size, scatman_forward, scatman_forward_noalloc, scatman_get_occupancy,
                  scatman_get_q, scatman_get_slices, scatman_last_error, scatman_n_pix, scatman_param_count,
                  scatman_photon_counts, scatman_set_wait_limit, scatman_debug_fail_allocation, scatman_debug_stall, scatman_sync,
                  scatman_version, scatman_voxelise)
from .types import Geometry, Shape

__all__ = [
    "Handle", "ScatmanError", "scatman_acquire", "scatman_acquire_batch", "scatman_backward", "scatman_contraction_flops", "scatman_create", "scatman_destroy",
    "scatman_device_bytes", "scatman_elem_size", "scatman_forward", "scatman_forward_noalloc", "scatman_get_occupancy", "scatman_get_q",
    "scatman_get_slices", "scatman_last_error", "scatman_n_pix", "scatman_param_count", "scatman_photon_counts",
    "scatman_sync", "scatman_set_wait_limit", "scatman_debug_fail_allocation", "scatman_debug_stall", "Geometry", "Shape", "types",
    "scatman_version", "scatman_voxelise",
]
