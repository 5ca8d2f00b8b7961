"""ctypes declarations of include/scatman.h (argument marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libscatman.so")

SCATMAN_OK = 0
SCATMAN_ERR_ARG = -1
SCATMAN_ERR_OOM = -2
SCATMAN_ERR_CUDA = -3
SCATMAN_ERR_TIMEOUT = -4
SCATMAN_ERR_ADMISSION = -5
SCATMAN_ERR_STATE = -6
SCATMAN_ERR_UNSUPPORTED = -7
SCATMAN_ERR_CANCELLED = -8

STATUS_NAMES = {
    0: "OK", -1: "ERR_ARG", -2: "ERR_OOM", -3: "ERR_CUDA", -4: "ERR_TIMEOUT", -5: "ERR_ADMISSION",
    -6: "ERR_STATE", -7: "ERR_UNSUPPORTED", -8: "ERR_CANCELLED",
}

SCATMAN_FP64 = 0
SCATMAN_FP32 = 1
SCATMAN_TC_F16_SPLIT = 2
SCATMAN_TC_BF16_SPLIT = 3
SCATMAN_TC_F16 = 4
SCATMAN_TC_BF16 = 5

PRECISIONS = {
    "fp64": SCATMAN_FP64, "fp32": SCATMAN_FP32, "tc_f16_split": SCATMAN_TC_F16_SPLIT,
    "tc_bf16_split": SCATMAN_TC_BF16_SPLIT, "tc_f16": SCATMAN_TC_F16, "tc_bf16": SCATMAN_TC_BF16,
}

SCATMAN_MAX_LMAX = 12

SCATMAN_SPHERE, SCATMAN_ELLIPSOID, SCATMAN_SPHHARM, SCATMAN_RADIALMAP, SCATMAN_VOLUMEMAP = 0, 1, 2, 3, 4
SCATMAN_DETECTOR_FLAT, SCATMAN_DETECTOR_UNIFORM_Q = 0, 1

_D = ctypes.POINTER(ctypes.c_double)


class scatman_config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("voxel", ctypes.c_double), ("wavelength", ctypes.c_double), ("theta_max_deg", ctypes.c_double),
        ("det_nx", ctypes.c_int), ("det_ny", ctypes.c_int),
        ("q_list", _D), ("n_q", ctypes.c_longlong),
        ("precision", ctypes.c_int), ("soft", ctypes.c_int), ("soft_width", ctypes.c_double),
        ("scan_fp64", ctypes.c_int), ("detector", ctypes.c_int),
    ]


class scatman_shape(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("r", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
        ("R0", ctypes.c_double), ("lmax", ctypes.c_int), ("alm", _D),
        ("delta", ctypes.c_double), ("beta", ctypes.c_double),
        ("latitude", ctypes.c_double), ("longitude", ctypes.c_double), ("rotation", ctypes.c_double),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
        ("radial_map", _D), ("map_ntheta", ctypes.c_int), ("map_nphi", ctypes.c_int),
        ("volume_map", ctypes.POINTER(ctypes.c_ubyte)), ("map_nx", ctypes.c_int), ("map_ny", ctypes.c_int),
        ("map_nz", ctypes.c_int), ("map_dx", ctypes.c_double), ("map_delta", _D), ("map_beta", _D),
    ]


class scatman_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_longlong), ("slots", ctypes.c_int), ("precision", ctypes.c_int),
                ("soft_width", ctypes.c_double)]


class scatman_request(ctypes.Structure):
    _fields_ = [("geometry", scatman_config), ("shape", scatman_shape), ("target", ctypes.POINTER(ctypes.c_float)),
                ("want_gradient", ctypes.c_int), ("I_out", ctypes.POINTER(ctypes.c_float)), ("grad_out", _D),
                ("loss_out", _D)]


class scatman_server_stats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong), ("failed", ctypes.c_longlong),
                ("bytes_reserved", ctypes.c_longlong), ("bytes_reserved_peak", ctypes.c_longlong),
                ("inflight", ctypes.c_int), ("inflight_peak", ctypes.c_int), ("cancelled", ctypes.c_longlong)]


# name -> (restype, argtypes); every symbol include/scatman.h declares
SIGNATURES = {
    "scatman_create": (ctypes.c_int, [ctypes.POINTER(scatman_config), ctypes.c_void_p,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "scatman_voxelise": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(scatman_shape)]),
    "scatman_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "scatman_acquire": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(scatman_shape), ctypes.c_void_p]),
    "scatman_acquire_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(scatman_shape), ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_void_p)]),
    "scatman_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, _D]),
    "scatman_photon_counts": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_ulonglong, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_void_p]),
    "scatman_param_count": (ctypes.c_int, [ctypes.c_void_p]),
    "scatman_n_pix": (ctypes.c_longlong, [ctypes.c_void_p]),
    "scatman_elem_size": (ctypes.c_int, [ctypes.c_void_p]),
    "scatman_device_bytes": (ctypes.c_longlong, [ctypes.c_void_p]),
    "scatman_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "scatman_get_occupancy": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "scatman_get_slices": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "scatman_get_q": (ctypes.c_int, [ctypes.c_void_p, _D]),
    "scatman_contraction_flops": (ctypes.c_int, [ctypes.c_void_p, _D, _D]),
    "scatman_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "scatman_destroy": (None, [ctypes.c_void_p]),
    "scatman_version": (ctypes.c_char_p, []),
    "scatman_server_create": (ctypes.c_int, [ctypes.POINTER(scatman_server_config), ctypes.POINTER(ctypes.c_void_p)]),
    "scatman_server_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(scatman_request),
                                             ctypes.POINTER(ctypes.c_longlong)]),
    "scatman_server_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong, ctypes.c_double,
                                           ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)]),
    "scatman_server_stats_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(scatman_server_stats)]),
    "scatman_server_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "scatman_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double]),
    "scatman_debug_stall": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "scatman_debug_fail_allocation": (None, [ctypes.c_longlong]),
    "scatman_server_destroy": (None, [ctypes.c_void_p]),
    "scatman_footprint_bytes": (ctypes.c_longlong, [ctypes.POINTER(scatman_config)]),
    "scatman_forward_noalloc": (ctypes.c_int, [ctypes.POINTER(scatman_config), ctypes.POINTER(scatman_shape),
                                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Loads libscatman.so.  Raises if it has not been built: there is no
    fallback implementation."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(
                f"{path} is missing; build it with paper_2202_03411_gb300.build.build() "
                "(nvcc for sm_103a).  There is no CPU or PyTorch fallback.")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib
