"""Thin Python binding of the C ABI, one function per C entry point.

Device memory and streams come from PyTorch (tensors' data pointers and
``torch.cuda.current_stream()``); every step of the computation runs in the
library's CUDA kernels.  Errors raise ``ScatmanError`` carrying the status
code and the library's message.
"""
from __future__ import annotations

import ctypes
from typing import Optional

import numpy as np

from . import _lib
from ._lib import scatman_config, scatman_shape
from .types import alm_array


class ScatmanError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_lib.STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def _check(code: int, handle: Optional["Handle"] = None, what: str = ""):
    if code != 0:
        msg = ""
        if handle is not None and handle.ptr:
            msg = _lib.load().scatman_last_error(handle.ptr).decode()
        raise ScatmanError(code, f"{what}: {msg}" if what else msg)


def _device_ptr(t, dtypes, n: int, what: str) -> ctypes.c_void_p:
    """Data pointer of a CUDA tensor after checking that the library may write
    (or read) n elements of one of `dtypes` there: a wrong type, a host
    tensor, a strided view or a short buffer raises ValueError instead of
    reaching a kernel."""
    if t is None:
        return ctypes.c_void_p(None)
    names = tuple(str(d).replace("torch.", "") for d in dtypes)
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{what} must be a CUDA tensor")
    if str(t.dtype).replace("torch.", "") not in names:
        raise ValueError(f"{what} must have dtype {' or '.join(names)}, not {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what} must be contiguous")
    if t.numel() < n:
        raise ValueError(f"{what} holds {t.numel()} elements; {n} are needed")
    return ctypes.c_void_p(t.data_ptr())


def _host_ptr(a, dtype_name: str, n: int, what: str) -> int:
    """Address of a host array (numpy or CPU tensor) that receives n elements."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype_name) or not a.flags["C_CONTIGUOUS"] or a.size < n:
            raise ValueError(f"{what} must be a contiguous {dtype_name} array of at least {n} elements")
        return a.ctypes.data
    if getattr(a, "is_cuda", True) or str(a.dtype).replace("torch.", "") != dtype_name or \
            not a.is_contiguous() or a.numel() < n:
        raise ValueError(f"{what} must be a contiguous CPU {dtype_name} tensor of at least {n} elements")
    return a.data_ptr()


class Handle:
    """Owns a scatman_handle*; keeps the q list and alm buffers alive."""

    def __init__(self, ptr: int, precision: int):
        self.ptr = ctypes.c_void_p(ptr)
        self.precision = precision
        self._keep = []

    @property
    def fp64(self) -> bool:
        return self.precision == _lib.SCATMAN_FP64

    def close(self):
        if self.ptr:
            _lib.load().scatman_destroy(self.ptr)
            self.ptr = ctypes.c_void_p(None)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def make_config(geometry, precision, soft: bool = False, soft_width: float = 0.5, scan_fp64: bool = False,
                q_list: Optional[np.ndarray] = None):
    g = geometry
    cfg = scatman_config()
    cfg.nx, cfg.ny, cfg.nz = g.nx, g.ny, g.nz
    cfg.voxel, cfg.wavelength, cfg.theta_max_deg = g.voxel, g.wavelength, g.theta_max_deg
    cfg.det_nx, cfg.det_ny = g.det_nx, g.det_ny
    keep = None
    if q_list is not None:
        keep = np.ascontiguousarray(q_list, dtype=np.float64)
        cfg.q_list = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.n_q = keep.shape[0]
    cfg.precision = _lib.PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    cfg.soft = int(bool(soft))
    cfg.soft_width = float(soft_width)
    cfg.scan_fp64 = int(bool(scan_fp64))
    cfg.detector = int(getattr(g, "detector", 0))
    return cfg, keep


def make_shape(shape):
    st = scatman_shape()
    st.kind = shape.kind
    st.r, st.a, st.b, st.c, st.R0 = shape.r, shape.a, shape.b, shape.c, shape.R0
    st.lmax = shape.lmax
    alm = alm_array(shape)
    st.alm = alm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    st.delta, st.beta = shape.delta, shape.beta
    st.latitude, st.longitude, st.rotation = shape.latitude, shape.longitude, shape.rotation
    st.cx, st.cy, st.cz = shape.cx, shape.cy, shape.cz
    keep = [alm]
    rm = getattr(shape, "radial_map", None)
    if rm is not None:
        rm = np.ascontiguousarray(rm, dtype=np.float64)
        st.radial_map = rm.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        st.map_ntheta, st.map_nphi = rm.shape
        keep.append(rm)
    vm = getattr(shape, "volume_map", None)
    if vm is not None:
        vm = np.ascontiguousarray(vm, dtype=np.uint8)
        st.volume_map = vm.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        st.map_nx, st.map_ny, st.map_nz = vm.shape
        st.map_dx = shape.map_dx
        keep.append(vm)
        for name in ("map_delta", "map_beta"):
            arr = getattr(shape, name, None)
            if arr is not None:
                arr = np.ascontiguousarray(arr, dtype=np.float64)
                assert arr.shape == vm.shape, name + " must match the volume map"
                setattr(st, name, arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
                keep.append(arr)
    return st, keep


def scatman_create(geometry, precision, soft: bool = False, soft_width: float = 0.5, scan_fp64: bool = False,
                   q_list: Optional[np.ndarray] = None, stream: Optional[int] = None) -> Handle:
    """scatman_create: the stream defaults to torch's current CUDA stream."""
    lib = _lib.load()
    cfg, keep = make_config(geometry, precision, soft, soft_width, scan_fp64, q_list)
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
        if stream == 0:
            stream = 1          # cudaStreamLegacy: torch's default stream, not a library-owned one
    out = ctypes.c_void_p()
    code = lib.scatman_create(ctypes.byref(cfg), ctypes.c_void_p(stream), ctypes.byref(out))
    if code != 0:
        raise ScatmanError(code, "scatman_create: " + lib.scatman_last_error(None).decode())
    h = Handle(out.value, cfg.precision)
    h._keep.append(keep)
    return h


def scatman_voxelise(h: Handle, shape) -> None:
    st, alm = make_shape(shape)
    _check(_lib.load().scatman_voxelise(h.ptr, ctypes.byref(st)), h, "voxelise")


def scatman_forward(h: Handle, I, A=None) -> None:
    """I, A: CUDA tensors (float64/complex128 in FP64 mode, float32/complex64 otherwise)."""
    n = scatman_n_pix(h)
    pi = _device_ptr(I, ["float64"] if h.fp64 else ["float32"], n, "I")
    pa = _device_ptr(A, ["complex128"] if h.fp64 else ["complex64"], n, "A")
    _check(_lib.load().scatman_forward(h.ptr, pi, pa), h, "forward")


def scatman_acquire(h: Handle, shape, I_host) -> None:
    """I_host: numpy array or pinned CPU tensor of n_pix elements."""
    st, alm = make_shape(shape)
    ptr = _host_ptr(I_host, "float64" if h.fp64 else "float32", scatman_n_pix(h), "I_host")
    _check(_lib.load().scatman_acquire(h.ptr, ctypes.byref(st), ctypes.c_void_p(ptr)), h, "acquire")


def scatman_acquire_batch(h: Handle, shapes, I_host) -> None:
    """I_host: one host array per shape (numpy arrays or pinned CPU tensors of
    n_pix elements), or a 2D array / tensor whose rows are the patterns."""
    n = len(shapes)
    arr = (scatman_shape * max(n, 1))()
    keep = []
    for i, s in enumerate(shapes):
        st, k = make_shape(s)
        arr[i] = st
        keep.append(k)
    rows = [I_host[i] for i in range(n)]
    dt, npx = ("float64" if h.fp64 else "float32"), scatman_n_pix(h)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[_host_ptr(r, dt, npx, f"I_host[{i}]") for i, r in enumerate(rows)])
    _check(_lib.load().scatman_acquire_batch(h.ptr, arr, n, ptrs), h, "acquire_batch")


def scatman_backward(h: Handle, dLdI) -> np.ndarray:
    lib = _lib.load()
    n = lib.scatman_param_count(h.ptr)
    out = np.zeros(n, dtype=np.float64)
    pd = _device_ptr(dLdI, ["float64"] if h.fp64 else ["float32"], scatman_n_pix(h), "dLdI")
    _check(lib.scatman_backward(h.ptr, pd, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h, "backward")
    return out


def scatman_photon_counts(h: Handle, photon_density: float, seed: int, I, want_lambda: bool = True,
                          want_counts: bool = True):
    """Ideal detector: (expected photons, Poisson counts) as CUDA tensors
    (float64 and int64); either may be skipped (None)."""
    import torch
    n = scatman_n_pix(h)
    pi = _device_ptr(I, ["float64"] if h.fp64 else ["float32"], n, "I")
    lam = torch.empty(n, dtype=torch.float64, device=I.device) if want_lambda else None
    cnt = torch.empty(n, dtype=torch.int64, device=I.device) if want_counts else None
    _check(_lib.load().scatman_photon_counts(
        h.ptr, float(photon_density), int(seed) & 0xFFFFFFFFFFFFFFFF, pi,
        ctypes.c_void_p(lam.data_ptr() if lam is not None else None),
        ctypes.c_void_p(cnt.data_ptr() if cnt is not None else None)), h, "photon counts")
    return lam, cnt


def scatman_param_count(h: Handle) -> int:
    return _lib.load().scatman_param_count(h.ptr)


def scatman_n_pix(h: Handle) -> int:
    return _lib.load().scatman_n_pix(h.ptr)


def scatman_elem_size(h: Handle) -> int:
    return _lib.load().scatman_elem_size(h.ptr)


def scatman_device_bytes(h: Handle) -> int:
    return _lib.load().scatman_device_bytes(h.ptr)


def scatman_sync(h: Handle) -> None:
    _check(_lib.load().scatman_sync(h.ptr), h, "sync")


def scatman_get_occupancy(h: Handle, shape_zxy) -> np.ndarray:
    out = np.zeros(shape_zxy, dtype=np.float64)
    _check(_lib.load().scatman_get_occupancy(h.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h)
    return out


def scatman_get_slices(h: Handle, shape_zxy) -> np.ndarray:
    buf = np.zeros(tuple(shape_zxy) + (2,), dtype=np.float64)
    _check(_lib.load().scatman_get_slices(h.ptr, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h)
    return buf[..., 0] + 1j * buf[..., 1]


def scatman_get_q(h: Handle) -> np.ndarray:
    n = scatman_n_pix(h)
    out = np.zeros((n, 3), dtype=np.float64)
    _check(_lib.load().scatman_get_q(h.ptr, out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))), h)
    return out


def scatman_contraction_flops(h: Handle):
    """(issued, dense) real flops of one contraction launch for the current shape."""
    a = ctypes.c_double()
    b = ctypes.c_double()
    _check(_lib.load().scatman_contraction_flops(h.ptr, ctypes.byref(a), ctypes.byref(b)), h)
    return a.value, b.value


def scatman_set_wait_limit(h: Handle, seconds: float) -> None:
    """Failure-path hook: the handle's tensor-core kernels give up their waits
    on other warps after `seconds` (<= 0: the default 2 s)."""
    _check(_lib.load().scatman_set_wait_limit(h.ptr, float(seconds)), h, "set_wait_limit")


def scatman_debug_stall(h: Handle, on: bool) -> None:
    """Failure-path hook: the handle's tensor-core MMA warps first wait on a
    barrier nothing arrives at, so the kernels take their time-out path."""
    _check(_lib.load().scatman_debug_stall(h.ptr, int(bool(on))), h, "debug_stall")


def scatman_debug_fail_allocation(after: int) -> None:
    """Failure-path hook: the device allocation after `after` more successful
    ones fails once (process-wide); a negative value disarms it."""
    _lib.load().scatman_debug_fail_allocation(int(after))


def scatman_destroy(h: Handle) -> None:
    h.close()


def scatman_version() -> str:
    return _lib.load().scatman_version().decode()


def scatman_last_error(h: Handle) -> str:
    return _lib.load().scatman_last_error(h.ptr).decode()


def scatman_forward_noalloc(geometry, shape, I, A=None, soft: bool = False, soft_width: float = 0.5,
                            scan_fp64: bool = False, q_list: Optional[np.ndarray] = None,
                            stream: Optional[int] = None) -> None:
    """scatman_forward_noalloc: the FP32 forward for callers that cannot
    allocate device memory (an application whose memory pool already holds
    nearly all of the GPU, or a loop that must not take the device-wide
    synchronisation of an allocation).  I (and A) are float32 (complex64) CUDA
    tensors of at least n_pix elements; the flat detector or a q_list only."""
    lib = _lib.load()
    cfg, keep = make_config(geometry, "fp32", soft, soft_width, scan_fp64, q_list)
    st, alm = make_shape(shape)
    n = int(q_list.shape[0]) if q_list is not None else geometry.det_nx * geometry.det_ny
    pi = _device_ptr(I, ["float32"], n, "I")
    pa = _device_ptr(A, ["complex64"], n, "A")
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    code = lib.scatman_forward_noalloc(ctypes.byref(cfg), ctypes.byref(st), ctypes.c_void_p(stream), pi, pa)
    if code != 0:
        raise ScatmanError(code, "scatman_forward_noalloc: " + lib.scatman_last_error(None).decode())
