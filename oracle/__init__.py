"""FP64 CPU oracle of the MSFT (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path never does: it shares no code
with the CUDA library.  ``msft_oracle.c`` holds the arithmetic (plain C, FP64,
OpenMP over pixels/slices); this module only builds it and marshals numpy
arrays.  ``brute.py`` is a second, independent NumPy restatement for tiny grids.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional

import numpy as np

from workloads import ELLIPSOID, SPHERE, SPHHARM, Geometry, Shape

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msft_oracle.c")
_LIB = os.path.join(_HERE, "liborc.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP contraction off so the compiler does not
    fuse multiply-adds on either host architecture)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class _OrcShape(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int),
        ("r", ctypes.c_double), ("a", ctypes.c_double), ("b", ctypes.c_double), ("c", ctypes.c_double),
        ("R0", ctypes.c_double),
        ("lmax", ctypes.c_int),
        ("alm", ctypes.POINTER(ctypes.c_double)),
        ("delta", ctypes.c_double), ("beta", ctypes.c_double),
        ("latitude", ctypes.c_double), ("longitude", ctypes.c_double), ("rotation", ctypes.c_double),
        ("cx", ctypes.c_double), ("cy", ctypes.c_double), ("cz", ctypes.c_double),
        ("radial_map", ctypes.POINTER(ctypes.c_double)), ("map_ntheta", ctypes.c_int), ("map_nphi", ctypes.c_int),
        ("volume_map", ctypes.POINTER(ctypes.c_ubyte)), ("map_nx", ctypes.c_int), ("map_ny", ctypes.c_int),
        ("map_nz", ctypes.c_int), ("map_dx", ctypes.c_double),
        ("map_delta", ctypes.POINTER(ctypes.c_double)), ("map_beta", ctypes.POINTER(ctypes.c_double)),
    ]


_D = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_rotation.argtypes = [ctypes.c_double] * 3 + [_D]
        lib.orc_legendre.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double]
        lib.orc_legendre.restype = ctypes.c_double
        lib.orc_real_sh.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double]
        lib.orc_real_sh.restype = ctypes.c_double
        lib.orc_voxelise.argtypes = [ctypes.POINTER(_OrcShape), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_int, ctypes.c_double, _D]
        lib.orc_voxelise.restype = ctypes.c_int
        lib.orc_slices.argtypes = [_D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, _D]
        lib.orc_detector_q.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D]
        lib.orc_detector_q_uniform.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, _D,
                                               ctypes.POINTER(ctypes.c_int)]
        lib.orc_voxel_index.argtypes = [ctypes.POINTER(_OrcShape), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, _D, _D]
        lib.orc_slices_n.argtypes = [_D, _D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_double, _D, _D]
        lib.orc_pixel_solid_angle.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_int, _D]
        lib.orc_philox.argtypes = [ctypes.c_uint] * 6 + [ctypes.POINTER(ctypes.c_uint)]
        lib.orc_photon_counts.argtypes = [_D, _D, ctypes.c_long, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                          ctypes.c_ulonglong, _D, ctypes.POINTER(ctypes.c_longlong)]
        lib.orc_msft.argtypes = [_D, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                 _D, ctypes.c_long, _D, _D]
        lib.orc_intensity.argtypes = [_D, _D, ctypes.c_long, _D]
        lib.orc_msft_adjoint.argtypes = [_D, _D, _D, ctypes.c_long, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_int, ctypes.c_double, _D, _D]
        lib.orc_gradient.argtypes = [ctypes.POINTER(_OrcShape), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_double, ctypes.c_double, _D, ctypes.c_long,
                                     _D, _D, _D, _D]
        lib.orc_gradient.restype = ctypes.c_int
        lib.orc_n_params.argtypes = [ctypes.POINTER(_OrcShape)]
        lib.orc_n_params.restype = ctypes.c_int
        lib.orc_num_threads.restype = ctypes.c_int
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _shape_struct(s: Shape):
    alm = s.alm_array()
    st = _OrcShape(s.kind, s.r, s.a, s.b, s.c, s.R0, s.lmax, _p(alm), s.delta, s.beta,
                   s.latitude, s.longitude, s.rotation, s.cx, s.cy, s.cz)
    keep = [alm]
    if getattr(s, "radial_map", None) is not None:
        rm = np.ascontiguousarray(s.radial_map, dtype=np.float64)
        st.radial_map = _p(rm)
        st.map_ntheta, st.map_nphi = rm.shape
        keep.append(rm)
    if getattr(s, "volume_map", None) is not None:
        vm = np.ascontiguousarray(s.volume_map, dtype=np.uint8)
        st.volume_map = vm.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        st.map_nx, st.map_ny, st.map_nz = vm.shape
        st.map_dx = s.map_dx
        keep.append(vm)
        for name in ("map_delta", "map_beta"):
            arr = getattr(s, name, None)
            if arr is not None:
                arr = np.ascontiguousarray(arr, dtype=np.float64)
                setattr(st, name, _p(arr))
                keep.append(arr)
    return st, keep  # keep the arrays alive


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(n)


def rotation(lat: float, lon: float, rot: float) -> np.ndarray:
    R = np.zeros(9)
    _load().orc_rotation(lat, lon, rot, _p(R))
    return R.reshape(3, 3)


def legendre(l: int, m: int, x: float) -> float:
    return _load().orc_legendre(l, m, x)


def real_sh(l: int, m: int, theta: float, phi: float) -> float:
    return _load().orc_real_sh(l, m, theta, phi)


def voxelise(shape: Shape, g: Geometry, soft: bool = False, width: float = 0.5):
    """Occupancy chi [z][x][y] (Block 5); returns (chi, clipped)."""
    chi = np.zeros((g.nz, g.nx, g.ny))
    st, keep = _shape_struct(shape)
    clipped = _load().orc_voxelise(ctypes.byref(st), g.nx, g.ny, g.nz, g.voxel, int(soft), width, _p(chi))
    return chi, bool(clipped)


def slices(chi: np.ndarray, g: Geometry, delta: float, beta: float) -> np.ndarray:
    """Effective slice strength rho_j = (n^2-1) chi T_j (Eq. 5-9), complex [z][x][y]."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    re = np.zeros_like(chi)
    im = np.zeros_like(chi)
    _load().orc_slices(_p(chi), g.nx, g.ny, g.nz, g.voxel, g.wavelength, delta, beta, _p(re), _p(im))
    return re + 1j * im


def voxel_index(shape: Shape, g: Geometry):
    """Per-voxel (delta, beta) [z][x][y] of a volume map with a per-cell index."""
    d = np.zeros((g.nz, g.nx, g.ny))
    b = np.zeros((g.nz, g.nx, g.ny))
    st, keep = _shape_struct(shape)
    _load().orc_voxel_index(ctypes.byref(st), g.nx, g.ny, g.nz, g.voxel, _p(d), _p(b))
    return d, b


def slices_n(chi: np.ndarray, g: Geometry, delta_v: np.ndarray, beta_v: np.ndarray) -> np.ndarray:
    """Slice strength with a voxel-resolved index: (n_v^2-1) chi T, T from Eq. 8 with n_v."""
    chi = np.ascontiguousarray(chi, dtype=np.float64)
    dv = np.ascontiguousarray(delta_v, dtype=np.float64)
    bv = np.ascontiguousarray(beta_v, dtype=np.float64)
    re = np.zeros_like(chi)
    im = np.zeros_like(chi)
    _load().orc_slices_n(_p(chi), _p(dv), _p(bv), g.nx, g.ny, g.nz, g.voxel, g.wavelength, _p(re), _p(im))
    return re + 1j * im


def detector_q(g: Geometry) -> np.ndarray:
    """q = k_out - k_in of every detector pixel (Eq. 3), [pixel][3]: the flat
    detector, or the uniform-q virtual detector when g.detector says so."""
    q = np.zeros((g.n_pix, 3))
    if getattr(g, "detector", 0) == 1:
        valid = np.zeros(g.n_pix, dtype=np.int32)
        _load().orc_detector_q_uniform(g.det_nx, g.det_ny, g.theta_max_deg, g.wavelength, _p(q),
                                       valid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        return q
    _load().orc_detector_q(g.det_nx, g.det_ny, g.theta_max_deg, g.wavelength, _p(q))
    return q


def detector_valid(g: Geometry) -> np.ndarray:
    """Pixels with a scattering direction (all of them on the flat detector)."""
    if getattr(g, "detector", 0) != 1:
        return np.ones(g.n_pix, dtype=bool)
    q = np.zeros((g.n_pix, 3))
    valid = np.zeros(g.n_pix, dtype=np.int32)
    _load().orc_detector_q_uniform(g.det_nx, g.det_ny, g.theta_max_deg, g.wavelength, _p(q),
                                   valid.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return valid.astype(bool)


def msft(rho: np.ndarray, q: np.ndarray, voxel: float = 1.0) -> np.ndarray:
    """A(q) = sum_j e^{-i q_z z_j} F[rho_j](q_x,q_y) (Eq. 9) for rho [z][x][y]."""
    nz, nx, ny = rho.shape
    re = np.ascontiguousarray(rho.real, dtype=np.float64)
    im = np.ascontiguousarray(rho.imag, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    ar = np.zeros(q.shape[0])
    ai = np.zeros(q.shape[0])
    _load().orc_msft(_p(re), _p(im), nx, ny, nz, voxel, _p(q), q.shape[0], _p(ar), _p(ai))
    return ar + 1j * ai


def msft_adjoint(gq: np.ndarray, q: np.ndarray, shape_zxy, voxel: float = 1.0) -> np.ndarray:
    """S_v = sum_q g_q e^{+i q.r_v}: adjoint of rho -> A."""
    nz, nx, ny = shape_zxy
    gr = np.ascontiguousarray(gq.real, dtype=np.float64)
    gi = np.ascontiguousarray(gq.imag, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    sr = np.zeros((nz, nx, ny))
    si = np.zeros((nz, nx, ny))
    _load().orc_msft_adjoint(_p(gr), _p(gi), _p(q), q.shape[0], nx, ny, nz, voxel, _p(sr), _p(si))
    return sr + 1j * si


def forward(shape: Shape, g: Geometry, q: Optional[np.ndarray] = None, soft: bool = False,
            width: float = 0.5):
    """Whole path: occupancy -> slices -> field -> intensity.  Returns (I, A)."""
    if q is None:
        q = detector_q(g)
    chi, _ = voxelise(shape, g, soft, width)
    if shape.varying_index():
        rho = slices_n(chi, g, *voxel_index(shape, g))
    else:
        rho = slices(chi, g, shape.delta, shape.beta)
    A = msft(rho, q, g.voxel)
    if getattr(g, "detector", 0) == 1 and len(A) == g.n_pix:
        A = np.where(detector_valid(g), A, 0.0)       # no scattering direction: no field
    return np.abs(A) ** 2, A


def gradient(shape: Shape, g: Geometry, dLdI: np.ndarray, A: np.ndarray,
             q: Optional[np.ndarray] = None, width: float = 0.5) -> np.ndarray:
    """dL/d(params) for soft occupancy, given dL/dI and the forward field A."""
    if shape.kind not in (SPHERE, ELLIPSOID, SPHHARM):
        raise ValueError("the oracle gradient covers sphere, ellipsoid and harmonics shapes")
    if q is None:
        q = detector_q(g)
    st, keep = _shape_struct(shape)
    lib = _load()
    n = lib.orc_n_params(ctypes.byref(st))
    out = np.zeros(n)
    dl = np.ascontiguousarray(dLdI, dtype=np.float64)
    ar = np.ascontiguousarray(A.real, dtype=np.float64)
    ai = np.ascontiguousarray(A.imag, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    lib.orc_gradient(ctypes.byref(st), g.nx, g.ny, g.nz, g.voxel, g.wavelength, width, _p(q),
                     q.shape[0], _p(dl), _p(ar), _p(ai), _p(out))
    return out


def pixel_solid_angle(g: Geometry) -> np.ndarray:
    """Solid angle of every pixel: the flat detector or the uniform-q one."""
    out = np.zeros(g.n_pix)
    _load().orc_pixel_solid_angle(g.det_nx, g.det_ny, g.theta_max_deg, g.wavelength,
                                  int(getattr(g, "detector", 0) == 1), _p(out))
    return out


def philox(counter, key) -> np.ndarray:
    """Philox-4x32-10 block for a 4-word counter and a 2-word key."""
    out = (ctypes.c_uint * 4)()
    _load().orc_philox(*[int(c) & 0xFFFFFFFF for c in counter], *[int(k) & 0xFFFFFFFF for k in key], out)
    return np.array(list(out), dtype=np.uint64)


def photon_counts(I: np.ndarray, g: Geometry, photon_density: float, seed: int, counts: bool = True):
    """Ideal detector: expected photons per pixel and Poisson counts."""
    I = np.ascontiguousarray(I, dtype=np.float64)
    dom = pixel_solid_angle(g)
    lam = np.zeros(I.shape[0])
    cnt = np.zeros(I.shape[0], dtype=np.int64) if counts else None
    _load().orc_photon_counts(_p(I), _p(dom), I.shape[0], photon_density, g.wavelength, g.voxel,
                              int(seed) & 0xFFFFFFFFFFFFFFFF, _p(lam),
                              cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_longlong)) if counts else None)
    return lam, cnt


def relative_l2(x: np.ndarray, ref: np.ndarray) -> float:
    den = float(np.linalg.norm(ref.ravel()))
    num = float(np.linalg.norm((x - ref).ravel()))
    return num / den if den > 0 else num
