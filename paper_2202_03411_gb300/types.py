"""Parameter types of the C ABI's scatman_shape and scatman_config, for users of
the binding.

Every function of the binding reads these objects by attribute only, so any
object with the same fields works as well.  Field meanings and units follow
include/scatman.h: lengths in the wavelength's unit, angles in degrees,
n = 1 - delta + i beta (Eq. 7), orientation as in Fig. 6.
"""
from __future__ import annotations

import copy
import dataclasses
from typing import Optional

import numpy as np

from . import _lib

SPHERE, ELLIPSOID, SPHHARM, RADIALMAP, VOLUMEMAP = (_lib.SCATMAN_SPHERE, _lib.SCATMAN_ELLIPSOID,
                                                    _lib.SCATMAN_SPHHARM, _lib.SCATMAN_RADIALMAP,
                                                    _lib.SCATMAN_VOLUMEMAP)
DETECTOR_FLAT, DETECTOR_UNIFORM_Q = _lib.SCATMAN_DETECTOR_FLAT, _lib.SCATMAN_DETECTOR_UNIFORM_Q


@dataclasses.dataclass
class Shape:
    """scatman_shape: kind, size parameters, index and orientation."""
    kind: int
    r: float = 0.0
    a: float = 0.0
    b: float = 0.0
    c: float = 0.0
    R0: float = 0.0
    lmax: int = 0
    alm: Optional[np.ndarray] = None        # (lmax+1)^2 coefficients, index l*l+l+m; alm[0] unused
    delta: float = 0.0
    beta: float = 0.0
    latitude: float = -90.0
    longitude: float = 0.0
    rotation: float = 0.0
    cx: float = 0.0
    cy: float = 0.0
    cz: float = 0.0
    radial_map: Optional[np.ndarray] = None     # [n_theta][n_phi] radii
    volume_map: Optional[np.ndarray] = None     # [mx][my][mz] occupancy
    map_dx: float = 1.0
    map_delta: Optional[np.ndarray] = None
    map_beta: Optional[np.ndarray] = None

    def n_params(self) -> int:
        return n_params(self)

    def alm_array(self) -> np.ndarray:
        return alm_array(self)

    def copy(self) -> "Shape":
        return copy.deepcopy(self)


@dataclasses.dataclass
class Geometry:
    """The grid and detector fields of scatman_config."""
    nx: int
    ny: int
    nz: int
    voxel: float
    wavelength: float
    theta_max_deg: float
    det_nx: int
    det_ny: int
    detector: int = DETECTOR_FLAT

    @property
    def n_pix(self) -> int:
        return self.det_nx * self.det_ny

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz


def n_params(shape) -> int:
    """Gradient entries of a shape (scatman_param_count's order)."""
    if shape.kind == SPHERE:
        return 3
    if shape.kind == ELLIPSOID:
        return 5
    if shape.kind == SPHHARM:
        return (shape.lmax + 1) ** 2 - 1 + 3
    return 0


def alm_array(shape) -> np.ndarray:
    """The harmonic coefficients as a contiguous float64 array (zeros if absent)."""
    alm = getattr(shape, "alm", None)
    if alm is None:
        return np.zeros(max(1, (shape.lmax + 1) ** 2), dtype=np.float64)
    return np.ascontiguousarray(alm, dtype=np.float64)
