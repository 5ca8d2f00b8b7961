"""Seeded synthetic workloads shared by the CUDA path's tests/bench and the oracle.

This module only *draws* inputs: grid and detector sizes, shape kinds and their
parameters (radii, semi-axes, spherical-harmonic coefficients, delta, beta and
orientation angles).  It holds none of the method's arithmetic (no voxelisation,
no q mapping, no transmission, no Fourier sums), so that the oracle and the GPU
path can both use it without sharing any computation.

Workload recipes (the paper's Sec. 5 examples and Sec. 6 timing study use
ellipsoids and spherical-harmonics shapes; sizes below are synthetic stand-ins):

* ``sphere_32``     homogeneous sphere r=12 centred in 32^3, delta=1e-3, beta=1e-4,
                    wavelength 8 voxels, flat 64x64 detector to 30 deg.
* ``ellipsoid_96``  ellipsoids with semi-axes U(20,40), uniform random orientation,
                    96^3, delta U(1e-3,2e-2), beta=delta/10, wavelength 10,
                    256x256 detector to 45 deg, 64 seeds.
* ``sh_128``        real spherical-harmonics radius l<=8, R0=48, a_lm ~ N(0, 0.05/l),
                    128^3, delta=0.01, beta=0.001 (the SphericalHarmonics example of
                    Listing 2), wavelength 10, 512x512 detector to 60 deg, 16 seeds.
* ``sh_grad_96``    l<=6 harmonics, R0=36, 96^3, soft occupancy w=0.5 voxel,
                    256x256 detector to 45 deg, 32 seeds.
* ``serving_mix``   Poisson stream of mixed sphere/ellipsoid/harmonics requests over
                    grids {48,64,96,128}^3 and detectors {128,256,512}^2.

Orientation draws: the main axis is uniform on the sphere (latitude = asin(U(-1,1)),
longitude U(-180,180)) and the rotation about it is U(0,360); composing an
axis-alignment with a uniform spin about the axis gives a Haar-uniform rotation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

SPHERE, ELLIPSOID, SPHHARM, RADIALMAP, VOLUMEMAP = 0, 1, 2, 3, 4
DETECTOR_FLAT, DETECTOR_UNIFORM_Q = 0, 1
KIND_NAMES = {SPHERE: "sphere", ELLIPSOID: "ellipsoid", SPHHARM: "sphharm", RADIALMAP: "radialmap",
              VOLUMEMAP: "volumemap"}


@dataclasses.dataclass
class Shape:
    """Shape parameters as the paper states them (Listings 1-2): geometry,
    refractive index n = 1 - delta + i*beta, and orientation in degrees."""
    kind: int
    r: float = 0.0                      # sphere radius
    a: float = 0.0                      # ellipsoid semi-axes (c lies along the main axis)
    b: float = 0.0
    c: float = 0.0
    R0: float = 0.0                     # harmonics mean radius
    lmax: int = 0
    alm: Optional[np.ndarray] = None    # (lmax+1)^2 real coefficients, index l*l+l+m; alm[0] unused
    delta: float = 0.0
    beta: float = 0.0
    latitude: float = -90.0             # -90 deg: main axis along +z (towards the detector)
    longitude: float = 0.0
    rotation: float = 0.0
    cx: float = 0.0                     # centre offset from the grid centre (length units)
    cy: float = 0.0
    cz: float = 0.0
    # radii map (Sec. 5.2 "Shape (2/3)"): [n_theta][n_phi] radii in length units at
    # latitudes -pi/2 + i pi/n_theta and longitudes 2 pi k/n_phi
    radial_map: Optional[np.ndarray] = None
    # volume map (Sec. 5.2 "Shape (3/3)"): [mx][my][mz] booleans, cell edge map_dx,
    # optional per-cell delta and beta (same shape) for a voxel-resolved index
    volume_map: Optional[np.ndarray] = None
    map_dx: float = 1.0
    map_delta: Optional[np.ndarray] = None
    map_beta: Optional[np.ndarray] = None

    def n_params(self) -> int:
        if self.kind == SPHERE:
            return 3
        if self.kind == ELLIPSOID:
            return 5
        if self.kind in (RADIALMAP, VOLUMEMAP):
            return 0                    # no gradient for map shapes
        return (self.lmax + 1) ** 2 - 1 + 3

    def varying_index(self) -> bool:
        return self.kind == VOLUMEMAP and (self.map_delta is not None or self.map_beta is not None)

    def alm_array(self) -> np.ndarray:
        if self.alm is None:
            return np.zeros(max(1, (self.lmax + 1) ** 2), dtype=np.float64)
        return np.ascontiguousarray(self.alm, dtype=np.float64)

    def copy(self) -> "Shape":
        s = dataclasses.replace(self)
        for f in ("alm", "radial_map", "volume_map", "map_delta", "map_beta"):
            v = getattr(self, f)
            if v is not None:
                setattr(s, f, np.array(v, copy=True))
        return s


@dataclasses.dataclass
class Geometry:
    """Grid and detector of one experiment (Sec. 3, Blocks 1-3)."""
    nx: int
    ny: int
    nz: int
    voxel: float
    wavelength: float
    theta_max_deg: float
    det_nx: int
    det_ny: int
    detector: int = 0                   # DETECTOR_FLAT or DETECTOR_UNIFORM_Q (the paper's virtual detector)

    @property
    def n_pix(self) -> int:
        return self.det_nx * self.det_ny

    @property
    def n_vox(self) -> int:
        return self.nx * self.ny * self.nz


def random_orientation(rng: np.random.Generator):
    lat = math.degrees(math.asin(rng.uniform(-1.0, 1.0)))
    lon = rng.uniform(-180.0, 180.0)
    rot = rng.uniform(0.0, 360.0)
    return lat, lon, rot


def random_alm(rng: np.random.Generator, lmax: int, sigma0: float = 0.05) -> np.ndarray:
    """a_lm ~ N(0, sigma0/l) for 1 <= l <= lmax (sigma0/l read as the standard deviation)."""
    alm = np.zeros((lmax + 1) ** 2, dtype=np.float64)
    for l in range(1, lmax + 1):
        for m in range(-l, l + 1):
            alm[l * l + l + m] = rng.normal(0.0, sigma0 / l)
    return alm


# ---------------------------------------------------------------------------
# The five workloads
# ---------------------------------------------------------------------------

def sphere_32():
    g = Geometry(32, 32, 32, 1.0, 8.0, 30.0, 64, 64)
    s = Shape(SPHERE, r=12.0, delta=1e-3, beta=1e-4)
    return g, [s]


def ellipsoid_96(n_shapes: int = 64, seed0: int = 0):
    g = Geometry(96, 96, 96, 1.0, 10.0, 45.0, 256, 256)
    shapes = []
    for k in range(n_shapes):
        rng = np.random.default_rng(seed0 + k)
        a, b, c = rng.uniform(20.0, 40.0, size=3)
        d = rng.uniform(1e-3, 2e-2)
        lat, lon, rot = random_orientation(rng)
        shapes.append(Shape(ELLIPSOID, a=a, b=b, c=c, delta=d, beta=d / 10.0,
                            latitude=lat, longitude=lon, rotation=rot))
    return g, shapes


def sh_128(n_shapes: int = 16, seed0: int = 0, lmax: int = 8):
    g = Geometry(128, 128, 128, 1.0, 10.0, 60.0, 512, 512)
    shapes = []
    for k in range(n_shapes):
        rng = np.random.default_rng(1000 + seed0 + k)
        alm = random_alm(rng, lmax)
        lat, lon, rot = random_orientation(rng)
        shapes.append(Shape(SPHHARM, R0=48.0, lmax=lmax, alm=alm, delta=0.01, beta=0.001,
                            latitude=lat, longitude=lon, rotation=rot))
    return g, shapes


def sh_grad_96(n_shapes: int = 32, seed0: int = 0, lmax: int = 6):
    g = Geometry(96, 96, 96, 1.0, 10.0, 45.0, 256, 256)
    shapes = []
    for k in range(n_shapes):
        rng = np.random.default_rng(2000 + seed0 + k)
        alm = random_alm(rng, lmax)
        lat, lon, rot = random_orientation(rng)
        shapes.append(Shape(SPHHARM, R0=36.0, lmax=lmax, alm=alm, delta=0.01, beta=0.001,
                            latitude=lat, longitude=lon, rotation=rot))
    return g, shapes


def perturbed(shape: Shape, rng: np.random.Generator, rel: float = 0.02) -> Shape:
    """A nearby shape used as a fitting target (same kind, parameters nudged)."""
    s = shape.copy()
    s.delta *= 1.0 + rng.normal(0.0, rel)
    s.beta *= 1.0 + rng.normal(0.0, rel)
    if s.kind == SPHERE:
        s.r *= 1.0 + rng.normal(0.0, rel)
    elif s.kind == ELLIPSOID:
        s.a *= 1.0 + rng.normal(0.0, rel)
        s.b *= 1.0 + rng.normal(0.0, rel)
        s.c *= 1.0 + rng.normal(0.0, rel)
    else:
        s.R0 *= 1.0 + rng.normal(0.0, rel)
        s.alm = s.alm + rng.normal(0.0, rel * 0.05, size=s.alm.shape)
        s.alm[0] = 0.0
    return s


SERVING_GRIDS = (48, 64, 96, 128)
SERVING_DETS = (128, 256, 512)


@dataclasses.dataclass
class Request:
    rid: int
    arrival_s: float
    geometry: Geometry
    shape: Shape
    target: Shape


def serving_mix(n_requests: int = 2000, rate_per_s: float = 100.0, seed: int = 0,
                lmax: int = 6) -> List[Request]:
    """Poisson stream of forward+gradient requests with mixed grid/detector sizes."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_per_s)
        n = int(rng.choice(SERVING_GRIDS))
        det = int(rng.choice(SERVING_DETS))
        theta = 45.0
        g = Geometry(n, n, n, 1.0, 10.0, theta, det, det)
        kind = int(rng.integers(0, 3))
        d = rng.uniform(1e-3, 3e-2)
        lat, lon, rot = random_orientation(rng)
        if kind == SPHERE:
            s = Shape(SPHERE, r=rng.uniform(0.25, 0.4) * n, delta=d, beta=d / 10.0)
        elif kind == ELLIPSOID:
            ax = rng.uniform(0.2, 0.4, size=3) * n
            s = Shape(ELLIPSOID, a=ax[0], b=ax[1], c=ax[2], delta=d, beta=d / 10.0,
                      latitude=lat, longitude=lon, rotation=rot)
        else:
            s = Shape(SPHHARM, R0=0.3 * n, lmax=lmax, alm=random_alm(rng, lmax), delta=d,
                      beta=d / 10.0, latitude=lat, longitude=lon, rotation=rot)
        tgt = perturbed(s, rng)
        out.append(Request(rid, t, g, s, tgt))
    return out


def listing2_sphharm(mean_radius: float, lmax_keep: int = 9) -> Shape:
    """The harmonics shape of Listing 2 (triplets [l, m, c] in nm: [0,0,200],
    [3,2,20], [6,4,4], [9,6,2]; delta 0.01, beta 0.001, latitude 30,
    longitude -40) rescaled so its mean radius is `mean_radius`."""
    trip = [(0, 0, 200.0), (3, 2, 20.0), (6, 4, 4.0), (9, 6, 2.0)]
    c00 = trip[0][2]
    lmax = min(lmax_keep, max(t[0] for t in trip))
    alm = np.zeros((lmax + 1) ** 2)
    for l, m, c in trip[1:]:
        if l <= lmax:
            alm[l * l + l + m] = c / c00 * math.sqrt(4 * math.pi)   # a_lm = c_lm / R0, R0 = c_00 Y_00
    return Shape(SPHHARM, R0=mean_radius, lmax=lmax, alm=alm, delta=0.01, beta=0.001, latitude=30.0,
                 longitude=-40.0, rotation=0.0)


def fig8b_case(radius_wavelengths: float, det: int, theta_max_deg: float = 30.0):
    """Timing study of Sec. 6 (Fig. 8b): the Listing-2 harmonics shape scaled to a
    mean radius of 3/5/10/20 wavelengths, uniform-q detector of det^2 pixels.
    Length unit = wavelength; voxel = lambda / (2 sin theta_max), the spacing
    whose Nyquist limit is the detector's q_max (Block 3)."""
    lam = 1.0
    voxel = lam / (2.0 * math.sin(math.radians(theta_max_deg)))
    R = radius_wavelengths * lam
    n = int(math.ceil(2.0 * 1.3 * R / voxel)) + 4
    g = Geometry(n, n, n, voxel, lam, theta_max_deg, det, det, DETECTOR_UNIFORM_Q)
    return g, listing2_sphharm(R)


def random_slices(rng: np.random.Generator, nz: int, nx: int, ny: int) -> np.ndarray:
    """Random complex slice strengths in the [z][x][y] layout, |s| <= 1."""
    mag = rng.uniform(0.0, 1.0, size=(nz, nx, ny))
    ph = rng.uniform(-math.pi, math.pi, size=(nz, nx, ny))
    return mag * np.cos(ph) + 1j * mag * np.sin(ph)


# ---------------------------------------------------------------------------
# Map shapes (Sec. 5.2, "Shape (2/3)" and "Shape (3/3)")
# ---------------------------------------------------------------------------

def random_radial_map(rng: np.random.Generator, n_theta: int, n_phi: int, R0: float, amp: float = 0.15,
                      terms: int = 6) -> np.ndarray:
    """A smooth random radii map: R0 times one plus a few random low-order
    cosine/sine products in latitude and longitude (periodic in both)."""
    lat = -math.pi / 2 + math.pi * np.arange(n_theta) / n_theta
    lon = 2 * math.pi * np.arange(n_phi) / n_phi
    L, P = np.meshgrid(lat, lon, indexing="ij")
    f = np.zeros((n_theta, n_phi))
    for _ in range(terms):
        a, b = int(rng.integers(1, 4)), int(rng.integers(0, 4))
        ph1, ph2 = rng.uniform(0, 2 * math.pi, size=2)
        f += rng.normal(0.0, 1.0) * np.cos(2 * a * L + ph1) * np.cos(b * P + ph2)
    f *= amp / max(1e-12, np.abs(f).max())
    return R0 * (1.0 + f)


def random_volume_map(rng: np.random.Generator, m: int, blobs: int = 6, fill: float = 0.35) -> np.ndarray:
    """A random solid in an m^3 box: the union of a few random axis-aligned
    boxes and a core block, as booleans [mx][my][mz]."""
    v = np.zeros((m, m, m), dtype=bool)
    c0, c1 = int(m * (0.5 - fill / 2)), int(m * (0.5 + fill / 2))
    v[c0:c1, c0:c1, c0:c1] = True
    for _ in range(blobs):
        lo = rng.integers(0, m - 2, size=3)
        size = rng.integers(2, max(3, m // 3), size=3)
        hi = np.minimum(lo + size, m)
        v[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] = True
    return v


def core_shell_index(volume_map: np.ndarray, core_delta: float, core_beta: float, shell_delta: float,
                     shell_beta: float, core_frac: float = 0.5):
    """Per-cell delta and beta for a two-material sample: cells in the central
    core_frac of the map's box take the core values, the rest the shell's."""
    m = np.array(volume_map.shape)
    idx = np.indices(volume_map.shape).reshape(3, -1).T
    centre = (m - 1) / 2.0
    core = (np.abs(idx - centre) <= core_frac * m / 2.0).all(axis=1).reshape(volume_map.shape)
    delta = np.where(core, core_delta, shell_delta)
    beta = np.where(core, core_beta, shell_beta)
    return delta.astype(np.float64), beta.astype(np.float64)


def radialmap_96(n_shapes: int = 4, seed0: int = 0, n_theta: int = 96, n_phi: int = 192):
    """Radii-map shapes on the 96^3 grid of the ellipsoid workload."""
    g = Geometry(96, 96, 96, 1.0, 10.0, 45.0, 256, 256)
    shapes = []
    for k in range(n_shapes):
        rng = np.random.default_rng(3000 + seed0 + k)
        lat, lon, rot = random_orientation(rng)
        shapes.append(Shape(RADIALMAP, radial_map=random_radial_map(rng, n_theta, n_phi, 30.0), delta=0.01,
                            beta=0.001, latitude=lat, longitude=lon, rotation=rot))
    return g, shapes


def volumemap_96(n_shapes: int = 4, seed0: int = 0, m: int = 40, dx: float = 1.7, core_shell: bool = True):
    """Volume-map shapes on the 96^3 grid, with a two-material index when asked."""
    g = Geometry(96, 96, 96, 1.0, 10.0, 45.0, 256, 256)
    shapes = []
    for k in range(n_shapes):
        rng = np.random.default_rng(4000 + seed0 + k)
        lat, lon, rot = random_orientation(rng)
        v = random_volume_map(rng, m)
        s = Shape(VOLUMEMAP, volume_map=v, map_dx=dx, delta=0.01, beta=0.001, latitude=lat, longitude=lon,
                  rotation=rot)
        if core_shell:
            s.map_delta, s.map_beta = core_shell_index(v, 0.02, 0.004, 0.006, 0.0005)
        shapes.append(s)
    return g, shapes

