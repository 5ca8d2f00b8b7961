"""Independent NumPy restatement of the MSFT for tiny grids (test infrastructure).

It shares no code with ``msft_oracle.c`` and computes each step another way, so
that agreement between the two pins the C oracle:

* q from the pixel's position vector (k_out = k0 (X, Y, 1)/|(X, Y, 1)|) instead
  of angles;
* rotation from an axis-angle (Rodrigues) composition instead of elementary
  matrix products;
* real spherical harmonics from ``scipy.special.sph_harm_y``;
* radii maps interpolated with ``scipy.ndimage.map_coordinates`` (linear,
  periodic grid) instead of an explicit four-point blend; volume-map cells
  looked up from an integer index grid;
* transmission as exp(i k0 dz (n-1) * exclusive cumulative sum) instead of the
  running product of Eq. 8;
* the field as one dense exp(-i q.r) matrix product over all voxels (the 3D
  sum of Eq. 1 evaluated at the Ewald-sphere q, which Eq. 2 slices).
"""
from __future__ import annotations

import math

import numpy as np
from scipy.ndimage import map_coordinates
from scipy.special import sph_harm_y

from workloads import ELLIPSOID, RADIALMAP, SPHERE, SPHHARM, VOLUMEMAP, Geometry, Shape


def q_pixels(g: Geometry) -> np.ndarray:
    k0 = 2 * math.pi / g.wavelength
    h = math.tan(math.radians(g.theta_max_deg))
    u = np.arange(g.det_nx)
    v = np.arange(g.det_ny)
    X = h * (2 * u + 1 - g.det_nx) / g.det_nx
    Y = h * (2 * v + 1 - g.det_ny) / g.det_ny
    YY, XX = np.meshgrid(Y, X, indexing="ij")          # [v][u]
    r = np.sqrt(XX ** 2 + YY ** 2 + 1.0)
    kout = k0 * np.stack([XX / r, YY / r, 1.0 / r], axis=-1)
    q = kout - np.array([0.0, 0.0, k0])
    return q.reshape(-1, 3)


def _rodrigues(axis, ang):
    axis = np.asarray(axis, dtype=float)
    axis = axis / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(ang) * K + (1 - math.cos(ang)) * (K @ K)


def rotation(lat, lon, rot):
    """Body->lab: spin by `rot` about z, tilt z onto the main axis, then turn by longitude."""
    lat_r, lon_r, rot_r = map(math.radians, (lat, lon, rot))
    spin = _rodrigues([0, 0, 1], rot_r)
    tilt = _rodrigues([0, 1, 0], math.pi / 2 + lat_r)
    turn = _rodrigues([0, 0, 1], lon_r)
    return turn @ tilt @ spin


def real_sh(l, m, theta, phi):
    if m == 0:
        return np.real(sph_harm_y(l, 0, theta, phi))
    if m > 0:
        return math.sqrt(2) * np.real(sph_harm_y(l, m, theta, phi))
    return math.sqrt(2) * np.imag(sph_harm_y(l, -m, theta, phi))


def voxel_centres(g: Geometry):
    z = (np.arange(g.nz) - (g.nz - 1) / 2) * g.voxel
    x = (np.arange(g.nx) - (g.nx - 1) / 2) * g.voxel
    y = (np.arange(g.ny) - (g.ny - 1) / 2) * g.voxel
    Z, X, Y = np.meshgrid(z, x, y, indexing="ij")     # [z][x][y]
    return X, Y, Z


def occupancy(s: Shape, g: Geometry, soft=False, width=0.5):
    X, Y, Z = voxel_centres(g)
    d = np.stack([X - s.cx, Y - s.cy, Z - s.cz], axis=-1)
    R = rotation(s.latitude, s.longitude, s.rotation)
    p = d @ R                                          # R^T d for every voxel
    rr = np.linalg.norm(p, axis=-1)
    safe = np.where(rr > 0, rr, 1.0)
    u = np.where(rr[..., None] > 0, p / safe[..., None], np.array([0.0, 0.0, 1.0]))
    if s.kind == SPHERE:
        rs = np.full(rr.shape, s.r)
        inside = (p ** 2).sum(-1) <= s.r ** 2
    elif s.kind == ELLIPSOID:
        rs = 1.0 / np.sqrt((u[..., 0] / s.a) ** 2 + (u[..., 1] / s.b) ** 2 + (u[..., 2] / s.c) ** 2)
        inside = (p[..., 0] / s.a) ** 2 + (p[..., 1] / s.b) ** 2 + (p[..., 2] / s.c) ** 2 <= 1.0
    elif s.kind == RADIALMAP:
        rm = np.asarray(s.radial_map, dtype=float)
        nt, npf = rm.shape
        lat = np.arcsin(np.clip(u[..., 2], -1, 1))            # the same angle as atan2(p_z, |p_xy|)
        lon = np.mod(np.arctan2(p[..., 1], p[..., 0]), 2 * math.pi)
        coords = np.stack([((lat + math.pi / 2) / math.pi * nt).ravel(), (lon / (2 * math.pi) * npf).ravel()])
        rs = map_coordinates(rm, coords, order=1, mode="grid-wrap").reshape(rr.shape)
        inside = rr <= rs
    elif s.kind == VOLUMEMAP:
        inside = _vmap_lookup(s, p, np.asarray(s.volume_map, dtype=bool), False)
        return inside.astype(float)
    else:
        theta = np.arccos(np.clip(u[..., 2], -1, 1))
        phi = np.arctan2(p[..., 1], p[..., 0])
        acc = np.zeros(rr.shape)
        for l in range(1, s.lmax + 1):
            for m in range(-l, l + 1):
                acc += s.alm[l * l + l + m] * real_sh(l, m, theta, phi)
        rs = s.R0 * (1 + acc)
        hw = (min(g.nx, g.ny, g.nz) - 1) / 2 * g.voxel
        rs = np.clip(rs, 0.1 * s.R0, hw - g.voxel)
        inside = rr <= rs
    if soft:
        return 1.0 / (1.0 + np.exp(-(rs - rr) / width))
    return inside.astype(float)


def _vmap_lookup(s: Shape, p, values, outside):
    """values of the volume-map cell holding each body point p (outside: `outside`)."""
    m = np.array(values.shape)
    cell = np.floor(p / s.map_dx + m / 2.0).astype(np.int64)
    ok = ((cell >= 0) & (cell < m)).all(axis=-1)
    cc = np.where(ok[..., None], cell, 0)
    return np.where(ok, values[cc[..., 0], cc[..., 1], cc[..., 2]], outside)


def body_points(s: Shape, g: Geometry):
    X, Y, Z = voxel_centres(g)
    d = np.stack([X - s.cx, Y - s.cy, Z - s.cz], axis=-1)
    return d @ rotation(s.latitude, s.longitude, s.rotation)


def voxel_index(s: Shape, g: Geometry):
    """Per-voxel delta, beta of a volume map with a per-cell index [z][x][y]."""
    p = body_points(s, g)
    dm = s.map_delta if s.map_delta is not None else np.full(s.volume_map.shape, s.delta)
    bm = s.map_beta if s.map_beta is not None else np.full(s.volume_map.shape, s.beta)
    return _vmap_lookup(s, p, np.asarray(dm, float), s.delta), _vmap_lookup(s, p, np.asarray(bm, float), s.beta)


def slices_n(chi, g: Geometry, delta_v, beta_v):
    """Slice strength with one index per voxel: exp of the exclusive cumulative
    sum of chi (n_v - 1) along z, times (n_v^2 - 1) chi."""
    k0 = 2 * math.pi / g.wavelength
    n = 1 - delta_v + 1j * beta_v
    e = chi * (n - 1)
    E = np.cumsum(e, axis=0) - e
    return (n * n - 1) * chi * np.exp(1j * k0 * g.voxel * E)


def slices(chi, g: Geometry, delta, beta):
    k0 = 2 * math.pi / g.wavelength
    n = 1 - delta + 1j * beta
    C = np.cumsum(chi, axis=0) - chi                   # exclusive sum along z
    T = np.exp(1j * k0 * g.voxel * (n - 1) * C)
    return (n * n - 1) * chi * T


def field(rho, q, g: Geometry):
    X, Y, Z = voxel_centres(g)
    r = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=-1)
    return np.exp(-1j * (q @ r.T)) @ rho.ravel()


def forward(s: Shape, g: Geometry, q=None, soft=False, width=0.5):
    if q is None:
        q = q_pixels(g)
    chi = occupancy(s, g, soft, width)
    if s.varying_index():
        rho = slices_n(chi, g, *voxel_index(s, g))
    else:
        rho = slices(chi, g, s.delta, s.beta)
    A = field(rho, q, g)
    return np.abs(A) ** 2, A
