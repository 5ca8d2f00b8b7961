"""Pins of the oracle's map shapes (Sec. 5.2, "Shape (2/3)" radii map and
"Shape (3/3)" volume map) and of the voxel-resolved refractive index.

Each pin checks the oracle against something it does not share code with: a
closed form, another shape kind that must give the same occupancy, or the
independent NumPy restatement in oracle/brute.py.  None needs a GPU.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from workloads import (RADIALMAP, SPHERE, SPHHARM, VOLUMEMAP, Geometry, Shape, core_shell_index, random_alm,
                       random_radial_map, random_volume_map)

G = Geometry(24, 24, 24, 1.0, 8.0, 30.0, 16, 16)


def test_constant_radii_map_is_a_sphere():
    """A radii map holding one radius everywhere is the sphere of that radius,
    whatever the orientation (non-integer radius: no voxel centre on the surface)."""
    rm = np.full((8, 16), 7.3)
    for lat, lon, rot in [(-90, 0, 0), (20, 40, 10), (-61, 133, 250)]:
        s = Shape(RADIALMAP, radial_map=rm, delta=0.01, beta=0.001, latitude=lat, longitude=lon, rotation=rot)
        chi, _ = oracle.voxelise(s, G)
        ref, _ = oracle.voxelise(Shape(SPHERE, r=7.3), G)
        assert np.array_equal(chi, ref)


def test_radii_map_sampled_from_harmonics():
    """The map conventions (latitude rows from -pi/2, longitude columns from +x
    towards +y, body z as the pole): a fine map sampled from a harmonics radius
    renders the harmonics shape up to the interpolation error."""
    g = Geometry(40, 40, 40, 1.0, 8.0, 30.0, 8, 8)
    rng = np.random.default_rng(5)
    alm = random_alm(rng, 4, 0.15)
    sh = Shape(SPHHARM, R0=12.0, lmax=4, alm=alm, delta=0.01, beta=0.001, latitude=25, longitude=-70, rotation=35)
    nt, npf = 180, 360
    lat = -math.pi / 2 + math.pi * np.arange(nt) / nt
    lon = 2 * math.pi * np.arange(npf) / npf
    rm = np.empty((nt, npf))
    for i in range(nt):
        for k in range(npf):
            acc = sum(alm[l * l + l + m] * oracle.real_sh(l, m, math.pi / 2 - lat[i], lon[k])
                      for l in range(1, 5) for m in range(-l, l + 1))
            rm[i, k] = 12.0 * (1 + acc)
    s = Shape(RADIALMAP, radial_map=rm, delta=0.01, beta=0.001, latitude=25, longitude=-70, rotation=35)
    chi, _ = oracle.voxelise(s, g)
    ref, _ = oracle.voxelise(sh, g)
    assert ref.sum() > 4000
    # only voxels within the interpolation error of the surface may differ
    assert np.abs(chi - ref).sum() <= 0.002 * ref.sum()
    # a latitude/longitude mix-up or a flipped pole would move whole surface patches
    wrong = rm[::-1, :]
    chi_w, _ = oracle.voxelise(Shape(RADIALMAP, radial_map=wrong, latitude=25, longitude=-70, rotation=35), g)
    assert np.abs(chi_w - ref).sum() > 0.02 * ref.sum()


@pytest.mark.parametrize("soft", [False, True])
def test_radii_map_matches_numpy_restatement(soft):
    rng = np.random.default_rng(2)
    s = Shape(RADIALMAP, radial_map=random_radial_map(rng, 12, 20, 6.5), delta=0.01, beta=0.001,
              latitude=20, longitude=40, rotation=10, cx=0.3, cy=-0.4, cz=0.2)
    chi, _ = oracle.voxelise(s, G, soft=soft)
    ref = brute.occupancy(s, G, soft=soft)
    if soft:
        np.testing.assert_allclose(chi, ref, rtol=1e-12, atol=1e-14)
    else:
        assert np.array_equal(chi, ref)
    I, _ = oracle.forward(s, G, soft=soft)
    Ib, _ = brute.forward(s, G, soft=soft)
    assert oracle.relative_l2(I, Ib) < 1e-12


def test_volume_map_cube_closed_form():
    """An all-inside 10^3 map with 1.3-unit cells is the cube [-6.5, 6.5)^3:
    13 voxel centres per axis on the 24^3 grid (centres at half-integers)."""
    s = Shape(VOLUMEMAP, volume_map=np.ones((10, 10, 10), bool), map_dx=1.3, delta=0.01, beta=0.001)
    chi, _ = oracle.voxelise(s, G)
    c = np.arange(24) - 11.5
    inside = (c >= -6.5) & (c < 6.5)
    ref = inside[:, None, None] & inside[None, :, None] & inside[None, None, :]
    assert np.array_equal(chi.astype(bool), ref)
    assert int(chi.sum()) == 13 ** 3


def test_volume_map_of_a_voxelised_sphere_is_the_sphere():
    """A volume map whose cells are the grid's own voxels, filled with a
    voxelised sphere, renders that sphere exactly (cell centres land on voxel
    centres: floor(i + 1/2) = i)."""
    sph = Shape(SPHERE, r=8.6, delta=0.01, beta=0.001)
    ref, _ = oracle.voxelise(sph, G)
    vm = ref.transpose(1, 2, 0).astype(bool)          # [z][x][y] -> [x][y][z]
    s = Shape(VOLUMEMAP, volume_map=vm, map_dx=1.0, delta=0.01, beta=0.001)
    chi, _ = oracle.voxelise(s, G)
    assert np.array_equal(chi, ref)
    I, _ = oracle.forward(s, G)
    Ir, _ = oracle.forward(sph, G)
    assert oracle.relative_l2(I, Ir) < 1e-14


def test_volume_map_with_index_matches_numpy_restatement():
    rng = np.random.default_rng(3)
    v = random_volume_map(rng, 10)
    s = Shape(VOLUMEMAP, volume_map=v, map_dx=1.3, delta=0.01, beta=0.001, latitude=-30, longitude=70,
              rotation=50, cz=0.4)
    s.map_delta, s.map_beta = core_shell_index(v, 0.02, 0.004, 0.006, 0.0005)
    chi, _ = oracle.voxelise(s, G)
    assert np.array_equal(chi, brute.occupancy(s, G))
    d, b = oracle.voxel_index(s, G)
    db, bb = brute.voxel_index(s, G)
    assert np.array_equal(d, db) and np.array_equal(b, bb)
    I, _ = oracle.forward(s, G)
    Ib, _ = brute.forward(s, G)
    assert oracle.relative_l2(I, Ib) < 1e-12


def test_uniform_cell_index_equals_the_shape_index():
    """Per-cell delta, beta all equal to the shape's give the uniform result
    (the voxel-resolved form reduces to Eq. 8-9 with one n)."""
    rng = np.random.default_rng(4)
    v = random_volume_map(rng, 10)
    s = Shape(VOLUMEMAP, volume_map=v, map_dx=1.3, delta=0.012, beta=0.002, latitude=10, longitude=20,
              rotation=30)
    I0, _ = oracle.forward(s, G)
    s.map_delta = np.full(v.shape, 0.012)
    s.map_beta = np.full(v.shape, 0.002)
    I1, _ = oracle.forward(s, G)
    assert oracle.relative_l2(I1, I0) < 1e-12


def test_two_material_index_changes_the_pattern():
    """A core with a different index changes the strength and the transmission:
    the pattern moves well away from the single-material one."""
    rng = np.random.default_rng(6)
    v = random_volume_map(rng, 10)
    s = Shape(VOLUMEMAP, volume_map=v, map_dx=1.3, delta=0.006, beta=0.0005)
    I0, _ = oracle.forward(s, G)
    s.map_delta, s.map_beta = core_shell_index(v, 0.02, 0.004, 0.006, 0.0005)
    I1, _ = oracle.forward(s, G)
    assert oracle.relative_l2(I1, I0) > 0.05
