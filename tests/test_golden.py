"""Stored fixtures: the paper's printed example parameters and oracle regression values."""
import json
import math
import os

import numpy as np

import oracle
import oracle.brute as brute
from workloads import ELLIPSOID, SPHHARM, Geometry, Shape, sphere_32

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _load(name):
    with open(os.path.join(HERE, name)) as f:
        return json.load(f)


def test_sphere_32_regression():
    """Values written by tests/golden/make_golden.py (oracle only)."""
    gold = _load("sphere_32_oracle.json")
    g, (s,) = sphere_32()
    I = oracle.forward(s, g)[0].reshape(g.det_ny, g.det_nx)
    np.testing.assert_allclose(I[32], gold["central_row_v32"], rtol=1e-12)
    np.testing.assert_allclose(np.diag(I), gold["diagonal"], rtol=1e-12)
    assert abs(I.sum() - gold["total"]) <= 1e-12 * gold["total"]


def test_listing1_ellipsoid():
    """Listing 1 (Sec. 5.1): ellipsoid a=100, b=60, c=60 nm, wavelength 40 nm, 30 deg.
    Rendered on 4 nm voxels with a 48x48 detector instead of 1024x1024."""
    p = _load("listings.json")
    e = p["listing1_ellipsoid"]
    x = p["listing1_experiment"]
    vox = 4.0
    g = Geometry(56, 56, 56, vox, float(x["wavelength"]), float(x["angle_deg"]), 48, 48)
    s = Shape(ELLIPSOID, a=e["a"], b=e["b"], c=e["c"], delta=e["delta"], beta=e["beta"],
              latitude=e["latitude"], longitude=e["longitude"], rotation=e["rotation"])
    chi, _ = oracle.voxelise(s, g)
    vol = chi.sum() * vox ** 3
    assert abs(vol / (4 / 3 * math.pi * 100 * 60 * 60) - 1) < 0.03
    I, A = oracle.forward(s, g)
    assert np.all(np.isfinite(I)) and np.all(I >= 0)
    # near q = 0 every voxel adds in phase: the central pixels carry the maximum
    Ic = I.reshape(48, 48)
    assert Ic.max() == Ic[23:25, 23:25].max()


def test_listing2_harmonics_triplets():
    """Listing 2 (Sec. 5.2): the radius is the sum of the triplets c * Y_lm.
    Maps to R0 = c_00 Y_00 and a_lm = c_lm / R0 in the r = R0 (1 + sum a Y) form."""
    p = _load("listings.json")
    sh = p["listing2_sphharm"]
    trip = sh["coefficients"]
    lmax = max(t[0] for t in trip)
    R0 = trip[0][2] / math.sqrt(4 * math.pi)
    alm = np.zeros((lmax + 1) ** 2)
    for l, m, c in trip[1:]:
        alm[l * l + l + m] = c / R0
    s = Shape(SPHHARM, R0=R0, lmax=lmax, alm=alm, delta=sh["delta"], beta=sh["beta"],
              latitude=sh["latitude"], longitude=sh["longitude"], rotation=sh["rotation"])
    vox = 4.0
    g = Geometry(44, 44, 44, vox, 40.0, 30.0, 8, 8)
    chi, clipped = oracle.voxelise(s, g)
    assert not clipped
    np.testing.assert_array_equal(chi, brute.occupancy(s, g))
    # the surface radius along a few body directions equals sum c*Y directly
    rng = np.random.default_rng(0)
    for _ in range(5):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        direct = sum(c * float(brute.real_sh(l, m, th, ph)) for l, m, c in trip)
        ours = R0 * (1 + sum(alm[l * l + l + m] * oracle.real_sh(l, m, th, ph)
                             for l in range(1, lmax + 1) for m in range(-l, l + 1)))
        assert abs(direct - ours) < 1e-10 * direct
