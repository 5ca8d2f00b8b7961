"""Pins of the oracle's Ideal detector (Sec. 5.2, Listing 2: photon statistics).

The counts come from a counter-based generator (Philox-4x32-10) and a Poisson
sampler (Knuth's multiplication method below lambda = 12, Hormann's PTRS
above); the expected counts from the pixel solid angle and the scattering
cross-section.  Each pin checks against something independent: the Poisson
law (scipy), closed-form solid angles, a fine numerical integral, the
textbook Born cross-section of a sphere.  None needs a GPU.
"""
import math

import numpy as np
import pytest
import scipy.stats as st

import oracle
from workloads import SPHERE, Geometry, Shape

G = Geometry(8, 8, 8, 1.0, 8.0, 30.0, 128, 128)


def _lambda_field(lams, g=G):
    """Intensities that give each pixel an expected count from `lams` (cycled)."""
    dom = oracle.pixel_solid_angle(g)
    k0 = 2 * math.pi / g.wavelength
    amp = k0 * k0 * g.voxel ** 3 / (4 * math.pi)
    target = np.resize(np.asarray(lams, float), g.n_pix)
    return target / (amp * amp * dom)                 # photon density 1


# Known-answer vectors of Philox-4x32-10 published with the generator by its
# authors (Salmon, Moraes, Dror and Shaw, "Parallel random numbers: as easy as
# 1, 2, 3", SC'11; the Random123 distribution's known-answer test list):
# (counter words 0-3, key words 0-1) -> output words 0-3.
PHILOX_KAT = [
    ((0x00000000, 0x00000000, 0x00000000, 0x00000000), (0x00000000, 0x00000000),
     (0x6627e8d5, 0xe169c58d, 0xbc57ac4c, 0x9b00dbd8)),
    ((0xffffffff, 0xffffffff, 0xffffffff, 0xffffffff), (0xffffffff, 0xffffffff),
     (0x408f276d, 0x41c83b0e, 0xa20bc7c6, 0x6d5451fd)),
    ((0x243f6a88, 0x85a308d3, 0x13198a2e, 0x03707344), (0xa4093822, 0x299f31d0),
     (0xd16cfe09, 0x94fdcceb, 0x5001e420, 0x24126ea1)),
]


@pytest.mark.parametrize("counter,key,expected", PHILOX_KAT)
def test_philox_known_answers(counter, key, expected):
    """A wrong round count, multiplier, Weyl key increment or word order fails
    at least one of the three published vectors."""
    got = [int(v) for v in oracle.philox(counter, key)]
    assert got == list(expected), [hex(v) for v in got]


def test_philox_uniform_and_avalanche():
    rng = np.random.default_rng(0)
    words = np.array([oracle.philox([i, 0, 0, 0], [123, 456]) for i in range(4000)]).ravel()
    # the top byte of every output word is uniform
    counts = np.bincount((words >> 24).astype(np.int64), minlength=256)
    assert st.chisquare(counts).pvalue > 1e-4
    # flipping one counter or key bit changes about half of the 128 output bits
    flips = []
    for _ in range(200):
        c = [int(v) for v in rng.integers(0, 2 ** 32, size=4)]
        k = [int(v) for v in rng.integers(0, 2 ** 32, size=2)]
        a = oracle.philox(c, k)
        c2 = list(c)
        bit = int(rng.integers(0, 128))
        c2[bit // 32] ^= 1 << (bit % 32)
        b = oracle.philox(c2, k)
        flips.append(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a, b)))
    assert 60 < np.mean(flips) < 68
    k = [1, 2]
    k2 = [1 ^ 1, 2]
    assert not np.array_equal(oracle.philox([5, 6, 7, 8], k), oracle.philox([5, 6, 7, 8], k2))


@pytest.mark.parametrize("lam", [0.3, 2.5, 11.9, 12.0, 37.0, 1000.0, 1.0e5])
def test_poisson_mean_and_variance(lam):
    I = _lambda_field([lam])
    lam_out, c = oracle.photon_counts(I, G, 1.0, seed=11)
    np.testing.assert_allclose(lam_out, lam, rtol=1e-12)
    n = c.size
    assert abs(c.mean() - lam) < 5 * math.sqrt(lam / n)
    # variance of the sample variance of a Poisson law ~ (lam + 2 lam^2) / n
    assert abs(c.var() - lam) < 5 * math.sqrt((lam + 2 * lam * lam) / n)
    assert c.min() >= 0


@pytest.mark.parametrize("lam", [3.0, 40.0])
def test_poisson_law_chi_square(lam):
    I = _lambda_field([lam])
    counts = np.concatenate([oracle.photon_counts(I, G, 1.0, seed=s)[1] for s in range(4)])
    kmax = int(lam + 6 * math.sqrt(lam)) + 1
    kmin = max(0, int(lam - 6 * math.sqrt(lam)))
    obs = np.array([(counts == k).sum() for k in range(kmin, kmax)], float)
    exp_ = st.poisson.pmf(np.arange(kmin, kmax), lam) * counts.size
    keep = exp_ > 20
    obs, exp_ = obs[keep], exp_[keep]
    exp_ *= obs.sum() / exp_.sum()
    assert st.chisquare(obs, exp_).pvalue > 1e-4


def test_zero_and_seeds():
    I = _lambda_field([0.0, 5.0])
    _, c1 = oracle.photon_counts(I, G, 1.0, seed=3)
    _, c2 = oracle.photon_counts(I, G, 1.0, seed=3)
    _, c3 = oracle.photon_counts(I, G, 1.0, seed=4)
    assert np.array_equal(c1, c2) and not np.array_equal(c1, c3)
    assert (c1[::2] == 0).all()


def test_flat_pixel_solid_angles():
    """The pixels tile the detector: their solid angles add up to the exact
    solid angle of a square of half-width h at distance 1,
    4 atan(h^2 / sqrt(1 + 2 h^2)); a corner pixel matches a fine integral."""
    for theta in (30.0, 60.0):
        g = Geometry(8, 8, 8, 1.0, 8.0, theta, 256, 256)
        dom = oracle.pixel_solid_angle(g)
        h = math.tan(math.radians(theta))
        exact = 4 * math.atan(h * h / math.sqrt(1 + 2 * h * h))
        assert abs(dom.sum() / exact - 1) < 1e-4
        # corner pixel (u = v = 0) by a 200 x 200 midpoint integral of dA / r^3
        w = 2 * h / 256
        s = -h + (np.arange(200) + 0.5) * w / 200
        X, Y = np.meshgrid(s, s)
        ref = ((w / 200) ** 2 / (1 + X ** 2 + Y ** 2) ** 1.5).sum()
        assert abs(dom[0] / ref - 1) < 1e-4


def test_uniform_q_pixel_solid_angles():
    """On the uniform-q detector d2q = k0^2 cos(theta) dOmega: the valid pixels
    add up to the solid angle of the directions whose q_perp lies in the
    square |q_x|, |q_y| <= q_max (a fine integral over the square)."""
    g = Geometry(8, 8, 8, 1.0, 8.0, 40.0, 128, 128, 1)
    dom = oracle.pixel_solid_angle(g)
    k0 = 2 * math.pi / g.wavelength
    qmax = k0 * math.sin(math.radians(40.0))
    s = (np.arange(1000) + 0.5) / 1000 * 2 * qmax - qmax
    QX, QY = np.meshgrid(s, s)
    c = np.sqrt(np.clip(1 - (QX ** 2 + QY ** 2) / k0 ** 2, 1e-300, None))
    ref = ((2 * qmax / 1000) ** 2 / (k0 ** 2 * c)).sum()
    assert abs(dom.sum() / ref - 1) < 1e-3
    # a pixel with no scattering direction collects nothing
    g2 = Geometry(8, 8, 8, 1.0, 8.0, 85.0, 64, 64, 1)
    assert oracle.pixel_solid_angle(g2)[0] == 0.0


def test_born_sphere_photon_normalisation():
    """With the transmission switched off (delta, beta -> 0 in T only is not
    available, so use a weak sphere) the expected counts follow the textbook
    cross-section dsigma/dOmega = (k0^2 |n^2 - 1| V / (4 pi))^2 F(qR)^2 with
    F the sphere form factor, times the photon density and the pixel's solid
    angle (up to the voxel staircase, 5 %)."""
    g = Geometry(32, 32, 32, 1.0, 8.0, 20.0, 48, 48)
    s = Shape(SPHERE, r=9.0, delta=1e-6, beta=0.0)
    I, _ = oracle.forward(s, g)
    lam, _ = oracle.photon_counts(I, g, 2.5, seed=0, counts=False)
    q = oracle.detector_q(g)
    qq = np.linalg.norm(q, axis=1)
    chi, _ = oracle.voxelise(s, g)
    V = chi.sum()
    k0 = 2 * math.pi / g.wavelength
    n = 1 - 1e-6
    x = qq * 9.0
    F = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    ref = 2.5 * (k0 ** 2 * abs(n * n - 1) * V / (4 * math.pi)) ** 2 * F ** 2 * oracle.pixel_solid_angle(g)
    sel = x < 3.0                     # the main lobe, where the staircase matters least
    assert oracle.relative_l2(lam[sel], ref[sel]) < 0.05
