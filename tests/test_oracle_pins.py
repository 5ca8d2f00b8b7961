"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test is chosen so that a plausible slip in the oracle (dropped term, wrong
sign or index, transposed operand, inclusive instead of exclusive scan) fails
at least one of them.  None of these tests needs a GPU.
"""
import math

import numpy as np
import pytest
import scipy.special as sps

import oracle
import oracle.brute as brute
from workloads import ELLIPSOID, SPHERE, SPHHARM, Geometry, Shape, random_alm, random_slices


def centre_phase(q, nz, nx, ny, voxel=1.0):
    """e^{+i q.c}: converts an index-origin DFT to centred voxel coordinates."""
    c = np.array([(nx - 1) / 2, (ny - 1) / 2, (nz - 1) / 2]) * voxel
    return np.exp(1j * (q @ c))


# --- Fourier sum, sign, axis order: Eq. 1-2 at on-grid q equals the 3D DFT -----

@pytest.mark.parametrize("dims", [(6, 8, 10), (1, 7, 5), (5, 4, 1)])
def test_fft_grid_pin(dims):
    nz, nx, ny = dims
    rng = np.random.default_rng(0)
    rho = random_slices(rng, nz, nx, ny)
    kz, kx, ky = np.meshgrid(np.arange(nz), np.arange(nx), np.arange(ny), indexing="ij")
    q = np.stack([2 * np.pi * kx / nx, 2 * np.pi * ky / ny, 2 * np.pi * kz / nz], -1).reshape(-1, 3)
    A = oracle.msft(rho, q)
    ref = np.fft.fftn(rho).reshape(-1) * centre_phase(q, nz, nx, ny)
    assert oracle.relative_l2(A, ref) < 1e-12


def test_small_angle_projection_pin():
    """q_z -> 0 (small-angle regime, Sec. 1): the pattern is the 2D Fourier
    transform of the projection along the beam."""
    nz, nx, ny = 7, 8, 6
    rho = random_slices(np.random.default_rng(1), nz, nx, ny)
    kx, ky = np.meshgrid(np.arange(nx), np.arange(ny), indexing="ij")
    q = np.stack([2 * np.pi * kx / nx, 2 * np.pi * ky / ny, np.zeros_like(kx, float)], -1).reshape(-1, 3)
    A = oracle.msft(rho, q)
    ref = np.fft.fft2(rho.sum(0)).reshape(-1) * centre_phase(q, 1, nx, ny)
    assert oracle.relative_l2(A, ref) < 1e-12


def test_single_slice_is_2d_dft():
    g = Geometry(9, 7, 1, 1.0, 6.0, 40.0, 11, 9)
    s = Shape(SPHERE, r=3.2, delta=0.05, beta=0.02)
    chi, _ = oracle.voxelise(s, g)
    rho = oracle.slices(chi, g, s.delta, s.beta)
    n = 1 - s.delta + 1j * s.beta
    np.testing.assert_allclose(rho, (n * n - 1) * chi, rtol=0, atol=1e-15)   # one slice: T = 1
    q = oracle.detector_q(g)
    A = oracle.msft(rho, q)
    x = np.arange(9) - 4.0
    y = np.arange(7) - 3.0
    ref = np.array([(rho[0] * np.exp(-1j * (qq[0] * x[:, None] + qq[1] * y[None, :]))).sum() for qq in q])
    assert oracle.relative_l2(A, ref) < 1e-13


# --- Detector mapping (Eq. 3) ---------------------------------------------------

def test_ewald_sphere_and_eq3():
    g = Geometry(8, 8, 8, 1.0, 7.0, 60.0, 33, 20)
    q = oracle.detector_q(g)
    k0 = 2 * math.pi / g.wavelength
    kout = q + np.array([0, 0, k0])
    np.testing.assert_allclose(np.linalg.norm(kout, axis=1), k0, rtol=1e-14)
    qxy2 = q[:, 0] ** 2 + q[:, 1] ** 2
    theta = np.arccos(np.sqrt(1 - qxy2 / k0 ** 2))      # Eq. 3
    np.testing.assert_allclose(-q[:, 2], k0 * (1 - np.cos(theta)), atol=1e-14)
    np.testing.assert_allclose(q, brute.q_pixels(g), atol=1e-14)
    # the outer pixel edge at the middle of a detector edge sits at theta_max
    h = math.tan(math.radians(g.theta_max_deg))
    pitch = 2 * h / g.det_nx
    u_last = g.det_nx - 1
    X_last = h * (2 * u_last + 1 - g.det_nx) / g.det_nx
    assert abs(math.degrees(math.atan(X_last + pitch / 2)) - g.theta_max_deg) < 1e-12
    # q_x follows the pixel column, q_y the pixel row
    qq = q.reshape(g.det_ny, g.det_nx, 3)
    assert np.all(np.diff(qq[g.det_ny // 2, :, 0]) > 0)
    assert np.all(np.diff(qq[:, g.det_nx // 2, 1]) > 0)


# --- Orientation (Fig. 6) --------------------------------------------------------

def test_rotation_conventions():
    z = np.array([0, 0, 1.0])
    np.testing.assert_allclose(oracle.rotation(90, 0, 0) @ z, [0, 0, -1], atol=1e-15)    # towards the beam
    np.testing.assert_allclose(oracle.rotation(-90, 0, 0) @ z, [0, 0, 1], atol=1e-15)    # towards the detector
    np.testing.assert_allclose(oracle.rotation(0, 0, 0) @ z, [1, 0, 0], atol=1e-15)
    np.testing.assert_allclose(oracle.rotation(0, 90, 0) @ z, [0, 1, 0], atol=1e-15)
    for lat, lon, rot in [(23, -40, 70), (-61, 170, 300), (5, 5, 5)]:
        R = oracle.rotation(lat, lon, rot)
        np.testing.assert_allclose(R.T @ R, np.eye(3), atol=1e-14)
        assert abs(np.linalg.det(R) - 1) < 1e-14
        # spinning about the main axis does not move the axis
        np.testing.assert_allclose(R @ z, oracle.rotation(lat, lon, rot + 37) @ z, atol=1e-14)
        lat_r, lon_r = math.radians(lat), math.radians(lon)
        axis = [math.cos(lat_r) * math.cos(lon_r), math.cos(lat_r) * math.sin(lon_r), -math.sin(lat_r)]
        np.testing.assert_allclose(R @ z, axis, atol=1e-14)
        np.testing.assert_allclose(R, brute.rotation(lat, lon, rot), atol=1e-14)


# --- Spherical harmonics (Eq. 10-11) ----------------------------------------------

def test_legendre_against_scipy():
    for l in range(0, 9):
        for m in range(0, l + 1):
            for x in (-0.93, -0.2, 0.0, 0.41, 0.999):
                assert abs(oracle.legendre(l, m, x) - sps.lpmv(m, l, x)) < 1e-9 * max(1, abs(sps.lpmv(m, l, x)))


def test_real_sh_against_scipy():
    rng = np.random.default_rng(3)
    for _ in range(20):
        th, ph = rng.uniform(0, math.pi), rng.uniform(-math.pi, math.pi)
        for l in range(0, 9):
            for m in range(-l, l + 1):
                assert abs(oracle.real_sh(l, m, th, ph) - float(brute.real_sh(l, m, th, ph))) < 1e-12


def test_real_sh_orthonormal():
    xg, wg = np.polynomial.legendre.leggauss(24)
    th = np.arccos(xg)
    nphi = 48
    ph = np.arange(nphi) * 2 * math.pi / nphi
    lm = [(l, m) for l in range(0, 5) for m in range(-l, l + 1)]
    Y = np.array([[[oracle.real_sh(l, m, t, p) for p in ph] for t in th] for (l, m) in lm])
    W = wg[:, None] * (2 * math.pi / nphi)
    G = np.einsum("atp,btp,tp->ab", Y, Y, np.broadcast_to(W, Y.shape[1:]))
    np.testing.assert_allclose(G, np.eye(len(lm)), atol=1e-12)


# --- Voxelisation (Block 5) ---------------------------------------------------------

def test_sphere_volume_and_sh_reduces_to_sphere():
    g = Geometry(40, 40, 40, 1.0, 8.0, 30.0, 8, 8)
    s = Shape(SPHERE, r=15.0)
    chi, _ = oracle.voxelise(s, g)
    assert abs(chi.sum() / (4 / 3 * math.pi * 15 ** 3) - 1) < 0.025   # lattice-count surface error
    alm = np.zeros(9)
    sh = Shape(SPHHARM, R0=15.0, lmax=2, alm=alm, latitude=31, longitude=12, rotation=5)
    chi2, clipped = oracle.voxelise(sh, g)
    assert not clipped
    np.testing.assert_array_equal(chi, chi2)
    el = Shape(ELLIPSOID, a=15.0, b=15.0, c=15.0, latitude=-90)
    np.testing.assert_array_equal(chi, oracle.voxelise(el, g)[0])


@pytest.mark.parametrize("soft", [False, True])
def test_voxelise_matches_numpy_restatement(soft):
    g = Geometry(14, 12, 16, 1.0, 8.0, 30.0, 4, 4)
    rng = np.random.default_rng(5)
    shapes = [
        Shape(SPHERE, r=4.7, cx=0.4, cy=-0.9, cz=0.25),
        Shape(ELLIPSOID, a=5.1, b=3.3, c=6.2, latitude=33, longitude=-120, rotation=17, cz=0.5),
        Shape(SPHHARM, R0=4.5, lmax=5, alm=random_alm(rng, 5, 0.1), latitude=-10, longitude=80, rotation=200),
    ]
    for s in shapes:
        a, _ = oracle.voxelise(s, g, soft=soft)
        b = brute.occupancy(s, g, soft=soft)
        if soft:
            np.testing.assert_allclose(a, b, atol=1e-12)
        else:
            np.testing.assert_array_equal(a, b)


# --- Transmission (Eq. 8) ------------------------------------------------------------

def test_exclusive_scan_on_one_column():
    g = Geometry(1, 1, 4, 1.0, 5.0, 30.0, 1, 1)
    chi = np.array([1.0, 1.0, 0.0, 1.0]).reshape(4, 1, 1)
    d, b = 0.03, 0.01
    rho = oracle.slices(chi, g, d, b)
    n = 1 - d + 1j * b
    ph = np.exp(1j * 2 * math.pi / g.wavelength * g.voxel * (n - 1))
    expect = (n * n - 1) * np.array([1.0, ph, 0.0, ph ** 2])   # slice 0 sees E_0 = 1
    np.testing.assert_allclose(rho.ravel(), expect, atol=1e-15)


def test_transmission_closed_form_convex():
    """Homogeneous convex body: C_j = j - j_entry inside (product form vs closed form)."""
    g = Geometry(20, 20, 20, 1.0, 8.0, 30.0, 4, 4)
    s = Shape(ELLIPSOID, a=7.5, b=5.5, c=8.5, delta=0.02, beta=0.005, latitude=20, longitude=10, rotation=40)
    chi, _ = oracle.voxelise(s, g)
    rho = oracle.slices(chi, g, s.delta, s.beta)
    n = 1 - s.delta + 1j * s.beta
    k0 = 2 * math.pi / g.wavelength
    inside = chi > 0
    first = np.where(inside.any(0), inside.argmax(0), 0)        # entry slice per column
    j = np.arange(g.nz)[:, None, None]
    T = np.exp(1j * k0 * g.voxel * (n - 1) * (j - first[None]))
    np.testing.assert_allclose(rho[inside], ((n * n - 1) * T)[inside], rtol=1e-13)
    assert np.all(rho[~inside] == 0)


def test_scan_direction_matters_with_absorption():
    g = Geometry(16, 16, 16, 1.0, 6.0, 45.0, 12, 12)
    s = Shape(ELLIPSOID, a=6.0, b=4.0, c=7.0, delta=0.03, beta=0.02, latitude=30, longitude=0, rotation=0)
    chi, _ = oracle.voxelise(s, g)
    q = oracle.detector_q(g)
    I1 = np.abs(oracle.msft(oracle.slices(chi, g, s.delta, s.beta), q)) ** 2
    rev = oracle.slices(chi[::-1].copy(), g, s.delta, s.beta)[::-1].copy()
    I2 = np.abs(oracle.msft(rev, q)) ** 2
    assert oracle.relative_l2(I2, I1) > 1e-3


# --- Born limit: homogeneous sphere form factor (Eq. 1) ----------------------------

def test_born_sphere_form_factor():
    g = Geometry(32, 32, 32, 1.0, 8.0, 30.0, 64, 64)
    s = Shape(SPHERE, r=12.0, delta=1e-3, beta=1e-4)
    chi, _ = oracle.voxelise(s, g)
    n = 1 - s.delta + 1j * s.beta
    q = oracle.detector_q(g)
    A = oracle.msft((n * n - 1) * chi, q)          # T = 1: Born approximation
    I = np.abs(A) ** 2
    V = chi.sum()
    Reff = (3 * V / (4 * math.pi)) ** (1 / 3)
    x = np.linalg.norm(q, axis=1) * Reff
    ff = 3 * (np.sin(x) - x * np.cos(x)) / x ** 3
    Iref = (abs(n * n - 1) * V) ** 2 * ff ** 2
    sel = x < 6
    assert oracle.relative_l2(I[sel], Iref[sel]) < 0.05
    # the first minimum (qR = 4.493) along the detector's central row
    row = I.reshape(64, 64)[32]
    xr = x.reshape(64, 64)[32]
    half = row[32:]
    imin = np.argmin(half[np.argmax(xr[32:] > 3.5):]) + np.argmax(xr[32:] > 3.5)
    pitch = xr[33] - xr[32]
    assert abs(xr[32:][imin] - 4.4934) < 1.5 * pitch


def test_born_limit_strength_scale():
    """delta, beta -> 0: I -> |n^2-1|^2 |F[chi]|^2 (strength ~ n^2-1, Eq. 5-6)."""
    g = Geometry(12, 12, 12, 1.0, 6.0, 40.0, 9, 9)
    s = Shape(ELLIPSOID, a=4.0, b=3.0, c=5.0, delta=1e-7, beta=3e-8, latitude=12, longitude=50)
    I, _ = oracle.forward(s, g)
    chi, _ = oracle.voxelise(s, g)
    n = 1 - s.delta + 1j * s.beta
    F = oracle.msft(chi.astype(complex), oracle.detector_q(g))
    np.testing.assert_allclose(I, abs(n * n - 1) ** 2 * np.abs(F) ** 2, rtol=1e-5)


# --- Exact discrete symmetries ---------------------------------------------------------

def test_mirror_and_c2_symmetry():
    g = Geometry(20, 20, 20, 1.0, 7.0, 45.0, 24, 24)
    s = Shape(ELLIPSOID, a=7.0, b=4.5, c=8.0, delta=0.02, beta=0.01, latitude=-90, longitude=0, rotation=0)
    I, _ = oracle.forward(s, g)
    I = I.reshape(24, 24)
    np.testing.assert_allclose(I, I[:, ::-1], rtol=1e-11)        # x mirror
    np.testing.assert_allclose(I, I[::-1, :], rtol=1e-11)        # y mirror
    np.testing.assert_allclose(I, I[::-1, ::-1], rtol=1e-11)     # C2 about z
    sph = Shape(SPHERE, r=7.3, delta=0.02, beta=0.01)
    I2, _ = oracle.forward(sph, g)
    I2 = I2.reshape(24, 24)
    np.testing.assert_allclose(I2, I2.T, rtol=1e-11)             # D4 diagonal
    # tilting the ellipsoid out of the mirror plane breaks the x mirror
    t = Shape(ELLIPSOID, a=7.0, b=4.5, c=8.0, delta=0.02, beta=0.01, latitude=-60, longitude=0, rotation=0)
    I3 = oracle.forward(t, g)[0].reshape(24, 24)
    assert oracle.relative_l2(I3[:, ::-1], I3) > 1e-3


def test_integer_translation_invariance():
    g = Geometry(22, 22, 22, 1.0, 7.0, 45.0, 16, 16)
    s = Shape(ELLIPSOID, a=6.0, b=4.0, c=7.0, delta=0.02, beta=0.01, latitude=20, longitude=60, rotation=10)
    I0, A0 = oracle.forward(s, g)
    t = s.copy()
    t.cx, t.cy, t.cz = 2.0, -1.0, 1.0
    I1, A1 = oracle.forward(t, g)
    np.testing.assert_allclose(I1, I0, rtol=1e-10, atol=1e-12 * I0.max())
    q = oracle.detector_q(g)
    np.testing.assert_allclose(A1, A0 * np.exp(-1j * (q @ np.array([2.0, -1.0, 1.0]))), rtol=1e-10,
                               atol=1e-10 * np.abs(A0).max())


# --- Whole path against the independent NumPy restatement (tiny grids) -------------------

@pytest.mark.parametrize("soft", [False, True])
def test_oracle_vs_bruteforce(soft):
    g = Geometry(8, 8, 8, 1.0, 5.0, 45.0, 16, 16)
    rng = np.random.default_rng(11)
    shapes = [
        Shape(SPHERE, r=3.1, delta=0.02, beta=0.002),
        Shape(ELLIPSOID, a=3.5, b=2.2, c=3.0, delta=0.05, beta=0.02, latitude=40, longitude=30, rotation=15),
        Shape(SPHHARM, R0=2.8, lmax=4, alm=random_alm(rng, 4, 0.1), delta=0.01, beta=0.001,
              latitude=30, longitude=-40, rotation=0),
    ]
    for s in shapes:
        I, A = oracle.forward(s, g, soft=soft)
        Ib, Ab = brute.forward(s, g, soft=soft)
        assert oracle.relative_l2(A, Ab) < 1e-13
        assert oracle.relative_l2(I, Ib) < 1e-13


# --- Adjoint and gradient ------------------------------------------------------------------

def test_adjoint_dot_product():
    rng = np.random.default_rng(2)
    nz, nx, ny = 5, 6, 7
    rho = random_slices(rng, nz, nx, ny)
    q = rng.uniform(-1, 1, size=(40, 3))
    g = rng.normal(size=40) + 1j * rng.normal(size=40)
    lhs = np.vdot(oracle.msft(rho, q), g)
    rhs = np.vdot(rho.ravel(), oracle.msft_adjoint(g, q, (nz, nx, ny)).ravel())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def _loss_and_grad(s, g, target_I, width):
    I, A = oracle.forward(s, g, soft=True, width=width)
    dLdI = 2 * (I - target_I)
    return float(((I - target_I) ** 2).sum()), oracle.gradient(s, g, dLdI, A, width=width)


def _params(s):
    if s.kind == SPHERE:
        return [("r", None)]
    if s.kind == ELLIPSOID:
        return [("a", None), ("b", None), ("c", None)]
    return [("alm", k) for k in range(1, (s.lmax + 1) ** 2)] + [("R0", None)]


def _bump(s, name, k, h):
    t = s.copy()
    if name == "alm":
        t.alm[k] += h
    else:
        setattr(t, name, getattr(t, name) + h)
    return t


@pytest.mark.parametrize("kind", [SPHERE, ELLIPSOID, SPHHARM])
def test_gradient_central_differences(kind):
    g = Geometry(14, 14, 14, 1.0, 5.0, 45.0, 10, 10)
    rng = np.random.default_rng(kind)
    if kind == SPHERE:
        s = Shape(SPHERE, r=4.3, delta=0.03, beta=0.004, cx=0.2)
    elif kind == ELLIPSOID:
        s = Shape(ELLIPSOID, a=4.5, b=3.1, c=5.2, delta=0.03, beta=0.004, latitude=25, longitude=40, rotation=60)
    else:
        s = Shape(SPHHARM, R0=4.0, lmax=2, alm=random_alm(rng, 2, 0.1), delta=0.03, beta=0.004,
                  latitude=15, longitude=-30, rotation=80)
    t = s.copy()
    t.delta *= 1.1
    t.beta *= 0.9
    for name, k in _params(s):
        t = _bump(t, name, k, 0.05 if name == "alm" else 0.2)
    width = 0.7
    target = oracle.forward(t, g, soft=True, width=width)[0]
    L0, grad = _loss_and_grad(s, g, target, width)
    names = _params(s) + [("delta", None), ("beta", None)]
    assert len(grad) == len(names) == s.n_params()
    for i, (name, k) in enumerate(names):
        base = s.alm[k] if name == "alm" else getattr(s, name)
        h = 1e-4 * (0.05 if name == "alm" else abs(base))
        Lp = _loss_and_grad(_bump(s, name, k, h), g, target, width)[0]
        Lm = _loss_and_grad(_bump(s, name, k, -h), g, target, width)[0]
        fd = (Lp - Lm) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(grad).max()), (name, k, fd, grad[i])


# --- The paper's uniform-q virtual detector (Block 1, Block 6) -------------------------

def test_uniform_q_detector():
    from workloads import DETECTOR_UNIFORM_Q
    g = Geometry(8, 8, 8, 1.0, 4.0, 60.0, 21, 17, DETECTOR_UNIFORM_Q)
    q = oracle.detector_q(g).reshape(17, 21, 3)
    valid = oracle.detector_valid(g).reshape(17, 21)
    k0 = 2 * math.pi / g.wavelength
    qmax = k0 * math.sin(math.radians(60.0))
    # separable: q_x depends on the column only, q_y on the row only, uniform spacing
    assert np.all(q[:, :, 0] == q[:1, :, 0]) and np.all(q[:, :, 1] == q[:, :1, 1])
    np.testing.assert_allclose(np.diff(q[0, :, 0]), 2 * qmax / 21, rtol=1e-12)
    np.testing.assert_allclose(q[0, -1, 0] + qmax / 21, qmax, rtol=1e-14)       # outer pixel edge at theta_max
    # Ewald sphere on the valid pixels; corners beyond k0 are invalid at 60 deg
    kout = q + np.array([0, 0, k0])
    np.testing.assert_allclose(np.linalg.norm(kout[valid], axis=-1), k0, rtol=1e-13)
    assert not valid.all() and valid[8, 10]
    np.testing.assert_array_equal(valid, q[:, :, 0] ** 2 + q[:, :, 1] ** 2 <= k0 ** 2)
    s = Shape(SPHERE, r=2.5, delta=0.02, beta=0.004)
    I, _ = oracle.forward(s, g)
    assert np.all(I.reshape(17, 21)[~valid] == 0) and np.all(I.reshape(17, 21)[valid] > 0)
