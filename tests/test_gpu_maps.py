"""Map shapes on the GPU (Sec. 5.2: radii map, volume map, voxel-resolved
index) against the FP64 oracle, through the C ABI.

Occupancy is integer work and is compared bit for bit (both sides decide it
in FP64 when the FP32 value is within its error bound of a surface or a cell
face).  Intensities use the modes' tolerances (relative L2): FP64 1e-10,
FP32 1e-5, tensor-core split phases 1e-3.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_l2, run_gpu
from workloads import (RADIALMAP, SPHERE, VOLUMEMAP, Geometry, Shape, core_shell_index, radialmap_96,
                       random_radial_map, random_volume_map, volumemap_96)

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "tc_f16_split": 1e-3, "tc_bf16_split": 1e-3}
G = Geometry(40, 36, 44, 1.0, 8.0, 40.0, 48, 40)


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _radial(seed=0):
    rng = np.random.default_rng(seed)
    return Shape(RADIALMAP, radial_map=random_radial_map(rng, 24, 40, 11.0), delta=0.01, beta=0.002,
                 latitude=27, longitude=-64, rotation=121, cx=0.3, cy=-0.2)


def _volume(seed=0, index=True):
    rng = np.random.default_rng(seed)
    v = random_volume_map(rng, 14)
    s = Shape(VOLUMEMAP, volume_map=v, map_dx=1.45, delta=0.012, beta=0.002, latitude=-38, longitude=71,
              rotation=40, cz=0.35)
    if index:
        s.map_delta, s.map_beta = core_shell_index(v, 0.025, 0.005, 0.007, 0.0006)
    return s


def _oracle(g, shape, soft=False, q=None):
    if q is None:
        q = oracle.detector_q(g)
    chi, _ = oracle.voxelise(shape, g, soft)
    if shape.varying_index():
        rho = oracle.slices_n(chi, g, *oracle.voxel_index(shape, g))
    else:
        rho = oracle.slices(chi, g, shape.delta, shape.beta)
    A = oracle.msft(rho, q, g.voxel)
    return chi, np.abs(A) ** 2


def _gpu_chi(g, shape, prec, soft=False):
    import paper_2202_03411_gb300 as sm
    h = sm.scatman_create(g, prec, soft=soft)
    sm.scatman_voxelise(h, shape)
    chi = sm.scatman_get_occupancy(h, (g.nz, g.nx, g.ny))
    h.close()
    return chi


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc_bf16_split"])
@pytest.mark.parametrize("which", ["radial", "volume", "volume_index"])
def test_map_occupancy_bit_exact(which, prec):
    shape = _radial() if which == "radial" else _volume(index=which == "volume_index")
    chi_ref, _ = oracle.voxelise(shape, G)
    chi = _gpu_chi(G, shape, prec)
    assert chi_ref.sum() > 500
    assert np.array_equal(chi, chi_ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc_f16_split", "tc_bf16_split"])
@pytest.mark.parametrize("which", ["radial", "volume", "volume_index"])
def test_map_intensity(which, prec):
    shape = _radial(1) if which == "radial" else _volume(1, index=which == "volume_index")
    _, I_ref = _oracle(G, shape)
    I, _ = run_gpu(G, shape, prec)
    assert rel_l2(I, I_ref) < TOL[prec], rel_l2(I, I_ref)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc_bf16_split"])
def test_soft_radial_map(prec):
    shape = _radial(2)
    chi_ref, I_ref = _oracle(G, shape, soft=True)
    chi = _gpu_chi(G, shape, prec, soft=True)
    # the occupancy buffer holds float values in every mode
    np.testing.assert_allclose(chi, chi_ref, rtol=2e-7 if prec == "fp64" else 0, atol=1e-12 if prec == "fp64" else 2e-6)
    I, _ = run_gpu(G, shape, prec, soft=True)
    assert rel_l2(I, I_ref) < TOL[prec]


def test_constant_radial_map_equals_sphere_on_gpu():
    shape = Shape(RADIALMAP, radial_map=np.full((6, 10), 9.4), delta=0.01, beta=0.002, latitude=12,
                  longitude=50, rotation=5)
    sph = Shape(SPHERE, r=9.4, delta=0.01, beta=0.002)
    for prec in ("fp64", "tc_bf16_split"):
        assert np.array_equal(_gpu_chi(G, shape, prec), _gpu_chi(G, sph, prec))
        I, _ = run_gpu(G, shape, prec)
        Is, _ = run_gpu(G, sph, prec)
        assert rel_l2(I, Is) < 1e-12


@pytest.mark.parametrize("prec", ["fp32", "tc_bf16_split"])
def test_maps_at_96_sampled_pixels(prec):
    """The 96^3 / 256^2 map workloads at the bench's launch shape: all pixels on
    the GPU, the oracle on a sample of 600 pixels."""
    rng = np.random.default_rng(0)
    for maker in (radialmap_96, volumemap_96):
        g, shapes = maker(n_shapes=1)
        s = shapes[0]
        I, _ = run_gpu(g, s, prec)
        sample = rng.choice(g.n_pix, size=600, replace=False)
        _, I_ref = _oracle(g, s, q=oracle.detector_q(g)[sample])
        assert rel_l2(I[sample], I_ref) < TOL[prec]


def test_map_shapes_have_no_gradient():
    import torch
    import paper_2202_03411_gb300 as sm
    from paper_2202_03411_gb300.api import ScatmanError
    h = sm.scatman_create(G, "tc_bf16_split", soft=True)
    I = torch.empty(G.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, _radial())
    sm.scatman_forward(h, I)
    assert sm.scatman_param_count(h) == 0
    with pytest.raises(ScatmanError) as e:
        sm.scatman_backward(h, torch.ones_like(I))
    assert e.value.code == -7                   # SCATMAN_ERR_UNSUPPORTED
    h.close()


def test_server_refuses_map_shapes():
    from paper_2202_03411_gb300.api import ScatmanError
    from paper_2202_03411_gb300.serving import Server
    srv = Server(1 << 30, slots=1)
    try:
        with pytest.raises(ScatmanError):
            srv.submit(G, _volume(), np.zeros(G.n_pix, dtype=np.float32))
    finally:
        srv.close()
