"""The uniform-q virtual detector's separable path against the oracle."""
import numpy as np
import pytest

import oracle
from gpu_helpers import oracle_field, rel_l2, run_gpu
from workloads import (DETECTOR_UNIFORM_Q, ELLIPSOID, SPHHARM, Geometry, Shape, fig8b_case, random_alm)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-5)])
def test_uniform_q_parity(prec, tol):
    rng = np.random.default_rng(0)
    cases = [
        (Geometry(21, 19, 23, 1.0, 7.0, 30.0, 45, 37, DETECTOR_UNIFORM_Q),
         Shape(ELLIPSOID, a=7.0, b=5.0, c=9.0, delta=0.02, beta=0.004, latitude=20, longitude=40, rotation=60)),
        (Geometry(24, 24, 24, 1.0, 5.0, 60.0, 64, 64, DETECTOR_UNIFORM_Q),      # corners off the Ewald sphere
         Shape(SPHHARM, R0=7.0, lmax=6, alm=random_alm(rng, 6), delta=0.01, beta=0.001, latitude=-10,
               longitude=80, rotation=200)),
        fig8b_case(3.0, 96),
    ]
    for g, s in cases:
        I, A = run_gpu(g, s, prec)
        Ir, Ar = oracle_field(g, s)
        Ar = np.where(oracle.detector_valid(g), Ar, 0.0)
        Ir = np.abs(Ar) ** 2
        assert rel_l2(I, Ir) < tol, (g, rel_l2(I, Ir))
        assert np.all(I[~oracle.detector_valid(g)] == 0.0)


def test_uniform_q_matches_the_general_path():
    """The separable sums equal the general per-pixel sum on the same q."""
    g, s = fig8b_case(5.0, 64)
    I_sep, _ = run_gpu(g, s, "fp64")
    q = oracle.detector_q(g)
    flat = Geometry(g.nx, g.ny, g.nz, g.voxel, g.wavelength, g.theta_max_deg, g.det_nx, g.det_ny)
    I_gen, _ = run_gpu(flat, s, "fp64", q_list=q)
    assert rel_l2(I_sep, I_gen) < 1e-11


def test_uniform_q_gradient_fp32():
    """The backward pass needs nothing detector-specific: gradient against the oracle."""
    import torch
    import paper_2202_03411_gb300 as sm
    from workloads import perturbed
    g = Geometry(18, 18, 18, 1.0, 5.0, 45.0, 30, 30, DETECTOR_UNIFORM_Q)
    s = Shape(ELLIPSOID, a=6.0, b=4.0, c=7.0, delta=0.03, beta=0.004, latitude=25, longitude=40, rotation=60)
    t = perturbed(s, np.random.default_rng(1), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=0.6)[0]
    I_ref, A = oracle.forward(s, g, soft=True, width=0.6)
    h = sm.scatman_create(g, "fp32", soft=True, soft_width=0.6)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I)
    w = 2 * (I - torch.as_tensor(target, dtype=torch.float32, device="cuda"))
    grad = sm.scatman_backward(h, w)
    h.close()
    ref = oracle.gradient(s, g, w.double().cpu().numpy(), A, width=0.6)
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) < 1e-4


TC_PRECISIONS = [("tc_f16_split", 1e-3), ("tc_bf16_split", 1e-3), ("tc_f16", 2e-3), ("tc_bf16", 3e-3)]


@pytest.mark.parametrize("prec,tol", TC_PRECISIONS)
def test_uniform_q_tensor_core_parity(prec, tol):
    """The x/z sum on the tensor cores: ragged pixel tiles (u), detector rows
    grouped 8/4/2/1 per GEMM column block with a ragged last group, padded z (16)
    and x (64) extents, pixels off the Ewald sphere, the largest grid the
    operand tile holds (nx = nz = 128)."""
    rng = np.random.default_rng(3)
    cases = [
        (Geometry(21, 19, 23, 1.0, 7.0, 30.0, 300, 137, DETECTOR_UNIFORM_Q),
         Shape(ELLIPSOID, a=7.0, b=5.0, c=9.0, delta=0.02, beta=0.004, latitude=20, longitude=40, rotation=60)),
        (Geometry(65, 30, 9, 1.0, 6.0, 60.0, 129, 40, DETECTOR_UNIFORM_Q),      # x pads to 128, z to 16
         Shape(ELLIPSOID, a=28.0, b=12.0, c=4.0, delta=0.01, beta=0.002, latitude=5, longitude=10, rotation=30)),
        (Geometry(24, 24, 24, 1.0, 5.0, 60.0, 64, 64, DETECTOR_UNIFORM_Q),      # corners off the Ewald sphere
         Shape(SPHHARM, R0=7.0, lmax=6, alm=random_alm(rng, 6), delta=0.01, beta=0.001, latitude=-10,
               longitude=80, rotation=200)),
        (Geometry(30, 26, 40, 1.0, 6.0, 40.0, 150, 51, DETECTOR_UNIFORM_Q),     # z pads to 48: 2 rows per group
         Shape(ELLIPSOID, a=12.0, b=9.0, c=17.0, delta=0.015, beta=0.002, latitude=-35, longitude=75, rotation=120)),
        (Geometry(128, 40, 128, 1.0, 12.0, 30.0, 131, 3, DETECTOR_UNIFORM_Q),  # the largest operand tile
         Shape(ELLIPSOID, a=50.0, b=15.0, c=55.0, delta=0.004, beta=0.0005, latitude=30, longitude=-50, rotation=10)),
        fig8b_case(3.0, 96),
    ]
    for g, s in cases:
        I, A = run_gpu(g, s, prec)
        Ir, Ar = oracle_field(g, s)
        Ar = np.where(oracle.detector_valid(g), Ar, 0.0)
        Ir = np.abs(Ar) ** 2
        assert rel_l2(I, Ir) < tol, (prec, g, rel_l2(I, Ir))
        assert np.all(I[~oracle.detector_valid(g)] == 0.0)


def test_uniform_q_tensor_core_gradient():
    """The backward pass after a tensor-core forward (the adjoint runs in FP32 on the
    CUDA cores from the tensor-core field)."""
    import torch
    import paper_2202_03411_gb300 as sm
    from workloads import perturbed
    g = Geometry(18, 18, 18, 1.0, 5.0, 45.0, 30, 30, DETECTOR_UNIFORM_Q)
    s = Shape(ELLIPSOID, a=6.0, b=4.0, c=7.0, delta=0.03, beta=0.004, latitude=25, longitude=40, rotation=60)
    t = perturbed(s, np.random.default_rng(1), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=0.6)[0]
    _, A = oracle.forward(s, g, soft=True, width=0.6)
    h = sm.scatman_create(g, "tc_bf16_split", soft=True, soft_width=0.6)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I)
    w = 2 * (I - torch.as_tensor(target, dtype=torch.float32, device="cuda"))
    grad = sm.scatman_backward(h, w)
    h.close()
    ref = oracle.gradient(s, g, w.double().cpu().numpy(), A, width=0.6)
    assert np.linalg.norm(grad - ref) / np.linalg.norm(ref) < 1e-3


def test_uniform_q_tensor_core_matches_fp32_on_fig8b_grids():
    """Fig. 8b grids (harmonics shape at 3 and 10 wavelengths) on a 256^2 detector:
    tensor-core modes within their tolerance of the FP32 CUDA-core sums."""
    for R in (3.0, 10.0):
        g, s = fig8b_case(R, 256)
        I32, _ = run_gpu(g, s, "fp32")
        for prec, tol in TC_PRECISIONS:
            I, _ = run_gpu(g, s, prec)
            assert rel_l2(I, I32) < tol, (R, prec, rel_l2(I, I32))


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc_bf16_split", "tc_f16"])
@pytest.mark.parametrize("detector", [0, DETECTOR_UNIFORM_Q])
def test_footprint_covers_the_handle(prec, detector):
    """The host-side footprint estimate (used for admission) is at least what a
    handle allocates after a forward and a backward."""
    import torch
    import paper_2202_03411_gb300 as sm
    from paper_2202_03411_gb300.serving import footprint_bytes
    g = Geometry(40, 36, 44, 1.0, 6.0, 30.0, 200, 170, detector)
    s = Shape(ELLIPSOID, a=14.0, b=11.0, c=16.0, delta=0.01, beta=0.001, latitude=10, longitude=20, rotation=30)
    h = sm.scatman_create(g, prec, soft=True, soft_width=0.6)
    I = torch.empty(g.n_pix, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I)
    sm.scatman_backward(h, torch.ones_like(I))
    used = sm.scatman_device_bytes(h)
    h.close()
    assert used <= footprint_bytes(g, prec), (used, footprint_bytes(g, prec))


@pytest.mark.parametrize("prec,tol", [("tc_bf16_split", 1e-3), ("fp32", 1e-5)])
def test_uniform_q_fig8b_worst_case_sampled(prec, tol):
    """Fig. 8b's largest case (harmonics shape at 20 wavelengths, 56^3, 2048^2
    uniform-q detector) in the configuration the benchmark times: the central
    pixels plus a uniform sample of the rest against the oracle."""
    g, s = fig8b_case(20.0, 2048)
    rng = np.random.default_rng(11)
    centre = [(g.det_ny // 2 + dv) * g.det_nx + g.det_nx // 2 + du for dv in range(-4, 4) for du in range(-4, 4)]
    sample = np.unique(np.concatenate([np.array(centre), rng.choice(g.n_pix, size=960, replace=False)]))
    Ir, Ar = oracle_field(g, s, sample=sample)
    valid = oracle.detector_valid(g)[sample]
    Ir = np.where(valid, Ir, 0.0)
    I, _ = run_gpu(g, s, prec)
    err = rel_l2(I[sample], Ir)
    assert err < tol, err
    assert np.all(I[sample][~valid] == 0.0)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc_f16_split", "tc_bf16"])
def test_uniform_q_edge_cases(prec):
    """Empty shape (exactly zero), a single slice, a single pixel, a one-row
    detector, and a one-voxel grid on the uniform-q detector."""
    from workloads import SPHERE
    # A handful of nearly coherent terms does not average rounding out: with one
    # BF16 phase product the bound is the coherent one, I off by at most
    # 2 (2^-9 phase + 2^-9 data) = 7.8e-3 (the 3e-3 of larger grids relies on
    # averaging over many terms).
    tol = {"fp64": 1e-10, "fp32": 1e-5, "tc_f16_split": 1e-3, "tc_bf16": 7.8e-3}[prec]
    g = Geometry(16, 16, 16, 1.0, 6.0, 30.0, 20, 20, DETECTOR_UNIFORM_Q)
    empty = Shape(SPHERE, r=0.1, cx=0.25, cy=0.25, cz=0.25, delta=0.01, beta=0.001)
    I, _ = run_gpu(g, empty, prec)
    assert np.all(I == 0.0)
    s = Shape(SPHERE, r=3.0, delta=0.02, beta=0.01)
    for g in (Geometry(9, 9, 1, 1.0, 6.0, 30.0, 5, 4, DETECTOR_UNIFORM_Q),
              Geometry(9, 9, 9, 1.0, 6.0, 30.0, 1, 1, DETECTOR_UNIFORM_Q),
              Geometry(9, 9, 9, 1.0, 6.0, 30.0, 131, 1, DETECTOR_UNIFORM_Q),
              Geometry(1, 1, 1, 1.0, 6.0, 30.0, 3, 2, DETECTOR_UNIFORM_Q)):
        I, _ = run_gpu(g, s, prec)
        Ir, Ar = oracle_field(g, s)
        Ir = np.abs(np.where(oracle.detector_valid(g), Ar, 0.0)) ** 2
        assert rel_l2(I, Ir) < tol, (g, prec, rel_l2(I, Ir))
