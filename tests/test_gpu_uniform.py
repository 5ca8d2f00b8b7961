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
