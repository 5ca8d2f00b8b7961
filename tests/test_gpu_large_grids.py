"""Grids past the old tensor-core limits, against the FP64 oracle.

nx = 160: slices wider than 128 columns are cut into two work units of the
contraction (each with its own y range), which must sum to the same field.
nz = 320: the voxeliser's transmission scan runs ten z values per lane, the
contraction's unit list and slice phases cover more than 256 slices, and the
gradient's per-voxel pass holds sixteen z values per lane.
Tolerances are the parity tests': tensor-core split modes 1e-3, FP32 1e-5
(relative L2 of I); gradients 1e-3 in the tensor-core modes.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import oracle_field, rel_l2, run_gpu
from workloads import ELLIPSOID, SPHHARM, Geometry, Shape, random_alm

pytestmark = pytest.mark.gpu

TOL = {"fp32": 1e-5, "tc_f16_split": 1e-3, "tc_bf16_split": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _sample(g, n, seed):
    rng = np.random.default_rng(seed)
    centre = [(g.det_ny // 2 + dv) * g.det_nx + g.det_nx // 2 + du for dv in range(-3, 3) for du in range(-3, 3)]
    return np.unique(np.concatenate([np.array(centre), rng.choice(g.n_pix, size=n, replace=False)]))


@pytest.mark.parametrize("prec", ["tc_f16_split", "tc_bf16_split", "fp32"])
def test_wide_grid_nx_160(prec):
    import paper_2202_03411_gb300 as sm
    g = Geometry(160, 56, 48, 1.0, 9.0, 45.0, 140, 120)
    s = Shape(ELLIPSOID, a=70.0, b=20.0, c=16.0, delta=0.015, beta=0.002, latitude=-85.0, longitude=12.0,
              rotation=30.0, cx=1.3)
    sample = _sample(g, 700, 1)
    Ir, _ = oracle_field(g, s, sample=sample)
    I, A, h = run_gpu(g, s, prec, want_A=True)
    issued, dense = sm.scatman_contraction_flops(h)
    h.close()
    assert rel_l2(I[sample], Ir) < TOL[prec], rel_l2(I[sample], Ir)
    assert 0 < issued <= dense


@pytest.mark.parametrize("prec", ["tc_bf16_split", "fp32"])
def test_deep_grid_nz_320(prec):
    g = Geometry(40, 36, 320, 1.0, 8.0, 40.0, 72, 64)
    rng = np.random.default_rng(5)
    shapes = [
        Shape(ELLIPSOID, a=14.0, b=12.0, c=140.0, delta=0.004, beta=0.0004, latitude=-88.0, longitude=20.0,
              rotation=10.0),
        Shape(SPHHARM, R0=15.0, lmax=4, alm=random_alm(rng, 4), delta=0.01, beta=0.001, latitude=5.0,
              longitude=-40.0, rotation=70.0, cz=60.0),
    ]
    sample = _sample(g, 500, 2)
    for s in shapes:
        Ir, _ = oracle_field(g, s, sample=sample)
        I, _ = run_gpu(g, s, prec)
        assert rel_l2(I[sample], Ir) < TOL[prec], (s.kind, rel_l2(I[sample], Ir))


def test_fp64_mode_rejects_nz_beyond_256():
    import paper_2202_03411_gb300 as sm
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_create(Geometry(16, 16, 300, 1.0, 8.0, 30.0, 8, 8), "fp64")
    assert e.value.code == -1


def test_gradient_nz_320():
    """Soft harmonics shape on a 320-slice grid: the tensor-core gradient
    against the oracle's gradient with the same upstream dL/dI."""
    import torch
    import paper_2202_03411_gb300 as sm
    g = Geometry(24, 24, 320, 1.0, 8.0, 40.0, 24, 24)
    rng = np.random.default_rng(7)
    s = Shape(SPHHARM, R0=9.0, lmax=3, alm=random_alm(rng, 3), delta=0.01, beta=0.001, latitude=20.0,
              longitude=10.0, rotation=30.0, cz=-40.0)
    h = sm.scatman_create(g, "tc_bf16_split", soft=True, soft_width=0.5)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    A = torch.empty(g.n_pix, dtype=torch.complex64, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I, A)
    w = torch.from_numpy(np.random.default_rng(8).uniform(-1, 1, g.n_pix).astype(np.float32)).cuda()
    grad = sm.scatman_backward(h, w)
    h.close()
    Ir, Ar = oracle.forward(s, g, soft=True, width=0.5)
    ref = oracle.gradient(s, g, w.cpu().double().numpy(), Ar, width=0.5)
    assert rel_l2(grad, ref) < 1e-3, rel_l2(grad, ref)
