"""Adjoint kernels vs the oracle's FP64 gradient and vs finite differences.

Loss L = sum (I - I_target)^2 with soft occupancy; the target comes from a
perturbed shape.  Tolerances on the gradient vector (relative L2): FP64 mode
1e-8, FP32 mode 1e-4, tensor-core modes 1e-3.
"""
import numpy as np
import pytest

import oracle
from workloads import ELLIPSOID, SPHERE, SPHHARM, Geometry, Shape, perturbed, random_alm, sh_grad_96

pytestmark = pytest.mark.gpu

GTOL = {"fp64": 1e-8, "fp32": 1e-4, "tc_f16_split": 1e-3, "tc_bf16_split": 1e-3}


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shape(kind, rng):
    if kind == SPHERE:
        return Shape(SPHERE, r=6.3, delta=0.03, beta=0.004, cx=0.2)
    if kind == ELLIPSOID:
        return Shape(ELLIPSOID, a=7.5, b=5.1, c=8.2, delta=0.03, beta=0.004, latitude=25, longitude=40, rotation=60)
    return Shape(SPHHARM, R0=6.5, lmax=4, alm=random_alm(rng, 4, 0.08), delta=0.03, beta=0.004, latitude=15,
                 longitude=-30, rotation=80)


def _gpu_grad(g, s, target, prec, width):
    import torch
    import paper_2202_03411_gb300 as sm
    h = sm.scatman_create(g, prec, soft=True, soft_width=width)
    f64 = prec == "fp64"
    I = torch.empty(g.n_pix, dtype=torch.float64 if f64 else torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I)
    t = torch.as_tensor(target, dtype=I.dtype, device="cuda")
    grad = sm.scatman_backward(h, 2 * (I - t))
    loss = float(((I.double() - t.double()) ** 2).sum())
    h.close()
    return loss, grad, I.double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32", "tc_f16_split", "tc_bf16_split"])
@pytest.mark.parametrize("kind", [SPHERE, ELLIPSOID, SPHHARM])
def test_gradient_vs_oracle_small(kind, prec):
    g = Geometry(20, 22, 18, 1.0, 5.0, 45.0, 24, 26)
    rng = np.random.default_rng(kind)
    s = _shape(kind, rng)
    width = 0.6
    t = perturbed(s, np.random.default_rng(100 + kind), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=width)[0]
    I, A = oracle.forward(s, g, soft=True, width=width)
    _, got, I_gpu = _gpu_grad(g, s, target, prec, width)
    # the oracle's adjoint with the upstream gradient the GPU used
    ref = oracle.gradient(s, g, 2 * (I_gpu - target), A, width=width)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < GTOL[prec], (kind, prec, err)


@pytest.mark.parametrize("prec", ["tc_f16_split", "tc_bf16_split"])
@pytest.mark.parametrize("nz", [5, 40])
def test_tensor_core_adjoint_slice_and_order_forms(nz, prec):
    """The tensor-core adjoint runs one GEMM per slice when the Jacobi-Anger
    expansion of e^{i q_z z} would need as many orders as there are slices
    (nz = 5 here), and N < nz order GEMMs otherwise (nz = 40: about 18 orders
    at this q_z range); both forms against the oracle's FP64 gradient."""
    g = Geometry(22, 20, nz, 1.0, 5.0, 45.0, 28, 24)
    rng = np.random.default_rng(40 + nz)
    s = Shape(SPHHARM, R0=min(6.5, 0.4 * nz), lmax=4, alm=random_alm(rng, 4, 0.08), delta=0.03, beta=0.004,
              latitude=15, longitude=-30, rotation=80)
    width = 0.6
    t = perturbed(s, np.random.default_rng(200 + nz), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=width)[0]
    I, A = oracle.forward(s, g, soft=True, width=width)
    _, got, I_gpu = _gpu_grad(g, s, target, prec, width)
    ref = oracle.gradient(s, g, 2 * (I_gpu - target), A, width=width)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < GTOL[prec], (nz, prec, err)



@pytest.mark.parametrize("prec", ["fp32", "tc_bf16_split"])
@pytest.mark.parametrize("lmax", [6, 10, 12])
def test_gradient_harmonic_degrees(lmax, prec):
    """The FP32 voxel gradient runs a short kernel for degree <= 6 and the full
    one (per-lane a_lm sums in up to 172 KB of shared memory) above; every
    d L / d a_lm of degrees 6, 10 and 12 against the oracle's FP64 gradient."""
    g = Geometry(24, 22, 26, 1.0, 5.0, 45.0, 30, 28)
    rng = np.random.default_rng(60 + lmax)
    s = Shape(SPHHARM, R0=7.0, lmax=lmax, alm=random_alm(rng, lmax, 0.03), delta=0.03, beta=0.004,
              latitude=-20, longitude=50, rotation=10)
    width = 0.6
    t = perturbed(s, np.random.default_rng(300 + lmax), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=width)[0]
    I, A = oracle.forward(s, g, soft=True, width=width)
    _, got, I_gpu = _gpu_grad(g, s, target, prec, width)
    ref = oracle.gradient(s, g, 2 * (I_gpu - target), A, width=width)
    assert got.shape == ref.shape == ((lmax + 1) ** 2 + 2,)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < GTOL[prec], (lmax, prec, err)


def test_gradient_fp64_deep_grid():
    """FP64 mode on 80 slices (three z per lane: the 16-per-lane form of the
    voxel gradient) against the oracle's FP64 gradient."""
    g = Geometry(20, 18, 80, 1.0, 5.0, 45.0, 22, 20)
    rng = np.random.default_rng(81)
    s = Shape(SPHHARM, R0=7.0, lmax=5, alm=random_alm(rng, 5, 0.05), delta=0.03, beta=0.004, latitude=10,
              longitude=-70, rotation=25, cz=4.0)
    width = 0.6
    t = perturbed(s, np.random.default_rng(82), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=width)[0]
    I, A = oracle.forward(s, g, soft=True, width=width)
    _, got, I_gpu = _gpu_grad(g, s, target, "fp64", width)
    ref = oracle.gradient(s, g, 2 * (I_gpu - target), A, width=width)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < GTOL["fp64"], err

def test_gradient_fp64_matches_central_differences_of_the_gpu_forward():
    """Directional derivative along a random direction, from the GPU's own forward."""
    g = Geometry(18, 18, 18, 1.0, 5.0, 45.0, 20, 20)
    rng = np.random.default_rng(3)
    s = _shape(SPHHARM, rng)
    from paper_2202_03411_gb300.autograd import params_of, shape_with
    width = 0.6
    target = oracle.forward(perturbed(s, rng, rel=0.05), g, soft=True, width=width)[0]
    L0, grad, _ = _gpu_grad(g, s, target, "fp64", width)
    p0 = params_of(s)
    v = rng.normal(size=p0.shape) * np.maximum(np.abs(p0), 0.05) * 1e-2
    h = 1e-3
    Lp = _gpu_grad(g, shape_with(s, p0 + h * v), target, "fp64", width)[0]
    Lm = _gpu_grad(g, shape_with(s, p0 - h * v), target, "fp64", width)[0]
    fd = (Lp - Lm) / (2 * h)
    assert abs(fd - grad @ v) < 1e-6 * abs(fd), (fd, grad @ v)


def test_autograd_function_and_a_fit_step():
    import torch
    import paper_2202_03411_gb300 as sm
    from paper_2202_03411_gb300.autograd import msft, params_of
    g = Geometry(20, 20, 20, 1.0, 5.0, 45.0, 24, 24)
    rng = np.random.default_rng(5)
    s = _shape(ELLIPSOID, rng)
    t = perturbed(s, rng, rel=0.05)
    h = sm.scatman_create(g, "fp32", soft=True, soft_width=0.6)
    with torch.no_grad():
        from paper_2202_03411_gb300.autograd import shape_with
        target = msft(torch.tensor(params_of(t)), h, s).clone()
    p = torch.tensor(params_of(s), requires_grad=True)
    I = msft(p, h, s)
    loss = ((I - target) ** 2).sum()
    loss.backward()
    ref_I, A = oracle.forward(s, g, soft=True, width=0.6)
    ref_grad = oracle.gradient(s, g, 2 * (ref_I - target.double().cpu().numpy()), A, width=0.6)
    err = np.linalg.norm(p.grad.numpy() - ref_grad) / np.linalg.norm(ref_grad)
    assert err < 1e-4
    # a few normalised gradient steps reduce the loss
    losses = [float(loss)]
    with torch.no_grad():
        q = p.detach().clone()
    for _ in range(3):
        q.requires_grad_(True)
        L = ((msft(q, h, s) - target) ** 2).sum()
        L.backward()
        with torch.no_grad():
            step = q.grad / q.grad.norm() * 0.01 * q.detach().abs().clamp(min=0.01)
            q = (q - step).detach()
        losses.append(float(L))
    h.close()
    assert losses[-1] < losses[0]


@pytest.fixture(scope="module")
def full_size_case():
    g, shapes = sh_grad_96(n_shapes=1)
    s = shapes[0]
    width = 0.5
    t = perturbed(s, np.random.default_rng(7), rel=0.02)
    target = oracle.forward(t, g, soft=True, width=width)[0]
    I, A = oracle.forward(s, g, soft=True, width=width)
    return g, s, width, target, A


@pytest.mark.parametrize("prec", ["fp32", "tc_bf16_split"])
def test_gradient_full_size_harmonics_96(prec, full_size_case):
    """The 96^3 / 256^2 l<=6 harmonics workload against the oracle's gradient."""
    g, s, width, target, A = full_size_case
    _, got, I_gpu = _gpu_grad(g, s, target, prec, width)
    ref = oracle.gradient(s, g, 2 * (I_gpu - target), A, width=width)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < GTOL[prec], err


@pytest.mark.parametrize("ny", [72, 128])
def test_gradient_tensor_core_adjoint_stage_counts(ny):
    """The tensor-core adjoint at y extents whose operand stages leave four
    (ny = 72) and three (ny = 128) pipeline stages, so both generator team
    layouts run, with enough pixels for many chunks per team."""
    from workloads import ELLIPSOID
    g = Geometry(20, ny, 16, 1.0, 5.0, 45.0, 48, 40)
    s = Shape(ELLIPSOID, a=6.0, b=0.4 * ny, c=5.5, delta=0.03, beta=0.004, latitude=10, longitude=80, rotation=30)
    width = 0.6
    t = perturbed(s, np.random.default_rng(9), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=width)[0]
    _, A = oracle.forward(s, g, soft=True, width=width)
    _, got, I_gpu = _gpu_grad(g, s, target, "tc_bf16_split", width)
    ref = oracle.gradient(s, g, 2 * (I_gpu - target), A, width=width)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    assert err < GTOL["tc_bf16_split"], (ny, err)
