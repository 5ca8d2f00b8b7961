"""The forward entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc -- a host application that
has reserved nearly all device memory for its own pool, or a latency-critical
loop that must not take an allocation's device-wide synchronisation.  Its
working memory is one fixed array inside the library that every call reuses,
so these tests run calls back to back with different sizes and check each
against the handle path and against the FP64 oracle.  This file is collected
last so that a run stopping at the first failure has already run every other
test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

import oracle
from workloads import ELLIPSOID, SPHERE, SPHHARM, Geometry, Shape, random_alm

pytestmark = pytest.mark.gpu

TOL_FP32 = 1e-5          # the FP32 tolerance of the parity tests (relative L2 of I and of A)


@pytest.fixture(scope="module")
def sm():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2202_03411_gb300 as sm
    return sm


def _rel_l2(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def _handle_path(sm, g, s, q_list=None):
    import torch
    h = sm.scatman_create(g, "fp32", q_list=q_list)
    n = sm.scatman_n_pix(h)
    I = torch.empty(n, dtype=torch.float32, device="cuda")
    A = torch.empty(n, dtype=torch.complex64, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I, A)
    sm.scatman_sync(h)
    h.close()
    return I.cpu().double().numpy(), A.cpu().numpy().astype(np.complex128)


def _noalloc(sm, g, s, with_A, q_list=None):
    import torch
    n = q_list.shape[0] if q_list is not None else g.n_pix
    I = torch.full((n,), float("nan"), dtype=torch.float32, device="cuda")
    A = torch.full((n,), complex("nan"), dtype=torch.complex64, device="cuda") if with_A else None
    sm.scatman_forward_noalloc(g, s, I, A, q_list=q_list)
    torch.cuda.synchronize()
    got_I = I.cpu().double().numpy()
    got_A = A.cpu().numpy().astype(np.complex128) if with_A else None
    assert np.all(np.isfinite(got_I))
    return got_I, got_A


def _oracle(g, s, q=None):
    if q is None:
        q = oracle.detector_q(g)
    chi, _ = oracle.voxelise(s, g)
    A = oracle.msft(oracle.slices(chi, g, s.delta, s.beta), q, g.voxel)
    return np.abs(A) ** 2, A


def test_noalloc_matches_handle_path_on_two_calls_in_a_row(sm):
    g = Geometry(40, 36, 44, 1.0, 8.0, 45.0, 96, 80)
    rng = np.random.default_rng(0)
    shapes = [
        Shape(ELLIPSOID, a=14.0, b=9.5, c=16.0, delta=0.02, beta=0.004, latitude=25, longitude=40, rotation=60),
        Shape(SPHHARM, R0=12.0, lmax=6, alm=random_alm(rng, 6), delta=0.01, beta=0.001, latitude=-10,
              longitude=80, rotation=200),
    ]
    for s in shapes:           # two calls in a row share (and overwrite) the scratch array
        got, _ = _noalloc(sm, g, s, with_A=False)
        ref, _ = _handle_path(sm, g, s)
        assert _rel_l2(got, ref) < TOL_FP32


def test_noalloc_larger_then_smaller_problem_with_field(sm):
    """A large call leaves its data in the shared array; the smaller call after
    it, with another grid and detector and a different scratch layout, must
    not read any of it.  The field A is compared as well as I."""
    rng = np.random.default_rng(1)
    big = (Geometry(64, 60, 56, 1.0, 9.0, 50.0, 112, 100),
           Shape(SPHHARM, R0=20.0, lmax=5, alm=random_alm(rng, 5), delta=0.015, beta=0.002, latitude=40,
                 longitude=-30, rotation=10))
    small = (Geometry(24, 30, 20, 1.0, 7.0, 35.0, 45, 38),
             Shape(ELLIPSOID, a=8.0, b=11.0, c=6.0, delta=0.02, beta=0.005, latitude=-60, longitude=15,
                   rotation=80))
    for g, s in (big, small, big):
        got_I, got_A = _noalloc(sm, g, s, with_A=True)
        ref_I, ref_A = _handle_path(sm, g, s)
        assert _rel_l2(got_I, ref_I) < TOL_FP32
        assert _rel_l2(got_A, ref_A) < TOL_FP32


def test_noalloc_against_the_oracle(sm):
    g = Geometry(32, 28, 30, 1.0, 8.0, 40.0, 60, 52)
    rng = np.random.default_rng(2)
    s = Shape(SPHHARM, R0=10.0, lmax=4, alm=random_alm(rng, 4), delta=0.02, beta=0.003, latitude=12,
              longitude=100, rotation=45, cx=0.7)
    got_I, got_A = _noalloc(sm, g, s, with_A=True)
    ref_I, ref_A = _oracle(g, s)
    assert _rel_l2(got_I, ref_I) < TOL_FP32
    assert _rel_l2(got_A, ref_A) < TOL_FP32


def test_noalloc_q_list_against_the_oracle(sm):
    g = Geometry(20, 24, 18, 1.0, 6.0, 40.0, 1, 1)
    rng = np.random.default_rng(3)
    q = rng.uniform(-0.8, 0.8, size=(333, 3))           # a ragged number of arbitrary q points
    s = Shape(SPHERE, r=7.5, delta=0.03, beta=0.006, cx=-0.4, cy=0.9)
    got_I, got_A = _noalloc(sm, g, s, with_A=True, q_list=q)
    ref_I, ref_A = _oracle(g, s, q=q)
    assert _rel_l2(got_I, ref_I) < TOL_FP32
    assert _rel_l2(got_A, ref_A) < TOL_FP32
    hand_I, _ = _handle_path(sm, g, s, q_list=q)
    assert _rel_l2(got_I, hand_I) < TOL_FP32


def test_noalloc_rejects_what_it_does_not_serve(sm):
    import torch
    s = Shape(ELLIPSOID, a=30, b=30, c=30, delta=0.01, beta=0.001)
    g = Geometry(128, 128, 128, 1.0, 10.0, 60.0, 512, 512)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_forward_noalloc(g, s, I)
    assert e.value.code == -1 and "scratch" in str(e.value)
    gu = Geometry(16, 16, 16, 1.0, 8.0, 30.0, 32, 32, 1)          # the uniform-q detector
    Iu = torch.empty(gu.n_pix, dtype=torch.float32, device="cuda")
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_forward_noalloc(gu, Shape(SPHERE, r=5.0, delta=0.01, beta=0.001), Iu)
    assert e.value.code == -1 and "flat detector" in str(e.value)
    gl = Geometry(16, 5000, 16, 1.0, 8.0, 30.0, 4, 4)              # ny beyond the handle path's limit
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_forward_noalloc(gl, Shape(SPHERE, r=5.0, delta=0.01, beta=0.001), Iu)
    assert e.value.code == -1
    short = torch.empty(10, dtype=torch.float32, device="cuda")    # checked before any kernel runs
    with pytest.raises(ValueError):
        sm.scatman_forward_noalloc(Geometry(16, 16, 16, 1.0, 8.0, 30.0, 32, 32), Shape(SPHERE, r=5.0), short)
