"""The forward entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc -- a host application that
has reserved nearly all device memory for its own pool, or a latency-critical
loop that must not take an allocation's device-wide synchronisation.  This
file is collected last so that a run stopping at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from workloads import ELLIPSOID, SPHHARM, Geometry, Shape, random_alm

pytestmark = pytest.mark.gpu


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


def _handle_path(sm, g, s):
    import torch
    h = sm.scatman_create(g, "fp32")
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I)
    sm.scatman_sync(h)
    h.close()
    return I.cpu().double().numpy()


def test_noalloc_matches_handle_path_on_two_calls_in_a_row(sm):
    import torch
    g = Geometry(40, 36, 44, 1.0, 8.0, 45.0, 96, 80)
    rng = np.random.default_rng(0)
    shapes = [
        Shape(ELLIPSOID, a=14.0, b=9.5, c=16.0, delta=0.02, beta=0.004, latitude=25, longitude=40, rotation=60),
        Shape(SPHHARM, R0=12.0, lmax=6, alm=random_alm(rng, 6), delta=0.01, beta=0.001, latitude=-10,
              longitude=80, rotation=200),
    ]
    for s in shapes:           # two calls in a row share (and overwrite) the scratch array
        I = torch.full((g.n_pix,), float("nan"), dtype=torch.float32, device="cuda")
        sm.scatman_forward_noalloc(g, s, I)
        torch.cuda.synchronize()
        got = I.cpu().double().numpy()
        ref = _handle_path(sm, g, s)
        assert np.all(np.isfinite(got))
        assert _rel_l2(got, ref) < 1e-5          # the FP32 tolerance of the parity tests


def test_noalloc_rejects_problems_beyond_its_scratch(sm):
    import torch
    g = Geometry(128, 128, 128, 1.0, 10.0, 60.0, 512, 512)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_forward_noalloc(g, Shape(ELLIPSOID, a=30, b=30, c=30, delta=0.01, beta=0.001), I)
    assert e.value.code == -1 and "scratch" in str(e.value)
