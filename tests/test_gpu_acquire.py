"""End-to-end acquisition with host memory: the pipelined batch equals the
per-pattern call, pattern by pattern and bit for bit."""
import numpy as np
import pytest

from workloads import ELLIPSOID, SPHERE, SPHHARM, Geometry, Shape, random_alm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _shapes(rng, n):
    out = []
    for k in range(n):
        if k % 3 == 0:
            out.append(Shape(SPHERE, r=rng.uniform(6, 10), delta=0.01, beta=0.001))
        elif k % 3 == 1:
            out.append(Shape(ELLIPSOID, a=rng.uniform(6, 11), b=rng.uniform(5, 9), c=rng.uniform(7, 12), delta=0.02,
                             beta=0.002, latitude=rng.uniform(-90, 90), longitude=rng.uniform(-180, 180),
                             rotation=rng.uniform(0, 360)))
        else:
            out.append(Shape(SPHHARM, R0=9.0, lmax=4, alm=random_alm(rng, 4), delta=0.015, beta=0.001,
                             latitude=rng.uniform(-90, 90), longitude=rng.uniform(-180, 180)))
    return out


@pytest.mark.parametrize("prec", ["tc_bf16_split", "fp32", "fp64"])
def test_acquire_batch_equals_acquire(prec):
    import torch
    import paper_2202_03411_gb300 as sm
    g = Geometry(32, 30, 28, 1.0, 8.0, 45.0, 70, 66)
    shapes = _shapes(np.random.default_rng(5), 5)
    h = sm.scatman_create(g, prec)
    dt = np.float64 if prec == "fp64" else np.float32
    one = [np.empty(g.n_pix, dtype=dt) for _ in shapes]
    for s, out in zip(shapes, one):
        sm.scatman_acquire(h, s, out)
    pinned = torch.empty((len(shapes), g.n_pix), dtype=torch.float64 if prec == "fp64" else torch.float32,
                         pin_memory=True)
    sm.scatman_acquire_batch(h, shapes, pinned)
    pageable = [np.zeros(g.n_pix, dtype=dt) for _ in shapes]
    sm.scatman_acquire_batch(h, shapes, pageable)
    sm.scatman_acquire_batch(h, [], [])                       # n = 0: nothing happens
    h.close()
    for i in range(len(shapes)):
        assert np.array_equal(pinned[i].numpy(), one[i]), i
        assert np.array_equal(pageable[i], one[i]), i
