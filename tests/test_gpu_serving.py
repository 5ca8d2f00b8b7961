"""Native fit server: continuous admission under a memory budget, results
independent of the request mix."""
import numpy as np
import pytest

import oracle
from workloads import ELLIPSOID, SPHERE, SPHHARM, Geometry, Request, Shape, perturbed, random_alm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mix(n, seed=0):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        nv = int(rng.choice([24, 32, 40]))
        det = int(rng.choice([32, 48, 64]))
        g = Geometry(nv, nv, nv, 1.0, 6.0, 45.0, det, det)
        kind = i % 3
        d = rng.uniform(1e-3, 3e-2)
        if kind == SPHERE:
            s = Shape(SPHERE, r=rng.uniform(0.25, 0.4) * nv, delta=d, beta=d / 10)
        elif kind == ELLIPSOID:
            a = rng.uniform(0.2, 0.4, 3) * nv
            s = Shape(ELLIPSOID, a=a[0], b=a[1], c=a[2], delta=d, beta=d / 10, latitude=rng.uniform(-90, 90),
                      longitude=rng.uniform(-180, 180), rotation=rng.uniform(0, 360))
        else:
            s = Shape(SPHHARM, R0=0.3 * nv, lmax=4, alm=random_alm(rng, 4), delta=d, beta=d / 10,
                      latitude=rng.uniform(-90, 90), longitude=rng.uniform(-180, 180), rotation=rng.uniform(0, 360))
        reqs.append(Request(i, 0.0, g, s, perturbed(s, rng)))
    return reqs


def _targets(reqs, prec):
    """Fit targets: the intensity of each request's perturbed shape (via the library)."""
    import torch
    import paper_2202_03411_gb300 as sm
    out = []
    for r in reqs:
        h = sm.scatman_create(r.geometry, prec, soft=True, soft_width=0.5)
        I = torch.empty(r.geometry.n_pix, dtype=torch.float64 if prec == "fp64" else torch.float32, device="cuda")
        sm.scatman_voxelise(h, r.target)
        sm.scatman_forward(h, I)
        sm.scatman_sync(h)
        out.append(I.float().cpu().numpy())
        h.close()
    return out


@pytest.mark.parametrize("prec", ["tc_bf16_split", "fp32"])
def test_results_identical_alone_and_in_the_mix(prec):
    from paper_2202_03411_gb300.serving import Server
    reqs = _mix(12)
    targets = _targets(reqs, prec)
    alone = []
    srv = Server(budget_bytes=64 << 30, slots=1, precision=prec)
    for r, t in zip(reqs, targets):
        tk, res = srv.submit(r.geometry, r.shape, t, want_I=True)
        st, _ = srv.wait(tk)
        assert st == 0
        alone.append(res)
    srv.close()
    srv = Server(budget_bytes=64 << 30, slots=4, precision=prec)
    tickets = [srv.submit(r.geometry, r.shape, t, want_I=True) for r, t in zip(reqs, targets)]
    mix = []
    for tk, res in tickets:
        st, _ = srv.wait(tk)
        assert st == 0
        mix.append(res)
    stats = srv.stats()
    srv.close()
    assert stats["inflight_peak"] > 1          # requests really overlapped
    assert stats["completed"] == len(reqs)
    for a, b in zip(alone, mix):
        np.testing.assert_array_equal(a["I"], b["I"])
        np.testing.assert_array_equal(a["grad"], b["grad"])
        assert a["loss"][0] == b["loss"][0]


def test_admission_respects_the_budget():
    from paper_2202_03411_gb300.serving import Server, footprint_bytes
    reqs = _mix(6, seed=1)
    for r in reqs:
        r.geometry = Geometry(40, 40, 40, 1.0, 6.0, 45.0, 64, 64)
    targets = _targets(reqs, "tc_bf16_split")
    one = footprint_bytes(reqs[0].geometry, "tc_bf16_split")
    budget = int(one * 1.5) + (16 << 20)         # room for one request at a time
    srv = Server(budget_bytes=budget, slots=4, precision="tc_bf16_split")
    tickets = [srv.submit(r.geometry, r.shape, t) for r, t in zip(reqs, targets)]
    for tk, _ in tickets:
        st, _ = srv.wait(tk)
        assert st == 0
    stats = srv.stats()
    assert stats["inflight_peak"] == 1
    assert stats["bytes_reserved_peak"] <= budget
    # a request that alone exceeds the budget is refused at submission
    big = Geometry(128, 128, 128, 1.0, 10.0, 60.0, 512, 512)
    import paper_2202_03411_gb300 as sm
    with pytest.raises(sm.ScatmanError) as e:
        srv.submit(big, reqs[0].shape, np.zeros(big.n_pix, np.float32))
    assert e.value.code == -5
    srv.close()


def test_served_gradient_matches_oracle():
    from paper_2202_03411_gb300.serving import Server
    g = Geometry(20, 20, 20, 1.0, 5.0, 45.0, 24, 24)
    s = Shape(ELLIPSOID, a=7.5, b=5.1, c=8.2, delta=0.03, beta=0.004, latitude=25, longitude=40, rotation=60)
    t = perturbed(s, np.random.default_rng(3), rel=0.05)
    target = oracle.forward(t, g, soft=True, width=0.5)[0].astype(np.float32)
    srv = Server(budget_bytes=8 << 30, slots=2, precision="fp64")
    tk, res = srv.submit(g, s, target, want_I=True)
    st, lat = srv.wait(tk)
    srv.close()
    assert st == 0 and lat > 0
    I, A = oracle.forward(s, g, soft=True, width=0.5)
    ref = oracle.gradient(s, g, 2 * (res["I"].astype(np.float64) - target.astype(np.float64)), A, width=0.5)
    assert np.linalg.norm(res["grad"] - ref) / np.linalg.norm(ref) < 1e-6
    assert abs(res["loss"][0] - ((I - target) ** 2).sum()) < 1e-6 * res["loss"][0]
