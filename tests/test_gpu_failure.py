"""Failure paths on the GPU, reached without faulting it.

* Bounded waits: with the handle's test flag set, the tensor-core kernels' MMA
  warps first wait on a barrier that nothing arrives at (a flag nothing sets);
  with the wait limit shortened to 10 ms that wait runs out, the kernel takes
  its abort path (the other warps stop at their next wait, the TMA copies and
  MMAs in flight are drained with the full limit, tensor memory is freed) and
  the call reports ERR_TIMEOUT.  The same handle, with the flag cleared and
  the limit restored, computes the right answer again.
* Allocation failure injected on the host (scatman_debug_fail_allocation):
  scatman_create returns ERR_OOM at every point of its allocation sequence and
  releases what it had; the server reports ERR_OOM for the request whose
  handle could not be created and serves the next ones.
* Cancellation of a queued server request.
"""
import time

import numpy as np
import pytest

import oracle
from gpu_helpers import oracle_field, rel_l2
from workloads import SPHERE, SPHHARM, Geometry, Shape, random_alm, sh_128, sh_grad_96

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__
    __graft_entry__.build()
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_forward_wait_timeout_is_reported_and_the_handle_recovers():
    import torch
    import paper_2202_03411_gb300 as sm
    g, shapes = sh_128(n_shapes=1)
    s = shapes[0]
    h = sm.scatman_create(g, "tc_bf16_split")
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_set_wait_limit(h, 0.01)
    sm.scatman_debug_stall(h, True)
    sm.scatman_forward(h, I)
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_sync(h)
    assert e.value.code == -4                       # ERR_TIMEOUT
    sm.scatman_debug_stall(h, False)
    sm.scatman_set_wait_limit(h, 0.0)               # the default limit again
    sm.scatman_forward(h, I)
    sm.scatman_sync(h)
    got = I.cpu().double().numpy()
    h2 = sm.scatman_create(g, "tc_bf16_split")      # a fresh handle gives the same pattern, bit for bit
    I2 = torch.empty_like(I)
    sm.scatman_voxelise(h2, s)
    sm.scatman_forward(h2, I2)
    sm.scatman_sync(h2)
    assert np.array_equal(got, I2.cpu().double().numpy())
    sample = np.random.default_rng(3).choice(g.n_pix, size=256, replace=False)
    Ir, _ = oracle_field(g, s, sample=sample)
    assert rel_l2(got[sample], Ir) < 1e-3
    h.close()
    h2.close()


def test_backward_wait_timeout_is_reported_and_the_handle_recovers():
    import torch
    import paper_2202_03411_gb300 as sm
    g, shapes = sh_grad_96(n_shapes=1)
    s = shapes[0]
    h = sm.scatman_create(g, "tc_bf16_split", soft=True, soft_width=0.5)
    I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
    sm.scatman_voxelise(h, s)
    sm.scatman_forward(h, I)
    sm.scatman_sync(h)
    w = torch.ones_like(I)
    ref = sm.scatman_backward(h, w)
    sm.scatman_set_wait_limit(h, 0.01)
    sm.scatman_debug_stall(h, True)
    with pytest.raises(sm.ScatmanError) as e:
        sm.scatman_backward(h, w)
    assert e.value.code == -4
    sm.scatman_debug_stall(h, False)
    sm.scatman_set_wait_limit(h, -1.0)
    again = sm.scatman_backward(h, w)
    assert np.array_equal(again, ref)               # fixed reduction orders: bit for bit
    h.close()


def test_wait_limit_argument_checks():
    import paper_2202_03411_gb300 as sm
    g = Geometry(16, 16, 16, 1.0, 8.0, 30.0, 8, 8)
    h = sm.scatman_create(g, "tc_f16_split")
    with pytest.raises(sm.ScatmanError):
        sm.scatman_set_wait_limit(h, float("nan"))
    sm.scatman_set_wait_limit(h, 5.0)               # longer than the maximum: the default 2 s
    h.close()


def test_create_reports_oom_at_every_allocation_and_cleans_up():
    import torch
    import paper_2202_03411_gb300 as sm
    g = Geometry(24, 20, 22, 1.0, 8.0, 40.0, 40, 36)
    s = Shape(SPHERE, r=7.0, delta=0.02, beta=0.003)
    for prec in ("fp32", "tc_bf16_split"):
        free0 = torch.cuda.mem_get_info()[0]
        k = 0
        while True:
            sm.scatman_debug_fail_allocation(k)
            try:
                h = sm.scatman_create(g, prec)
            except sm.ScatmanError as e:
                assert e.code == -2, e                  # ERR_OOM
                k += 1
                assert k < 64
                continue
            finally:
                sm.scatman_debug_fail_allocation(-1)
            break
        # the k-th allocation was the first that create did not make: k > 0 allocations happened
        assert k >= 4
        I = torch.empty(g.n_pix, dtype=torch.float32, device="cuda")
        sm.scatman_voxelise(h, s)
        sm.scatman_forward(h, I)
        sm.scatman_sync(h)
        Ir, _ = oracle_field(g, s)
        assert rel_l2(I.cpu().double().numpy(), Ir) < 1e-3
        h.close()
        torch.cuda.synchronize()
        # every failed create released its buffers (within allocator granularity)
        assert torch.cuda.mem_get_info()[0] >= free0 - (64 << 20)


def _fit_requests(n, seed):
    rng = np.random.default_rng(seed)
    g = Geometry(32, 32, 32, 1.0, 8.0, 40.0, 48, 48)
    out = []
    for _ in range(n):
        s = Shape(SPHHARM, R0=9.0, lmax=3, alm=random_alm(rng, 3), delta=0.02, beta=0.002,
                  latitude=float(rng.uniform(-90, 90)), longitude=float(rng.uniform(-180, 180)))
        out.append((g, s))
    return out


def test_server_reports_oom_for_one_request_and_serves_the_rest():
    from paper_2202_03411_gb300 import scatman_debug_fail_allocation
    from paper_2202_03411_gb300.serving import Server
    reqs = _fit_requests(3, 1)
    target = np.zeros(reqs[0][0].n_pix, dtype=np.float32)
    srv = Server(1 << 30, slots=1, precision="tc_bf16_split")
    try:
        scatman_debug_fail_allocation(0)            # the first handle the slot creates fails
        t0, _ = srv.submit(*reqs[0], target)
        st0, _ = srv.wait(t0, timeout_s=60.0)
        scatman_debug_fail_allocation(-1)
        assert st0 == -2                            # ERR_OOM
        res = []
        for g, s in reqs[1:]:
            t, r = srv.submit(g, s, target)
            res.append((t, r))
        for t, r in res:
            st, _ = srv.wait(t, timeout_s=60.0)
            assert st == 0 and np.all(np.isfinite(r["grad"]))
        stats = srv.stats()
        assert stats["failed"] == 1 and stats["completed"] == 2
        assert stats["bytes_reserved"] > 0          # the failed handle's bytes were given back, the good one kept
    finally:
        scatman_debug_fail_allocation(-1)
        srv.close()


def test_server_cancels_a_queued_request():
    from paper_2202_03411_gb300.serving import Server
    big = Geometry(96, 96, 96, 1.0, 10.0, 45.0, 256, 256)
    rng = np.random.default_rng(4)
    s_big = Shape(SPHHARM, R0=30.0, lmax=4, alm=random_alm(rng, 4), delta=0.01, beta=0.001)
    small = _fit_requests(3, 2)
    srv = Server(8 << 30, slots=1, precision="tc_bf16_split")
    try:
        t_big, _ = srv.submit(big, s_big, np.zeros(big.n_pix, dtype=np.float32))   # occupies the only slot
        deadline = time.time() + 30.0
        while srv.stats()["inflight"] < 1 and time.time() < deadline:
            time.sleep(1e-3)
        assert srv.stats()["inflight"] == 1
        tickets = [srv.submit(g, s, np.zeros(g.n_pix, dtype=np.float32))[0] for g, s in small]
        assert not srv.cancel(t_big)                # admitted: it runs to completion
        assert srv.cancel(tickets[-1])              # still queued behind the big request
        for t in [t_big] + tickets[:-1]:
            st, _ = srv.wait(t, timeout_s=120.0)
            assert st == 0
        st, _ = srv.wait(tickets[-1], timeout_s=5.0)
        assert st == -8                             # ERR_CANCELLED
        assert srv.stats()["cancelled"] == 1 and srv.stats()["completed"] == 3
        with pytest.raises(Exception):
            srv.cancel(tickets[-1])                 # collected already: unknown ticket
    finally:
        srv.close()
