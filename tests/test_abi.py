"""The C ABI library loads and exports every symbol include/scatman.h declares;
host-side argument checks answer without touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_2202_03411_gb300 import _lib, build
from paper_2202_03411_gb300.api import ScatmanError, make_config
from workloads import Geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def header_symbols():
    text = open(os.path.join(ROOT, "include", "scatman.h")).read()
    return re.findall(r"SCATMAN_API[^;(]*?\b(scatman_\w+)\s*\(", text)


def test_every_declared_symbol_is_exported(lib):
    names = header_symbols()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
        assert n in _lib.SIGNATURES, n
    assert set(_lib.SIGNATURES) == set(names)


def test_version(lib):
    assert b"sm_103a" in lib.scatman_version()


def _create(lib, g, prec, **kw):
    cfg, keep = make_config(g, prec, **kw)
    out = ctypes.c_void_p()
    code = lib.scatman_create(ctypes.byref(cfg), None, ctypes.byref(out))
    return code, out.value, lib.scatman_last_error(None).decode()


@pytest.mark.parametrize("g,prec,kw,frag", [
    (Geometry(0, 8, 8, 1.0, 8.0, 30.0, 8, 8), "fp32", {}, "grid"),
    (Geometry(8, 8, 600, 1.0, 8.0, 30.0, 8, 8), "fp32", {}, "nz"),
    (Geometry(8, 8, 300, 1.0, 8.0, 30.0, 8, 8), "fp64", {}, "nz"),
    (Geometry(8, 8, 8, 0.0, 8.0, 30.0, 8, 8), "fp32", {}, "positive"),
    (Geometry(8, 8, 8, 1.0, 8.0, 95.0, 8, 8), "fp32", {}, "theta"),
    (Geometry(8, 8, 8, 1.0, 8.0, 30.0, 0, 8), "fp32", {}, "detector"),
    (Geometry(8, 8, 8, 1.0, 8.0, 30.0, 8, 8), 17, {}, "precision"),
    (Geometry(8, 8, 8, 1.0, 8.0, 30.0, 8, 8), "fp32", {"soft": True, "soft_width": 0.0}, "soft"),
])
def test_create_rejects_bad_arguments(lib, g, prec, kw, frag):
    code, ptr, msg = _create(lib, g, prec, **kw)
    assert code == _lib.SCATMAN_ERR_ARG and not ptr
    assert frag in msg


def test_null_arguments(lib):
    assert lib.scatman_create(None, None, None) == _lib.SCATMAN_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.scatman_create(None, None, ctypes.byref(out)) == _lib.SCATMAN_ERR_ARG
    assert lib.scatman_voxelise(None, None) == _lib.SCATMAN_ERR_ARG
    assert lib.scatman_forward(None, None, None) == _lib.SCATMAN_ERR_ARG
    assert lib.scatman_param_count(None) == 0
    lib.scatman_destroy(None)


def test_no_device_is_reported(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    code, ptr, msg = _create(lib, Geometry(8, 8, 8, 1.0, 8.0, 30.0, 8, 8), "fp32")
    assert code == _lib.SCATMAN_ERR_UNSUPPORTED and not ptr
    assert msg


def test_footprint_is_a_host_calculation(lib):
    from paper_2202_03411_gb300.serving import footprint_bytes
    small = Geometry(48, 48, 48, 1.0, 10.0, 45.0, 128, 128)
    big = Geometry(128, 128, 128, 1.0, 10.0, 45.0, 512, 512)
    for prec in ("fp64", "fp32", "tc_bf16_split"):
        assert 0 < footprint_bytes(small, prec) < footprint_bytes(big, prec)
    # tensor-core handles hold the adjoint's y-phase operand tiles:
    # 4 bytes per pixel and y row of each of the two real parts
    assert footprint_bytes(big, "tc_bf16_split") > 512 * 512 * 2 * 128 * 4
    # the largest serving request fits many times into a 120 GB budget
    assert footprint_bytes(big, "tc_bf16_split") < (120 << 30) // 100


def test_footprint_counts_the_uniform_q_buffers(lib):
    """The uniform-q detector's y-contracted operand and q_z table are part of
    the estimate: the tensor-core planes grow with the detector rows and with
    the padded z extent, the FP32 slices with rows x nx x nz."""
    from paper_2202_03411_gb300.serving import footprint_bytes
    from workloads import DETECTOR_UNIFORM_Q
    g = Geometry(56, 56, 56, 1.0, 1.0, 30.0, 2048, 2048, DETECTOR_UNIFORM_Q)
    flat = Geometry(56, 56, 56, 1.0, 1.0, 30.0, 2048, 2048)
    # tensor cores: 2048 rows x 3 planes x 64 padded z x 64 padded x x 2 bytes = 48 MiB of planes,
    # plus an 8-byte q_z per pixel (32 MiB), on top of the flat detector's buffers
    extra = footprint_bytes(g, "tc_bf16_split") - footprint_bytes(flat, "tc_bf16_split")
    assert extra >= (48 << 20) + (32 << 20) - (4 << 20)
    # FP32: q (96 MiB), 2048 rows x 56 x 56 complex slices (49 MiB) and the q_z table
    # (32 MiB); no split partial fields (the flat detector's 2 GiB)
    n = 2048 * 2048
    assert footprint_bytes(g, "fp32") >= 24 * n + 2048 * 56 * 56 * 8 + 8 * n
    assert footprint_bytes(g, "fp32") < footprint_bytes(flat, "fp32")
    g_small = Geometry(56, 56, 56, 1.0, 1.0, 30.0, 256, 256, DETECTOR_UNIFORM_Q)
    assert 0 < footprint_bytes(g_small, "fp32") < footprint_bytes(g, "fp32")


def test_noalloc_host_checks(lib):
    """Checks that answer before any device is touched (no GPU needed)."""
    from paper_2202_03411_gb300.api import make_shape
    from workloads import SPHERE, Shape
    st, keep = make_shape(Shape(SPHERE, r=4.0, delta=0.01, beta=0.001))
    fake = ctypes.c_void_p(16)          # never dereferenced: the calls fail their argument checks first
    for g, frag in ((Geometry(16, 16, 16, 1.0, 8.0, 30.0, 8, 8, 1), "flat detector"),
                    (Geometry(16, 5000, 16, 1.0, 8.0, 30.0, 8, 8), "4096"),
                    (Geometry(16, 16, 16, 1.0, 8.0, 30.0, 8, 8, 7), "detector")):
        cfg, _ = make_config(g, "fp32")
        assert lib.scatman_forward_noalloc(ctypes.byref(cfg), ctypes.byref(st), None, fake, None) == \
            _lib.SCATMAN_ERR_ARG
        assert frag in lib.scatman_last_error(None).decode()
    cfg, _ = make_config(Geometry(16, 16, 16, 1.0, 8.0, 30.0, 8, 8), "tc_bf16_split")
    assert lib.scatman_forward_noalloc(ctypes.byref(cfg), ctypes.byref(st), None, fake, None) == \
        _lib.SCATMAN_ERR_ARG


def test_failure_hooks_reject_null(lib):
    assert lib.scatman_set_wait_limit(None, 1.0) == _lib.SCATMAN_ERR_ARG
    assert lib.scatman_debug_stall(None, 1) == _lib.SCATMAN_ERR_ARG
    assert lib.scatman_server_cancel(None, 1) == _lib.SCATMAN_ERR_ARG
    lib.scatman_debug_fail_allocation(-1)


class _FakeTensor:
    def __init__(self, is_cuda=True, dtype="torch.float32", contiguous=True, n=100):
        self.is_cuda, self.dtype, self._c, self._n = is_cuda, dtype, contiguous, n

    def is_contiguous(self):
        return self._c

    def numel(self):
        return self._n

    def data_ptr(self):
        return 4096


def test_binding_checks_output_buffers_before_any_kernel():
    from paper_2202_03411_gb300.api import _device_ptr
    assert _device_ptr(_FakeTensor(), ["float32"], 100, "I").value == 4096
    assert _device_ptr(None, ["float32"], 100, "A").value is None
    for bad in (_FakeTensor(is_cuda=False), _FakeTensor(dtype="torch.float64"), _FakeTensor(contiguous=False),
                _FakeTensor(n=99)):
        with pytest.raises(ValueError):
            _device_ptr(bad, ["float32"], 100, "I")
