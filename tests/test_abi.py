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
    (Geometry(8, 8, 300, 1.0, 8.0, 30.0, 8, 8), "fp32", {}, "nz"),
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
