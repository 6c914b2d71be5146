"""The C ABI library loads and exports every symbol include/ddflb.h declares,
and its host-side validation behaves (no GPU needed: nothing here launches)."""
import ctypes
import os
import re

import pytest

from paper_1908_06742_gb300 import build as B
from paper_1908_06742_gb300 import ddflb as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    txt = open(os.path.join(ROOT, "include", "ddflb.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(ddflb_\w+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load()


def test_every_declared_symbol_is_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    # the binding wraps exactly the declared set
    assert set(D.SIGNATURES) == set(names)


def test_version(lib):
    assert b"sm_103a" in lib.ddflb_version()


def good():
    return D.Config(nx=64, ny=32, bc="cavity", u_lid=0.1)


def test_workspace_bytes_layout(lib):
    n32 = D.workspace_bytes(good())
    c16 = good(); c16.storage = "fp16"
    n16 = D.workspace_bytes(c16)
    # two ping-pong buffers of 18 planes [32][64] (pitch 64): 2*18*2048*4 B dominate
    assert n32 >= 2 * 18 * 64 * 32 * 4
    assert n16 < n32
    cio = good(); cio.host_io = True
    assert D.workspace_bytes(cio) >= n32 + 10 * 64 * 32 * 4


@pytest.mark.parametrize("field,value,msg", [
    ("nx", 1, "too small"),
    ("bc", 7, "bc"),
    ("storage", 5, "storage"),
    ("beta2", 1.0, "beta1 != beta2"),
    ("cs2", 0.0, "cs2"),
    ("check_every", -1, "check_every"),
    ("scale_f", 3.0, "power of two"),
])
def test_invalid_parameters(lib, field, value, msg):
    p = good().to_c()
    setattr(p, field, value)
    assert lib.ddflb_workspace_bytes(ctypes.byref(p)) == 0
    assert msg in lib.ddflb_last_error().decode()


def test_conserved_rates_must_be_zero(lib):
    c = good(); c.omega_f = (0, 0.5, 0, 1.2, 1.5, 1.5, 1, 1, 1)
    p = c.to_c()
    assert lib.ddflb_workspace_bytes(ctypes.byref(p)) == 0
    assert "conserved" in lib.ddflb_last_error().decode()
    c = good(); c.omega_g = (2.5,) + (1.0,) * 8
    p = c.to_c()
    assert lib.ddflb_workspace_bytes(ctypes.byref(p)) == 0


def test_create_rejects_bad_workspace(lib):
    p = good().to_c()
    h = ctypes.c_void_p()
    assert lib.ddflb_create(ctypes.byref(p), None, 1 << 30, None, ctypes.byref(h)) == D.EINVAL
    assert lib.ddflb_create(ctypes.byref(p), 4096 + 8, 1 << 30, None, ctypes.byref(h)) == D.EINVAL
    assert "aligned" in lib.ddflb_last_error().decode()
    assert lib.ddflb_create(ctypes.byref(p), 4096, 100, None, ctypes.byref(h)) == D.ENOMEM
    assert lib.ddflb_step(None, 1) == D.EINVAL


def test_binding_fails_loudly_without_library(tmp_path):
    old = D._lib
    D._lib = None
    try:
        with pytest.raises(RuntimeError, match="no CPU fallback"):
            D.load(str(tmp_path / "missing.so"))
    finally:
        D._lib = old
