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


def test_grid_size_limit(lib):
    """Population planes are indexed with 32-bit offsets: a padded plane (rows
    rounded up to 64 nodes) must hold fewer than 2^32 elements.  Checked
    without allocating: the workspace query validates the parameters."""
    c = good(); c.nx, c.ny = 65536, 65536          # exactly 2^32 nodes
    p = c.to_c()
    assert lib.ddflb_workspace_bytes(ctypes.byref(p)) == 0
    assert "2^32" in lib.ddflb_last_error().decode()
    c = good(); c.nx, c.ny = 65537, 65535          # pads to 65600 x 65535 > 2^32
    p = c.to_c()
    assert lib.ddflb_workspace_bytes(ctypes.byref(p)) == 0
    c = good(); c.nx, c.ny = 65536, 65535          # the largest square-ish plane that fits
    c.storage = "fp16"
    p = c.to_c()
    n = lib.ddflb_workspace_bytes(ctypes.byref(p))
    assert n >= 2 * 18 * 65536 * 65535 * 2


def test_run_to_tolerance_rejects_null_handle(lib):
    assert lib.ddflb_run_to_tolerance(None, 1e-8, 10, 0, None) == D.EINVAL


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


def test_params_struct_layout_matches_header(tmp_path):
    """The ctypes mirror has the size and field offsets the C compiler gives
    ddflb_params (compiled here with gcc against include/ddflb.h)."""
    fields = [f[0] for f in D.Params._fields_]
    src = ['#include <stddef.h>', '#include <stdio.h>', '#include "ddflb.h"', "int main(void) {",
           'printf("%zu\\n", sizeof(ddflb_params));']
    src += [f'printf("%zu\\n", offsetof(ddflb_params, {f}));' for f in fields]
    src += ["return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(src))
    exe = tmp_path / "layout"
    import subprocess
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(c), "-o", str(exe)], check=True)
    out = [int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                          text=True).stdout.split()]
    assert out[0] == ctypes.sizeof(D.Params)
    assert out[1:] == [getattr(D.Params, f).offset for f in fields]


def test_force_parameters_validated(lib):
    p = good().to_c()
    p.fx = float("nan")
    assert lib.ddflb_workspace_bytes(ctypes.byref(p)) == 0
    assert "body force" in lib.ddflb_last_error().decode()


def test_batch_and_noalloc_reject_forcing(lib):
    c = good(); c.fx = 1e-6
    arr = (D.Params * 2)(good().to_c(), c.to_c())
    assert lib.ddflb_batch_workspace_bytes(2, arr) == 0
    assert "unforced" in lib.ddflb_last_error().decode()
    p = c.to_c()
    out = lib.ddflb_reduce_noalloc(ctypes.byref(p), 4096, 1 << 30, 0, 4096, None)
    assert out == D.EINVAL and "unforced" in lib.ddflb_last_error().decode()
