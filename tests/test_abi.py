"""The C-ABI library builds, loads and exports every symbol include/sgn.h declares.

These tests run without a GPU: they make no compute call, only argument
validation that the library performs before touching the device.
"""
import ctypes
import os
import re

import pytest

from paper_2306_09731_gb300 import build as B
from paper_2306_09731_gb300 import sgn as S

INCLUDE = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include")
HEADER = os.path.join(INCLUDE, "sgn.h")
UNET_HEADER = os.path.join(INCLUDE, "sgn_unet.h")


def declared_symbols(header=HEADER):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sgn_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return S.load_library()


def test_header_and_binding_agree():
    from paper_2306_09731_gb300 import unet as UN
    assert declared_symbols() == sorted(S.EXPORTS)
    assert declared_symbols(UNET_HEADER) == sorted(UN.UNET_EXPORTS)
    assert sorted(os.listdir(INCLUDE)) == ["sgn.h", "sgn_unet.h"]


def test_library_exports_every_declared_symbol(lib):
    for name in declared_symbols() + declared_symbols(UNET_HEADER):
        assert hasattr(lib, name), name


@pytest.mark.parametrize("n,batch", [(8, 1), (24, 1), (1024, 1), (64, 0), (64, 65)])
def test_unet_create_rejects_bad_sizes(lib, n, batch):
    from paper_2306_09731_gb300 import unet as UN
    UN.load_library()
    h = ctypes.c_void_p()
    assert lib.sgn_unet_create(n, batch, 1, 0, ctypes.byref(h)) == 1  # SGN_EINVAL, before any device work
    assert not h.value


@pytest.mark.parametrize("n,levels,widths", [(64, 1, [32]), (64, 7, [16] * 7), (64, 3, [16, 24, 32]),
                                             (64, 3, [16, 32, 512]), (16, 4, [16, 16, 16, 16]), (64, 2, None)])
def test_unet_create_arch_rejects_bad_architectures(lib, n, levels, widths):
    from paper_2306_09731_gb300 import unet as UN
    UN.load_library()
    h = ctypes.c_void_p()
    wa = None if widths is None else (ctypes.c_int * len(widths))(*widths)
    assert lib.sgn_unet_create_arch(n, 1, 1, 0, levels, wa, ctypes.byref(h)) == 1
    assert not h.value


@pytest.mark.parametrize("H,W,C0,C1,Co", [(12, 16, 16, 0, 16), (16, 16, 8, 0, 16), (16, 16, 16, 8, 16),
                                          (16, 16, 16, 0, 24), (16, 16, 16, 0, 512), (16, 16, 1024, 16, 16)])
def test_conv3_tc_rejects_bad_shapes(lib, H, W, C0, C1, Co):
    from paper_2306_09731_gb300 import unet as UN
    UN.load_library()
    dummy = ctypes.c_void_p(16)  # never dereferenced: the shape checks come first
    assert lib.sgn_conv3_relu_bf16(1, H, W, dummy, C0, 0, dummy, C1, dummy, dummy, Co, dummy, dummy, 1 << 30,
                                   None) == 1
    assert lib.sgn_conv3_workspace_bytes(32, 32) == ((9 * 32 * 32 * 2 + 15) // 16) * 16 + 16


def test_default_options(lib):
    o = S.sgn_default_options()
    assert (o.precision, o.restart, o.maxit, o.tol, o.krasny, o.krasny_thr, o.dealias, o.guess) == \
        (0, 20, 1000, 1e-10, 0, 1e-12, 0, 0)


@pytest.mark.parametrize("Nx,Ny", [(12, 16), (16, 4), (8192, 16), (16, 8192), (0, 8), (16, -8)])
def test_create_rejects_bad_sizes(lib, Nx, Ny):
    h = ctypes.c_void_p()
    st = lib.sgn_create(Nx, Ny, 1.0, 1.0, 1.0, None, ctypes.byref(h))
    assert st == S.SGN_EINVAL and not h.value
    assert b"power" in lib.sgn_last_error(None)


def test_create_rejects_bad_options(lib):
    o = S.sgn_default_options()
    o.restart = 0
    h = ctypes.c_void_p()
    assert lib.sgn_create(16, 16, 1.0, 1.0, 1.0, ctypes.byref(o), ctypes.byref(h)) == S.SGN_EINVAL
    o = S.sgn_default_options()
    o.precision = 7
    assert lib.sgn_create(16, 16, 1.0, 1.0, 1.0, ctypes.byref(o), ctypes.byref(h)) == S.SGN_EINVAL
    assert lib.sgn_create(16, 16, -1.0, 1.0, 1.0, None, ctypes.byref(h)) == S.SGN_EINVAL


def test_null_handle_is_einval(lib):
    assert lib.sgn_rk4_step(None, None, None, None, None, 1e-3, 1) == S.SGN_EINVAL
    assert lib.sgn_destroy(None) == S.SGN_EINVAL
