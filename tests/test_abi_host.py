"""Host-side checks of the C ABI: the library builds, loads and exports every
function declared in include/funnel.h, and argument validation answers before
any GPU work.  No compute call is made here (there may be no GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1904_09409_gb300 import funnel as f

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "funnel.h")


@pytest.fixture(scope="module")
def L():
    if not os.path.exists(f.LIB_PATH):
        from paper_1904_09409_gb300 import build
        build.build()
    return f.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\**\s+\**(ft_[a-z_0-9]+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ft_plan_create", "ft_plan_destroy", "ft_forward", "ft_backward", "ft_peaks",
              "ft_status_string"):
        assert n in names
    assert set(names) == set(f.EXPORTED)


def test_library_exports_every_declared_symbol(L):
    out = subprocess.run(["nm", "-D", "--defined-only", f.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (ft_[a-z_0-9]+)", out))
    missing = set(declared_functions()) - exported
    assert not missing, missing
    for n in declared_functions():
        assert hasattr(L, n)


def test_status_strings(L):
    for s in range(6):
        assert L.ft_status_string(s)
    assert L.ft_status_string(99) == b"unknown status"
    assert f.ft_status_string(f.FT_ERR_UNSUPPORTED_SIZE) == "unsupported size"


@pytest.mark.parametrize("H,W,S,Hp", [
    (16, 15, 16, 16),       # odd width
    (16, 16, 14, 16),       # n_slope < W
    (16, 16, 16, 10),       # n_intercept < H
    (16, 16, 16, 22),       # 22 = 2 * 11 is not 2^a 3^b
    (16, 16, 10, 16),       # n_slope 10 = 2 * 5
    (16, 16, 16, 16384),    # above FT_MAX_LENGTH
    (0, 16, 16, 16),        # empty image
    (16, 16, 16, 9),        # odd n_intercept
])
def test_unsupported_sizes_are_rejected(L, H, W, S, Hp):
    h = ctypes.c_void_p(123)
    st = L.ft_plan_create(ctypes.byref(h), H, W, S, Hp, 0)
    assert st == f.FT_ERR_UNSUPPORTED_SIZE
    assert h.value is None


def test_invalid_arguments(L):
    h = ctypes.c_void_p()
    assert L.ft_plan_create(None, 16, 16, 16, 16, 0) == f.FT_ERR_INVALID_ARG
    assert L.ft_plan_create(ctypes.byref(h), 16, 16, 16, 16, 7) == f.FT_ERR_INVALID_ARG
    assert L.ft_forward(None, None, None, 1, None) == f.FT_ERR_INVALID_ARG
    assert L.ft_backward(None, None, None, 1, None) == f.FT_ERR_INVALID_ARG
    assert L.ft_peaks(None, None, 1, 3, 0.0, None, None, None) == f.FT_ERR_INVALID_ARG
    assert L.ft_detect_host(None, None, 1, 3, 0.0, None, None, None) == f.FT_ERR_INVALID_ARG
    assert L.ft_detect(None, None, None, 1, 3, 0.0, None, None, None) == f.FT_ERR_INVALID_ARG
    assert L.ft_detect_launches(None, 4, 32) == 0
    # a NaN threshold is an argument error (checked before any GPU work)
    assert L.ft_peaks_noalloc(ctypes.c_void_p(256), 16, 16, 1, 3, float("nan"), ctypes.c_void_p(256),
                              ctypes.c_void_p(256), None) == f.FT_ERR_INVALID_ARG
    assert L.ft_plan_destroy(None) == f.FT_OK
    assert L.ft_workspace_bytes(None, 4) == 0
    assert L.ft_forward_launches(None, 4) == 0


def test_python_binding_raises_without_gpu_work(L):
    with pytest.raises(f.FunnelError) as e:
        f.ft_plan_create(16, 15, 16, 16, 0)
    assert e.value.status == f.FT_ERR_UNSUPPORTED_SIZE
