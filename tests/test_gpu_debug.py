"""The bounds-checked debug build (libfunnel_debug.so, FT_DEBUG): every gather /
scatter index of the fixed-length kernels and the peak pass is checked on the
device; the transform, its adjoint and both peak passes on 8 x 8 ... 256 x 128
and odd-radix (2^a 3^b) sizes must match the oracle with no check firing.
Runs in a child process, which loads the debug library in place of the normal
one."""
import os
import subprocess
import sys

import pytest

from tests import _gpu

pytestmark = pytest.mark.gpu


def test_debug_build_index_checks_stay_clean():
    _gpu.torch_cuda()                                   # the normal library (built if missing)
    from paper_1904_09409_gb300 import funnel as f
    if not os.path.exists(os.path.join(f.PKG, "libfunnel_debug.so")):
        from paper_1904_09409_gb300 import build
        build.build()
    child = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_debug_child.py")
    r = subprocess.run([sys.executable, child], capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK"), r.stdout + r.stderr


def test_normal_build_has_no_checks():
    _gpu.torch_cuda()
    from paper_1904_09409_gb300 import funnel as f
    if os.environ.get("FT_DEBUG") == "1":
        pytest.skip("this process runs the debug build")
    assert not f.ft_debug_build()
    assert f.ft_debug_flags() == 0
