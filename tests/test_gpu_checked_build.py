"""The bounds-checked build (-DOPENFFT_CHECKED) on the small parity shapes.

A child pytest process loads libopenfft_gb_checked.so (OPENFFT_GB_CHECKED=1)
and runs the parity tests of every C2C form on small shapes: every candidate
of 32^3 P = 4 and of the small mixed-radix shapes, the transposes of every
exchange method, the longest axes, the 256- and 512-point axes of the
power-of-two warp kernels and their asynchronous-output form (with ragged
tiles), the host-buffer entry points (line-range launches), the D-dimensional
plans and the multi-device steps on one device.  Each test there still compares with the
oracle at its own bar, and additionally every kernel's global indices are
checked: openfft_sync fails with OPENFFT_ERR_BOUNDS on a plan's word and the
conftest fixture reads the per-device word after each test.  No test plants
an index outside an array.
"""
import os
import subprocess
import sys

import pytest

from paper_1501_07350_gb300 import _build
from paper_1501_07350_gb300 import openfft as of

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SELECTION = [
    ("tests/test_gpu_fft.py", "32cubed or small_shapes or transposes_bit_exact or longest_axes or mixed_radix"),
    ("tests/test_gpu_parity_bench.py", "long_power_of_two_axes or ragged_tiles"),
    ("tests/test_gpu_host_exec.py", ""),
    ("tests/test_gpu_nd.py", ""),
    ("tests/test_gpu_dist.py", ""),
]


def test_checked_build_exports_and_reports():
    import torch
    assert torch.cuda.is_available()
    _build.build()
    lib = _build.build(checked=True)
    assert os.path.exists(lib)
    # the normal library answers that it is not the checked one
    assert not of.openfft_checked_build()
    with pytest.raises(of.OpenFFTError) as e:
        of.openfft_debug_bounds_status()
    assert e.value.status == of.ERR_UNSUPPORTED


@pytest.mark.parametrize("path,expr", SELECTION, ids=[os.path.basename(p)[:-3] for p, _ in SELECTION])
def test_parity_suite_under_the_checked_build(path, expr):
    _build.build(checked=True)
    env = dict(os.environ, OPENFFT_GB_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-q", "-x", "-m", "gpu", "-p", "no:cacheprovider", path]
    if expr:
        cmd += ["-k", expr]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    assert " passed" in r.stdout and " failed" not in r.stdout, tail
