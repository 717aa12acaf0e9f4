"""The allocation-free entry point against the plan-based one.

openfft_exec_c2c_noalloc serves callers that may not allocate device memory
(its scratch is a static device array).  Its output must equal, within the
tolerances of the other GPU tests, what openfft_exec_c2c returns for the same
input, on two calls in a row (the second reuses the static array the first
one left behind).  This file sorts last so that a run stopping at the first
failure has run every other test before it.
"""
import numpy as np
import pytest

from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {of.C2C_F64: 1e-12, of.C2C_F32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [((32, 32, 32), 4, of.C2C_F64), ((24, 40, 30), 6, of.C2C_F64), ((100, 108, 96), 8, of.C2C_F64),
         ((64, 64, 64), 8, of.C2C_F32), ((120, 144, 60), 32, of.C2C_F32)]


@pytest.mark.parametrize("shape,P,dtype", CASES)
def test_noalloc_matches_plan_on_two_calls(torch, shape, P, dtype):
    Na, Nb, Nc = shape
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    stream = torch.cuda.current_stream()
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        of.openfft_set_stream(plan, stream)
        for call, seed in enumerate((11, 12)):
            x = torch.from_numpy(synth.complex_field((Na * Nb * Nc,), seed=seed)).to("cuda", tdt)
            for direction in (of.FORWARD, of.BACKWARD):
                ref = torch.empty_like(x)
                got = torch.full_like(x, float("nan"))
                of.openfft_exec_c2c(plan, x, ref, direction)
                of.openfft_exec_c2c_noalloc(Na, Nb, Nc, P, dtype, x, got, direction, stream)
                torch.cuda.synchronize()
                err = _rel(got.cpu().numpy().astype(np.complex128), ref.cpu().numpy().astype(np.complex128))
                assert err < TOL[dtype], (shape, dtype, call, direction, err)
    finally:
        of.openfft_destroy(plan)


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_exec_c2c_noalloc(128, 128, 128, 4, of.C2C_F64, x, y, of.FORWARD)
    assert ei.value.status == of.ERR_UNSUPPORTED
    assert "16 MiB" in str(ei.value)
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_exec_c2c_noalloc(8, 8, 8, 2, of.C2C_F64, x, x, of.FORWARD)
    assert ei.value.status == of.ERR_ALIAS
