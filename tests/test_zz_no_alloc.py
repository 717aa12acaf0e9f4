"""The allocation-free entry point, against the oracle and the plan-based one.

openfft_exec_c2c_noalloc serves callers that may not allocate device memory
(a host framework whose own allocator owns the device budget, or a path that
must not pay for the synchronisation a cudaMalloc / cudaFree can imply): its
scratch is a static device array.  Its output must match the FP64 oracle and
what openfft_exec_c2c returns for the same input, within the tolerances of the
other GPU tests, on two calls in a row (the second reuses the static array the
first one left behind), and a warm call must leave the device's free memory
unchanged.  Sizes at the array's 16 MiB limit are accepted, sizes beyond it
refused.  This file sorts last so that a run stopping at the first failure
has run every other test before it.
"""
import numpy as np
import pytest

import oracle
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


# the last two sit exactly at the 16 MiB limit (N * 16 bytes = 2^24), one of
# them with an axis of 2048, the longest the entry point accepts
CASES = [((32, 32, 32), 4, of.C2C_F64), ((24, 40, 30), 6, of.C2C_F64), ((100, 108, 96), 8, of.C2C_F64),
         ((64, 64, 64), 8, of.C2C_F32), ((120, 144, 60), 32, of.C2C_F32),
         ((128, 128, 64), 64, of.C2C_F64), ((2048, 32, 16), 16, of.C2C_F64)]


@pytest.mark.parametrize("shape,P,dtype", CASES)
def test_noalloc_matches_oracle_and_plan_on_two_calls(torch, shape, P, dtype):
    Na, Nb, Nc = shape
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    stream = torch.cuda.current_stream()
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        of.openfft_set_stream(plan, stream)
        for call, seed in enumerate((11, 12)):
            xh = synth.complex_field((Na * Nb * Nc,), seed=seed)
            x = torch.from_numpy(xh).to("cuda", tdt)
            xin = x.cpu().numpy().astype(np.complex128)       # the input as the plan sees it
            for direction in (of.FORWARD, of.BACKWARD):
                want = oracle.fft3d(xin, Na, Nb, Nc, P, direction)
                ref = torch.empty_like(x)
                got = torch.full_like(x, float("nan"))
                of.openfft_exec_c2c(plan, x, ref, direction)
                of.openfft_exec_c2c_noalloc(Na, Nb, Nc, P, dtype, x, got, direction, stream)
                torch.cuda.synchronize()
                g = got.cpu().numpy().astype(np.complex128)
                e_oracle = oracle.rel_l2(g, want)
                e_plan = _rel(g, ref.cpu().numpy().astype(np.complex128))
                assert e_oracle < TOL[dtype], (shape, dtype, call, direction, e_oracle)
                assert e_plan < TOL[dtype], (shape, dtype, call, direction, e_plan)
    finally:
        of.openfft_destroy(plan)


def test_noalloc_warm_call_leaves_free_memory_unchanged(torch):
    Na, Nb, Nc, P = 64, 48, 40, 8
    stream = torch.cuda.current_stream()
    x = torch.from_numpy(synth.complex_field((Na * Nb * Nc,), seed=5)).cuda()
    y = torch.empty_like(x)
    of.openfft_exec_c2c_noalloc(Na, Nb, Nc, P, of.C2C_F64, x, y, of.FORWARD, stream)    # warm-up
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    of.openfft_exec_c2c_noalloc(Na, Nb, Nc, P, of.C2C_F64, x, y, of.FORWARD, stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    want = oracle.fft3d(x.cpu().numpy(), Na, Nb, Nc, P, oracle.FORWARD)
    assert oracle.rel_l2(y.cpu().numpy(), want) < TOL[of.C2C_F64]


def test_noalloc_rejects_sizes_beyond_its_scratch(torch):
    x = torch.zeros(8, dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    # one c-line past the 16 MiB limit, and an axis past 2048
    for shape in [(128, 128, 65), (128, 128, 128), (4096, 2, 2)]:
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_c2c_noalloc(*shape, 4, of.C2C_F64, x, y, of.FORWARD)
        assert ei.value.status == of.ERR_UNSUPPORTED, shape
        assert "16 MiB" in str(ei.value)
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_exec_c2c_noalloc(8, 8, 8, 2, of.C2C_F64, x, x, of.FORWARD)
    assert ei.value.status == of.ERR_ALIAS
