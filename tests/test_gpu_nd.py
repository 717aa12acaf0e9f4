"""D-dimensional transforms on the GPU (openfft_nd_*) against the oracle.

Whole outputs, element by element (relative L2): 1e-12 for complex128
(double-float arithmetic), 1e-5 for complex64 against the oracle on the same
input upcast; both directions; 4-D and 5-D shapes with mixed radices, slab
and pencil decompositions, and 256- / 512-point axes that run the
asynchronous-output stage kernel.  The D = 3 case must agree with the 3-D
plan.
"""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {of.C2C_F64: 1e-12, of.C2C_F32: 1e-5}

CASES = [((4, 3, 5, 2), 8), ((6, 4, 2, 3), 5), ((2, 3, 2, 2, 3), 6), ((3, 4, 2, 2, 5), 7), ((8, 8, 4, 4), 16),
         ((12, 10, 9, 14), 40), ((16, 16, 16, 16), 64), ((8, 6, 10, 12, 4), 24), ((32, 256, 4, 8), 32),
         ((4, 8, 512, 16), 32), ((256, 8, 8, 16), 128), ((1, 7, 5, 3), 1)]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


@pytest.mark.parametrize("dtype", [of.C2C_F64, of.C2C_F32])
@pytest.mark.parametrize("dims,P", CASES)
def test_nd_transform_matches_oracle(torch, dims, P, dtype):
    N = int(np.prod(dims))
    x = synth.complex_field((N,), seed=N + P)
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    xd = torch.from_numpy(x).to("cuda", tdt)
    xin = xd.cpu().numpy().astype(np.complex128)
    plan = of.openfft_nd_plan(dims, P, dtype)
    try:
        of.openfft_nd_set_stream(plan, torch.cuda.current_stream())
        for direction in (of.FORWARD, of.BACKWARD):
            yd = torch.full_like(xd, float("nan"))
            of.openfft_nd_exec(plan, xd, yd, direction)
            torch.cuda.synchronize()
            ref = oracle.fftnd(xin, dims, P, direction)
            e = oracle.rel_l2(yd.cpu().numpy().astype(np.complex128), ref)
            assert e < TOL[dtype], (dims, P, direction, e)
        assert np.array_equal(xd.cpu().numpy().astype(np.complex128), xin)     # input untouched
        D = len(dims)
        for which, s in ((0, 1), (1, D)):
            xs = oracle.nd_boundaries(dims, P, s)
            for r in (0, P // 2, P - 1):
                assert of.openfft_nd_box(plan, which, r) == (xs[r], xs[r + 1] - xs[r])
    finally:
        of.openfft_nd_destroy(plan)


def test_three_dims_agrees_with_the_3d_plan(torch):
    dims, P = (24, 20, 30), 6
    x = torch.from_numpy(synth.complex_field((24 * 20 * 30,), seed=1)).cuda()
    y3, yn = torch.empty_like(x), torch.empty_like(x)
    p3 = of.openfft_plan(*dims, P, of.C2C_F64)
    pn = of.openfft_nd_plan(dims, P, of.C2C_F64)
    try:
        of.openfft_set_stream(p3, torch.cuda.current_stream())
        of.openfft_nd_set_stream(pn, torch.cuda.current_stream())
        for d in (of.FORWARD, of.BACKWARD):
            of.openfft_exec_c2c(p3, x, y3, d)
            of.openfft_nd_exec(pn, x, yn, d)
            torch.cuda.synchronize()
            assert oracle.rel_l2(yn.cpu().numpy(), y3.cpu().numpy()) < 1e-13
    finally:
        of.openfft_destroy(p3)
        of.openfft_nd_destroy(pn)


def test_nd_errors(torch):
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_nd_plan((4, 3, 5, 2), 9, of.C2C_F64)
    assert ei.value.status == of.ERR_P_TOO_LARGE
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_nd_plan((4, 11, 5, 2), 2, of.C2C_F64)
    assert ei.value.status == of.ERR_UNSUPPORTED_RADIX
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_nd_plan((4, 3, 5, 2), 2, of.C2C_SPLIT_TF32)
    assert ei.value.status == of.ERR_UNSUPPORTED
    plan = of.openfft_nd_plan((4, 4, 4, 4), 4, of.C2C_F64)
    try:
        x = torch.zeros(256, dtype=torch.complex128, device="cuda")
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_nd_exec(plan, x, x, of.FORWARD)
        assert ei.value.status == of.ERR_ALIAS
    finally:
        of.openfft_nd_destroy(plan)
