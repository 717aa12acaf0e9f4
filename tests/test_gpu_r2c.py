"""Real transforms (OPENFFT_R2C_F64 / _F32) against the FP64 oracle, through the C ABI.

Bars (the same as for the complex plans, fixed before the first GPU run):
FP64-accurate plans <= 1e-12 relative L2, FP32 plans <= 1e-5, boxes bit-exact.
Half spectra are [Nc//2+1][Nb][Na] (cba order), real arrays [Na][Nb][Nc].
"""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {of.R2C_F64: 1e-12, of.R2C_F32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _types(torch, dtype):
    return (torch.float64, torch.complex128) if dtype == of.R2C_F64 else (torch.float32, torch.complex64)


def _r2c(torch, plan, x, dtype, Nch):
    rt, ct = _types(torch, dtype)
    Na_Nb = x.size // x.shape[-1]
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to(device="cuda", dtype=rt)
    yd = torch.full((Nch * Na_Nb,), float("nan"), dtype=ct, device="cuda")
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_r2c(plan, xd, yd)
    of.openfft_sync(plan)
    assert np.array_equal(xd.cpu().numpy(), x.reshape(-1).astype(xd.cpu().numpy().dtype))   # input untouched
    return yd.cpu().numpy().astype(np.complex128)


def _c2r(torch, plan, h, dtype, N):
    rt, ct = _types(torch, dtype)
    hd = torch.from_numpy(np.ascontiguousarray(h.reshape(-1))).to(device="cuda", dtype=ct)
    h0 = hd.clone()
    xd = torch.full((N,), float("nan"), dtype=rt, device="cuda")
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_c2r(plan, hd, xd)
    of.openfft_sync(plan)
    assert torch.equal(hd, h0)
    return xd.cpu().numpy().astype(np.float64)


SHAPES = [((32, 32, 32), 4), ((120, 144, 160), 32), ((12, 10, 15), 6), ((64, 48, 256), 64),
          ((16, 20, 24), 200), ((9, 7, 2), 14), ((40, 36, 1), 8), ((3, 2, 2048), 3), ((2, 5, 1792), 4)]


@pytest.mark.parametrize("dtype", [of.R2C_F64, of.R2C_F32])
@pytest.mark.parametrize("shape,P", SHAPES)
def test_r2c_and_c2r_match_the_oracle(torch, dtype, shape, P):
    Na, Nb, Nc = shape
    N, Nch = Na * Nb * Nc, Nc // 2 + 1
    x = synth.uniform_pm1(synth.config_seed(21) + Nc, N).reshape(shape)
    ref = oracle.rfft3d(x, Na, Nb, Nc, P)
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        y = _r2c(torch, plan, x, dtype, Nch)
        assert oracle.rel_l2(y, ref) < TOL[dtype], (shape, P)
        # inverse of an arbitrary half spectrum (not Hermitian-consistent)
        h = synth.complex_field((Nch, Nb, Na), seed=synth.config_seed(22) + Nc).reshape(-1)
        xr = oracle.rfft3d(h, Na, Nb, Nc, P, oracle.BACKWARD)
        xg = _c2r(torch, plan, h, dtype, N)
        assert np.linalg.norm(xg - xr) <= TOL[dtype] * np.linalg.norm(xr), (shape, P)
        # round trip
        back = _c2r(torch, plan, y, dtype, N)
        assert np.linalg.norm(back - x.reshape(-1)) <= 2 * TOL[dtype] * np.linalg.norm(x)
    finally:
        of.openfft_destroy(plan)


@pytest.mark.parametrize("dtype", [of.R2C_F64, of.R2C_F32])
def test_r2c_every_candidate(torch, dtype):
    Na, Nb, Nc, P = 48, 40, 64, 12
    x = synth.normal(synth.config_seed(23), Na * Nb * Nc).reshape(Na, Nb, Nc)
    ref = oracle.rfft3d(x, Na, Nb, Nc, P)
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        n = of.openfft_num_candidates(plan)
        assert n == (10 if dtype == of.R2C_F64 else 5)
        for c in range(n):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            y = _r2c(torch, plan, x, dtype, Nc // 2 + 1)
            assert oracle.rel_l2(y, ref) < TOL[dtype], of.openfft_candidate(plan, c)
            back = _c2r(torch, plan, y, dtype, x.size)
            assert np.linalg.norm(back - x.reshape(-1)) <= 2 * TOL[dtype] * np.linalg.norm(x)
        of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
        assert oracle.rel_l2(_r2c(torch, plan, x, dtype, Nc // 2 + 1), ref) < TOL[dtype]
    finally:
        of.openfft_destroy(plan)


def test_r2c_256cubed_sampled_lines(torch):
    """The bench size: sampled output lines against the 3-D DFT by its definition."""
    n, P = 256, 64
    x = synth.normal(synth.config_seed(2), n ** 3).reshape(n, n, n)
    plan = of.openfft_plan(n, n, n, P, of.R2C_F64)
    try:
        y = _r2c(torch, plan, x, of.R2C_F64, n // 2 + 1)
    finally:
        of.openfft_destroy(plan)
    for kb, kc in [(0, 0), (1, 2), (255, 128), (77, 100)]:
        ref = oracle.dft3d_line(x.astype(np.complex128), kb, kc, oracle.FORWARD)
        got = y[(kc * n + kb) * n:(kc * n + kb + 1) * n]
        assert oracle.rel_l2(got, ref) < TOL[of.R2C_F64], (kb, kc)


@pytest.mark.parametrize("shape,P", [((24, 20, 30), 16), ((8, 8, 8), 40), ((16, 12, 9), 5)])
def test_r2c_boxes_follow_the_half_orderings(torch, shape, P):
    Na, Nb, Nc = shape
    Nch = Nc // 2 + 1
    plan = of.openfft_plan(Na, Nb, Nc, P, of.R2C_F64)
    try:
        def want(N1, N2, N3, r):
            xs, xe, s3, e3 = oracle.box(N1, N2, N3, P, r)
            return s3, e3, xs, xe - xs + 1
        for r in range(P):
            assert of.openfft_box(plan, 0, r) == want(Na, Nb, Nc, r)
            assert of.openfft_box(plan, 1, r) == want(Nch, Nb, Na, r)
        for ex in (1, 2):
            want = oracle.rfft3d(np.zeros(Na * Nb * Nc), Na, Nb, Nc, P, counts=True)[ex]
            assert np.array_equal(of.openfft_counts(plan, ex, P), want)
    finally:
        of.openfft_destroy(plan)


def test_r2c_errors(torch):
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_plan(3, 4, 5, 12, of.R2C_F64)          # cab half (3, 3, 4): 9 < 12
    assert ei.value.status == of.ERR_P_TOO_LARGE
    rp = of.openfft_plan(8, 8, 8, 4, of.R2C_F64)
    cp = of.openfft_plan(8, 8, 8, 4, of.C2C_F64)
    try:
        a = torch.zeros(512, dtype=torch.complex128, device="cuda")
        b = torch.zeros(512, dtype=torch.complex128, device="cuda")
        for call in (lambda: of.openfft_exec_c2c(rp, a, b, of.FORWARD), lambda: of.openfft_exec_r2c(cp, a, b),
                     lambda: of.openfft_exec_c2r(cp, a, b)):
            with pytest.raises(of.OpenFFTError) as ei:
                call()
            assert ei.value.status == of.ERR_INVALID_ARG
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_r2c(rp, a, a)
        assert ei.value.status == of.ERR_ALIAS
    finally:
        of.openfft_destroy(rp)
        of.openfft_destroy(cp)
