"""Split-precision tensor-core DFT-GEMM form against the FP64 oracle.

Stated bounds (fixed before the first GPU run): relative L2 <= 1e-5 for the
tf32 hi/lo form, <= 1e-4 for the bf16 hi/lo form, on the same complex64
input as the oracle's (upcast)."""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

FORMS = [(of.C2C_SPLIT_TF32, 1e-5), (of.C2C_SPLIT_BF16, 1e-4)]


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    return _t


def _run(torch, plan, x, direction):
    xd = torch.from_numpy(np.ascontiguousarray(x.reshape(-1))).to("cuda", torch.complex64)
    yd = torch.full_like(xd, float("nan"))
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_c2c(plan, xd, yd, direction)
    of.openfft_sync(plan)
    return yd.cpu().numpy().astype(np.complex128)


@pytest.mark.parametrize("dtype,tol", FORMS)
@pytest.mark.parametrize("shape,P", [((120, 144, 160), 32), ((32, 32, 32), 4), ((12, 10, 16), 20), ((64, 256, 48), 16)])
def test_dftgemm_forward_and_round_trip(torch, dtype, tol, shape, P):
    Na, Nb, Nc = shape
    x = synth.complex_field(shape, seed=synth.config_seed(3)).astype(np.complex64)
    ref = oracle.fft3d(x.astype(np.complex128), Na, Nb, Nc, P, oracle.FORWARD)
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        y = _run(torch, plan, x, of.FORWARD)
        assert oracle.rel_l2(y, ref) < tol, (shape, dtype, oracle.rel_l2(y, ref))
        z = _run(torch, plan, y.astype(np.complex64), of.BACKWARD)
        assert oracle.rel_l2(z, x.reshape(-1).astype(np.complex128)) < 2 * tol
    finally:
        of.openfft_destroy(plan)


@pytest.mark.parametrize("dtype,tol", FORMS)
@pytest.mark.parametrize("k0", [(0, 0, 0), (1, 2, 3), (59, 71, 79), (119, 143, 159)])
def test_dftgemm_plane_waves(torch, dtype, tol, k0):
    Na, Nb, Nc = 120, 144, 160
    N = Na * Nb * Nc
    x = synth.plane_wave(Na, Nb, Nc, k0).astype(np.complex64)
    exact = np.zeros((Na, Nb, Nc), complex)
    exact[k0] = N
    plan = of.openfft_plan(Na, Nb, Nc, 32, dtype)
    try:
        y = _run(torch, plan, x, of.FORWARD)
        assert np.linalg.norm(y - oracle.abc_to_cba(exact)) / (N * np.sqrt(N)) < tol
    finally:
        of.openfft_destroy(plan)


def test_dftgemm_rejects_unfactorable_axes(torch):
    for shape in [(37, 8, 8), (8, 8, 2)]:
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_plan(*shape, 2, of.C2C_SPLIT_TF32)
        assert ei.value.status == of.ERR_UNSUPPORTED_RADIX


def test_dftgemm_wait_timeout_is_reported(torch):
    """A completion wait that runs out (no MMA issued: nothing in flight) is
    reported as OPENFFT_ERR_TIMEOUT, and the context stays usable."""
    Na = Nb = Nc = 32
    x = synth.complex_field((Na, Nb, Nc), seed=synth.config_seed(3)).astype(np.complex64)
    ref = oracle.fft3d(x.astype(np.complex128), Na, Nb, Nc, 4, oracle.FORWARD)
    plan = of.openfft_plan(Na, Nb, Nc, 4, of.C2C_SPLIT_TF32)
    try:
        xd = torch.from_numpy(x.reshape(-1)).to("cuda")
        yd = torch.empty_like(xd)
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        try:
            of.openfft_tc_debug(1, 2_000_000)            # about 1 ms of clock cycles
            of.openfft_tc_debug(2, 1)                    # no MMA is issued or committed
            of.openfft_exec_c2c(plan, xd, yd, of.FORWARD)
            with pytest.raises(of.OpenFFTError) as ei:
                of.openfft_sync(plan)
            assert ei.value.status == of.ERR_TIMEOUT
        finally:
            of.openfft_tc_debug(2, 0)
            of.openfft_tc_debug(1, 0)
        y = _run(torch, plan, x, of.FORWARD)
        assert oracle.rel_l2(y, ref) < 1e-5
    finally:
        of.openfft_destroy(plan)
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_tc_debug(3, 0)
    assert ei.value.status == of.ERR_INVALID_ARG
