"""Batched persistent form (openfft_plan_many / openfft_exec_many) against the oracle.

Every transform of a batch is compared with the FP64 oracle on its own input:
complex64 plans within 1e-5 relative L2, complex128 (double-float) within
1e-12.  A host-side test hook makes one dependency wait of the persistent
kernel run out; the kernel must report OPENFFT_ERR_TIMEOUT through the status
word and leave the context usable (no trap, no hang).
"""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _inputs(torch, shapes, seed0, dtype):
    tdt = torch.complex64 if dtype == of.C2C_F32 else torch.complex128
    xs = [synth.complex_field(s, seed=seed0 + i) for i, s in enumerate(shapes)]
    xd = [torch.from_numpy(x.reshape(-1)).to("cuda", tdt) for x in xs]
    return xs, xd


def _check_batch(torch, plan, shapes, Ps, xs, xd, dtype, tol):
    yd = [torch.full_like(x, float("nan")) for x in xd]
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_many(plan, xd, yd, of.FORWARD)
    of.openfft_sync(plan)
    for (Na, Nb, Nc), P, x, y in zip(shapes, Ps, xs, yd):
        xin = x.astype(np.complex64).astype(np.complex128) if dtype == of.C2C_F32 else x
        ref = oracle.fft3d(xin, Na, Nb, Nc, P, oracle.FORWARD)
        assert oracle.rel_l2(y.cpu().numpy().astype(np.complex128), ref) < tol, (Na, Nb, Nc)
    zd = [torch.full_like(x, float("nan")) for x in xd]
    of.openfft_exec_many(plan, yd, zd, of.BACKWARD)
    of.openfft_sync(plan)
    for x, z in zip(xd, zd):
        assert float(torch.linalg.vector_norm(z - x) / torch.linalg.vector_norm(x)) < tol


def test_batch_uneven_complex64(torch):
    shapes = synth.batch_shapes(synth.config_seed(4), 12)
    Ps = [8] * len(shapes)
    plan = of.openfft_plan_many(shapes, Ps, of.C2C_F32)
    try:
        xs, xd = _inputs(torch, shapes, synth.config_seed(4) + 1, of.C2C_F32)
        _check_batch(torch, plan, shapes, Ps, xs, xd, of.C2C_F32, 1e-5)
        # second replay with a new pointer set
        xs2, xd2 = _inputs(torch, shapes, 777, of.C2C_F32)
        _check_batch(torch, plan, shapes, Ps, xs2, xd2, of.C2C_F32, 1e-5)
    finally:
        of.openfft_destroy(plan)


def test_batch_complex128_and_generic_lengths(torch):
    # 36, 25, 49 and 14 have no specialised tile body: the generic body runs them
    shapes = [(48, 48, 48), (9, 25, 14), (7, 49, 6), (100, 108, 120), (36, 40, 30), (1, 8, 1)]
    Ps = [8, 7, 42, 8, 64, 1]
    plan = of.openfft_plan_many(shapes, Ps, of.C2C_F64)
    try:
        xs, xd = _inputs(torch, shapes, 4242, of.C2C_F64)
        _check_batch(torch, plan, shapes, Ps, xs, xd, of.C2C_F64, 1e-12)
    finally:
        of.openfft_destroy(plan)
    plan = of.openfft_plan_many(shapes, Ps, of.C2C_F32)
    try:
        xs, xd = _inputs(torch, shapes, 4343, of.C2C_F32)
        _check_batch(torch, plan, shapes, Ps, xs, xd, of.C2C_F32, 1e-5)
    finally:
        of.openfft_destroy(plan)


def test_batch_wait_timeout_is_reported(torch):
    shapes = [(48, 48, 48), (64, 64, 64)]
    Ps = [8, 8]
    plan = of.openfft_plan_many(shapes, Ps, of.C2C_F32)
    try:
        xs, xd = _inputs(torch, shapes, 5, of.C2C_F32)
        yd = [torch.empty_like(x) for x in xd]
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        of.openfft_batch_debug(plan, 1, 2_000_000)       # ~1 ms of clock cycles
        of.openfft_batch_debug(plan, 2, 1)               # a first-stage tile that never comes
        of.openfft_exec_many(plan, xd, yd, of.FORWARD)
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_sync(plan)
        assert ei.value.status == of.ERR_TIMEOUT
        # the context is intact: undo the hook and run again
        of.openfft_batch_debug(plan, 2, 0)
        of.openfft_batch_debug(plan, 1, 2_000_000_000)
        _check_batch(torch, plan, shapes, Ps, xs, xd, of.C2C_F32, 1e-5)
    finally:
        of.openfft_destroy(plan)


def test_batch_argument_errors(torch):
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_plan_many([(8, 8, 8), (11, 8, 8)], [2, 2], of.C2C_F32)
    assert ei.value.status == of.ERR_UNSUPPORTED_RADIX
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_plan_many([(8, 8, 8)], [65], of.C2C_F32)
    assert ei.value.status == of.ERR_P_TOO_LARGE
    plan = of.openfft_plan_many([(8, 8, 8)], [2], of.C2C_F32)
    try:
        x = torch.zeros(512, dtype=torch.complex64, device="cuda")
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_many(plan, [x], [x], of.FORWARD)
        assert ei.value.status == of.ERR_ALIAS
        with pytest.raises(of.OpenFFTError):
            of.openfft_exec_c2c(plan, x, torch.zeros_like(x), of.FORWARD)
    finally:
        of.openfft_destroy(plan)
