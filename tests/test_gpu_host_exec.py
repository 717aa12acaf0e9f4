"""Host-buffer execution (openfft_exec_c2c_host) through the C ABI.

The copies run on a second stream in ranges of lines that overlap the first
and the last stage.  The same kernels then run on the same lines as in
openfft_exec_c2c, so the result must equal the device-buffer result bit for
bit: for every candidate, range count and direction, with page-locked and
pageable buffers and in place.  The default candidate is also checked against
the FP64 oracle (relative L2 <= 1e-12 for FP64, 1e-5 for complex64 forms).
"""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {of.C2C_F64: 1e-12, of.C2C_F32: 1e-5, of.C2C_SPLIT_TF32: 1e-5}


@pytest.fixture(scope="module")
def torch():
    import torch as _t
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    assert _t.cuda.is_available()
    return _t


def _device(torch, plan, x, direction):
    xd = torch.from_numpy(x).to("cuda")
    yd = torch.empty_like(xd)
    of.openfft_set_stream(plan, torch.cuda.current_stream())
    of.openfft_exec_c2c(plan, xd, yd, direction)
    of.openfft_sync(plan)
    return yd.cpu().numpy()


def _bits(a):
    return a.view(np.uint64 if a.dtype == np.complex128 else np.uint32)


# (shape, P, dtype): ragged line counts for every range count, one axis of 7,
# the tensor-core form, and slabs as well as pencils (P > Na)
CASES = [((48, 40, 36), 6, of.C2C_F64), ((30, 28, 50), 5, of.C2C_F32), ((21, 9, 32), 40, of.C2C_F64),
         ((64, 48, 40), 12, of.C2C_SPLIT_TF32), ((16, 12, 20), 3, of.C2C_F64)]


@pytest.mark.parametrize("shape,P,dtype", CASES)
def test_host_exec_equals_device_exec(torch, shape, P, dtype):
    Na, Nb, Nc = shape
    cdt = np.complex128 if dtype == of.C2C_F64 else np.complex64
    tdt = torch.complex128 if dtype == of.C2C_F64 else torch.complex64
    x = synth.complex_field(shape, seed=Na * 10007 + Nb * 101 + Nc).reshape(-1).astype(cdt)
    hx = torch.from_numpy(x.copy()).pin_memory()
    hy = torch.empty_like(hx).pin_memory()
    plan = of.openfft_plan(Na, Nb, Nc, P, dtype)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        ref = oracle.fft3d(x.astype(np.complex128), Na, Nb, Nc, P, oracle.FORWARD)
        for c in range(of.openfft_num_candidates(plan)):
            of.openfft_set_tuning(plan, of.TUNE_USER, c)
            for direction in (of.FORWARD, of.BACKWARD):
                want = _device(torch, plan, x, direction)
                if c == 0 and direction == of.FORWARD:
                    assert oracle.rel_l2(want.astype(np.complex128), ref) < TOL[dtype]
                for chunks in (0, 1, 3, 7, 32):
                    of.openfft_set_host_chunks(plan, chunks)
                    hy.fill_(float("nan"))
                    of.openfft_exec_c2c_host(plan, hx.numpy(), hy.numpy(), direction)
                    assert np.array_equal(_bits(hy.numpy()), _bits(want)), (of.openfft_candidate(plan, c), chunks, direction)
        assert np.array_equal(_bits(hx.numpy()), _bits(x))                 # input untouched
    finally:
        of.openfft_destroy(plan)


def test_host_exec_in_place_and_pageable(torch):
    Na, Nb, Nc, P = 40, 36, 48, 8
    x = synth.complex_field((Na, Nb, Nc), seed=77).reshape(-1)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        want = _device(torch, plan, x, of.FORWARD)
        for chunks in (0, 5):
            of.openfft_set_host_chunks(plan, chunks)
            y = np.empty_like(x)                                            # pageable
            of.openfft_exec_c2c_host(plan, x, y, of.FORWARD)
            assert np.array_equal(_bits(y), _bits(want))
            h = torch.from_numpy(x.copy()).pin_memory()                    # one buffer, in place
            of.openfft_exec_c2c_host(plan, h.numpy(), h.numpy(), of.FORWARD)
            assert np.array_equal(_bits(h.numpy()), _bits(want))
            z = np.empty_like(x)                                            # pageable, in place
            z[:] = x
            of.openfft_exec_c2c_host(plan, z, z, of.FORWARD)
            assert np.array_equal(_bits(z), _bits(want))
    finally:
        of.openfft_destroy(plan)


def test_host_chunks_errors(torch):
    plan = of.openfft_plan(8, 8, 8, 2, of.C2C_F64)
    rplan = of.openfft_plan(8, 8, 8, 2, of.R2C_F64)
    try:
        for bad in (-1, 33):
            with pytest.raises(of.OpenFFTError) as ei:
                of.openfft_set_host_chunks(plan, bad)
            assert ei.value.status == of.ERR_INVALID_ARG
        a = np.zeros(512, np.complex128)
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_c2c_host(plan, a, a.copy(), 0)
        assert ei.value.status == of.ERR_INVALID_ARG
        with pytest.raises(of.OpenFFTError) as ei:
            of.openfft_exec_c2c_host(rplan, a, a.copy(), of.FORWARD)
        assert ei.value.status == of.ERR_INVALID_ARG
    finally:
        of.openfft_destroy(plan)
        of.openfft_destroy(rplan)


@pytest.mark.parametrize("shared_copy_streams", [False, True])
def test_async_host_exec_across_plans(torch, shared_copy_streams):
    """Asynchronous host-buffer calls on three plans, enqueued back to back and
    then synchronised, give the synchronous results bit for bit, forward and
    backward, with each plan's own copy streams or with one upload and one
    download stream shared by all three; calls queued on one plan run in order."""
    Na, Nb, Nc = 40, 36, 48
    x = synth.complex_field((Na, Nb, Nc), seed=81).reshape(-1)
    hx = torch.from_numpy(x.copy()).pin_memory()
    plans = [of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64) for P in (4, 12, 60)]
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    try:
        for h in plans:
            of.openfft_set_stream(h, torch.cuda.current_stream())
            of.openfft_set_host_chunks(h, 5)
            if shared_copy_streams:
                of.openfft_set_copy_streams(h, up, down)
        want_f = [_device(torch, h, x, of.FORWARD) for h in plans]
        ys = [torch.empty_like(hx).pin_memory() for _ in plans]
        zs = [torch.empty_like(hx).pin_memory() for _ in plans]
        for h, y in zip(plans, ys):
            y.fill_(float("nan"))
            of.openfft_exec_c2c_host_async(h, hx.numpy(), y.numpy(), of.FORWARD)
        for h in plans:
            of.openfft_sync(h)
        for y, w in zip(ys, want_f):
            assert np.array_equal(_bits(y.numpy()), _bits(w))
        want_b = [_device(torch, h, y.numpy(), of.BACKWARD) for h, y in zip(plans, ys)]
        for h, y, z in zip(plans, ys, zs):
            of.openfft_exec_c2c_host_async(h, y.numpy(), z.numpy(), of.BACKWARD)
        for h in plans:
            of.openfft_sync(h)
        for z, w in zip(zs, want_b):
            assert np.array_equal(_bits(z.numpy()), _bits(w))
            assert oracle.rel_l2(z.numpy(), x) < 1e-12
        # the benchmark's step: every forward, then every backward (each reading
        # its plan's forward output in host memory), one synchronisation at the end
        for y, z in zip(ys, zs):
            y.fill_(float("nan")); z.fill_(float("nan"))
        for h, y in zip(plans, ys):
            of.openfft_exec_c2c_host_async(h, hx.numpy(), y.numpy(), of.FORWARD)
        for h, y, z in zip(plans, ys, zs):
            of.openfft_exec_c2c_host_async(h, y.numpy(), z.numpy(), of.BACKWARD)
        for h in plans:
            of.openfft_sync(h)
        for y, z, wf, wb in zip(ys, zs, want_f, want_b):
            assert np.array_equal(_bits(y.numpy()), _bits(wf))
            assert np.array_equal(_bits(z.numpy()), _bits(wb))
        # two calls on one plan: the second reads the first one's output
        h, a, b = plans[0], ys[0], zs[0]
        a.fill_(float("nan")); b.fill_(float("nan"))
        of.openfft_exec_c2c_host_async(h, hx.numpy(), a.numpy(), of.FORWARD)
        of.openfft_sync(h)
        of.openfft_exec_c2c_host_async(h, a.numpy(), b.numpy(), of.BACKWARD)
        of.openfft_exec_c2c_host_async(h, b.numpy(), a.numpy(), of.FORWARD)
        of.openfft_sync(h)
        want = _device(torch, h, _device(torch, h, want_f[0], of.BACKWARD), of.FORWARD)
        assert np.array_equal(_bits(a.numpy()), _bits(want))
    finally:
        for h in plans:
            of.openfft_destroy(h)


def test_copy_streams_errors_and_reset(torch):
    plan = of.openfft_plan(8, 8, 8, 2, of.C2C_F64)
    s = torch.cuda.Stream()
    try:
        for h2d, d2h in ((s, None), (None, s)):
            with pytest.raises(of.OpenFFTError) as ei:
                of.openfft_set_copy_streams(plan, h2d, d2h)
            assert ei.value.status == of.ERR_INVALID_ARG
        x = synth.complex_field((8, 8, 8), seed=3).reshape(-1)
        want = _device(torch, plan, x, of.FORWARD)
        for streams in ((s, s), (None, None)):          # one stream for both; back to the plan's own
            of.openfft_set_copy_streams(plan, *streams)
            y = np.empty_like(x)
            of.openfft_exec_c2c_host(plan, x, y, of.FORWARD)
            assert np.array_equal(_bits(y), _bits(want))
    finally:
        of.openfft_destroy(plan)
