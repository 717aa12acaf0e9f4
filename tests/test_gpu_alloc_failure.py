"""Out-of-memory handling, by host-side injection (no real exhaustion).

openfft_debug_alloc_fail(k) makes the k-th device allocation of the library
fail as cudaMalloc does when the device is full.  For every k up to the
number of allocations a plan makes, creating the plan must return
OPENFFT_ERR_NOMEM and free everything it had allocated (the device's free
memory is back where it was), and afterwards the same plan must build and
compute correctly.  The same for the batched and distributed plans and for
the host-buffer staging that a plan allocates on its first host-buffer call.
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


def _free(torch):
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _sweep(torch, make, destroy, max_k=64):
    """Fail the k-th allocation for k = 1, 2, ... until `make` succeeds."""
    h = make()                      # warm: kernels loaded, caches filled
    destroy(h)
    free0 = _free(torch)
    for k in range(1, max_k + 1):
        of.openfft_debug_alloc_fail(k)
        try:
            h = make()
        except of.OpenFFTError as e:
            assert e.status == of.ERR_NOMEM, (k, e)
            assert _free(torch) == free0, ("leak after failing allocation", k)
            continue
        finally:
            of.openfft_debug_alloc_fail(0)
        destroy(h)
        assert _free(torch) == free0
        return k - 1                # allocations the call makes
    raise AssertionError("more than %d allocations" % max_k)


def test_plan_creation_failures_free_everything(torch):
    Na, Nb, Nc, P = 24, 20, 30, 6
    for dtype in (of.C2C_F64, of.C2C_F32, of.C2C_SPLIT_TF32):
        n = _sweep(torch, lambda: of.openfft_plan(Na, Nb, Nc, P, dtype), of.openfft_destroy)
        assert n >= 10, n                    # workspace, twiddles, transpose tables, status word
    # a plan built afterwards computes correctly
    x = synth.complex_field((Na, Nb, Nc), seed=3)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        xd = torch.from_numpy(x.reshape(-1)).cuda()
        yd = torch.empty_like(xd)
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        of.openfft_exec_c2c(plan, xd, yd, of.FORWARD)
        of.openfft_sync(plan)
        assert oracle.rel_l2(yd.cpu().numpy(), oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)) < 1e-12
    finally:
        of.openfft_destroy(plan)


def test_batched_and_distributed_plan_failures(torch):
    shapes, Ps = [(16, 12, 10), (8, 8, 8)], [4, 2]
    _sweep(torch, lambda: of.openfft_plan_many(shapes, Ps, of.C2C_F32), of.openfft_destroy)
    _sweep(torch, lambda: of.openfft_dist_plan(16, 12, 10, 8, 2, 1, of.C2C_F64), of.openfft_dist_destroy)


def test_host_staging_failure_then_success(torch):
    Na, Nb, Nc, P = 16, 12, 10, 4
    x = synth.complex_field((Na * Nb * Nc,), seed=9)
    y = np.empty_like(x)
    plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
    try:
        for k in (1, 2):                      # the two staging arrays
            of.openfft_debug_alloc_fail(k)
            try:
                with pytest.raises(of.OpenFFTError) as ei:
                    of.openfft_exec_c2c_host(plan, x, y, of.FORWARD)
                assert ei.value.status == of.ERR_NOMEM
            finally:
                of.openfft_debug_alloc_fail(0)
        of.openfft_exec_c2c_host(plan, x, y, of.FORWARD)
        assert oracle.rel_l2(y, oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)) < 1e-12
    finally:
        of.openfft_destroy(plan)


def test_control_rejects_negative(torch):
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_debug_alloc_fail(-1)
    assert ei.value.status == of.ERR_INVALID_ARG
