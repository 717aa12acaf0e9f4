"""Split-precision tensor-core GEMM (tcgen05) against an FP64 product.

D = A B^T with operands split into a tf32 / bf16 high part and the rounded
remainder: the split result must be close to FP32 accuracy, and clearly more
accurate than the high parts alone (so that the low-part products are really
accumulated)."""
import numpy as np
import pytest

from paper_1501_07350_gb300 import openfft as of
from paper_1501_07350_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_1501_07350_gb300 import _build
    _build.build()
    return of.load()


def _err(D, ref):
    return float(np.max(np.abs(D - ref)) / np.max(np.abs(ref)))


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 32, 32), (300, 64, 64), (128, 48, 48)])
def test_tc_gemm_tf32(lib, M, N, K):
    A = synth.uniform_pm1(M * 10 + N, M * K).reshape(M, K).astype(np.float32)
    B = synth.uniform_pm1(N * 10 + K, N * K).reshape(N, K).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    e_split = _err(of.openfft_tc_gemm(A, B, tf32=True, split=True), ref)
    e_hi = _err(of.openfft_tc_gemm(A, B, tf32=True, split=False), ref)
    assert e_split < 2e-6, e_split
    assert 1e-5 < e_hi < 5e-3, e_hi


@pytest.mark.parametrize("M,N,K", [(128, 16, 16), (256, 32, 32), (300, 64, 64)])
def test_tc_gemm_bf16(lib, M, N, K):
    A = synth.uniform_pm1(M * 7 + N, M * K).reshape(M, K).astype(np.float32)
    B = synth.uniform_pm1(N * 7 + K, N * K).reshape(N, K).astype(np.float32)
    ref = A.astype(np.float64) @ B.astype(np.float64).T
    e_split = _err(of.openfft_tc_gemm(A, B, tf32=False, split=True), ref)
    e_hi = _err(of.openfft_tc_gemm(A, B, tf32=False, split=False), ref)
    assert e_split < 1e-4, e_split
    assert 1e-4 < e_hi < 5e-2, e_hi
