"""Host-only queries of the D-dimensional decomposition (no GPU): the
library's closed-form boxes and its count matrices against the oracle's
literal Eq. 2-4 boundaries and redistribution, bit-exact."""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of

CASES = [((4, 3, 5, 2), 2), ((4, 3, 5, 2), 8), ((6, 4, 2, 3), 5), ((2, 3, 2, 2, 3), 6), ((3, 4, 2, 2, 5), 7),
         ((8, 8, 4, 4), 16), ((5, 6, 7, 2), 10), ((6, 5, 4), 20)]


@pytest.fixture(scope="module")
def lib():
    from paper_1501_07350_gb300 import _build
    _build.build()
    oracle.build()
    return of.load()


@pytest.mark.parametrize("dims,P", CASES)
def test_boxes_and_counts_match_the_oracle(lib, dims, P):
    D = len(dims)
    N = int(np.prod(dims))
    for s in range(1, D + 1):
        xs = oracle.nd_boundaries(dims, P, s)
        for r in range(P):
            assert of.openfft_nd_decomp_box(dims, P, s, r) == (xs[r], xs[r + 1] - xs[r])
    x = np.arange(N).astype(np.complex128)
    for s in range(1, D):
        for e in (s, -s):
            _, C = oracle.nd_redistribute(dims, P, s, e > 0, x)
            assert np.array_equal(of.openfft_nd_decomp_counts(dims, P, e), C), e


def test_refusals(lib):
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_nd_decomp_box((4, 3, 5, 2), 9, 1, 0)
    assert ei.value.status == of.ERR_P_TOO_LARGE
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_nd_decomp_box((4, 3), 2, 1, 0)
    assert ei.value.status == of.ERR_INVALID_ARG
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_nd_decomp_counts((4, 3, 5, 2), 4, 4)
    assert ei.value.status == of.ERR_INVALID_ARG
