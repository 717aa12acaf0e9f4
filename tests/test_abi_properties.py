"""Randomised host-side checks of the library's closed-form decomposition.

Shapes and P are drawn by hypothesis over every legal combination: the
library's boxes, degrees and count matrices (closed forms in csrc/decomp.h)
must equal the oracle's literal enumeration bit for bit (Eqs. 2-9), and P
beyond the smallest leading-dimension product must be refused.  No GPU needed.
"""
import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

SETTINGS = settings(max_examples=80, deadline=None, derandomize=True)
ORDER_DIMS = {of.LAYOUT_ABC: lambda a, b, c: (a, b, c), of.LAYOUT_CAB: lambda a, b, c: (c, a, b),
              of.LAYOUT_CBA: lambda a, b, c: (c, b, a)}


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1501_07350_gb300 import _build
    _build.build()
    return of.load()


@st.composite
def shape_and_p(draw, max_dim=24):
    Na, Nb, Nc = (draw(st.integers(1, max_dim)) for _ in range(3))
    P = draw(st.integers(1, min(Na * Nb, Nc * Na, Nc * Nb)))
    return Na, Nb, Nc, P


@SETTINGS
@given(shape_and_p())
def test_boxes_and_degrees_equal_the_oracle(sp):
    Na, Nb, Nc, P = sp
    for layout, dims in ORDER_DIMS.items():
        D = dims(Na, Nb, Nc)
        assert of.openfft_decomp_degree(Na, Nb, Nc, P, layout) == oracle.degree(D[0], D[1], P)
        for r in range(P):
            s3, e3, off, cnt = of.openfft_decomp_box(Na, Nb, Nc, P, layout, r)
            xs, xe, os3, oe3 = oracle.box(D[0], D[1], D[2], P, r)
            assert (s3, e3, off, cnt) == (os3, oe3, xs, xe - xs + 1), (layout, r)


@SETTINGS
@given(shape_and_p(max_dim=12))
def test_count_matrices_equal_the_oracle(sp):
    Na, Nb, Nc, P = sp
    src = np.zeros(Na * Nb * Nc, complex)
    for which, code in [("abc->cab", 1), ("cab->cba", 2), ("cba->cab", -2), ("cab->abc", -1)]:
        _, C_ref = oracle.redistribute(Na, Nb, Nc, P, which, src)
        C = of.openfft_decomp_counts(Na, Nb, Nc, P, code)
        assert np.array_equal(C, C_ref), which
        assert C.sum() == Na * Nb * Nc                   # every element moves exactly once


@SETTINGS
@given(st.integers(1, 24), st.integers(1, 24), st.integers(1, 24), st.integers(1, 40))
def test_p_beyond_the_decomposition_is_refused(Na, Nb, Nc, extra):
    P = min(Na * Nb, Nc * Na, Nc * Nb) + extra
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_decomp_counts(Na, Nb, Nc, P, 1)
    assert ei.value.status == of.ERR_P_TOO_LARGE
