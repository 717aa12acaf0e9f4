"""Randomised properties of the oracle (shapes and P drawn by hypothesis).

Each property compares the oracle with a statement independent of it: the
Eq. 2-4 boxes must partition the index space in rank order, with slab or
pencil boundaries as Eqs. 2 and 8-9 say; every transpose must equal the
numpy axis permutation, with the count matrix of a searchsorted enumeration;
forward / backward 3-D transforms must equal numpy's fftn / ifftn (reordered);
real transforms must equal rfftn.
"""
import numpy as np
import pytest

import oracle
from tests.test_oracle import _count_matrix_numpy, _perm_target

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

SETTINGS = settings(max_examples=60, deadline=None, derandomize=True)


@st.composite
def shape_and_p(draw, max_dim=9, real=False):
    Na = draw(st.integers(1, max_dim))
    Nb = draw(st.integers(1, max_dim))
    Nc = draw(st.integers(1, max_dim))
    Ncx = Nc // 2 + 1 if real else Nc
    limit = min(Na * Nb, Ncx * Na, Ncx * Nb)
    P = draw(st.integers(1, limit))
    return Na, Nb, Nc, P


@SETTINGS
@given(st.integers(1, 12), st.integers(1, 12), st.integers(1, 12), st.data())
def test_boxes_partition_the_index_space(N1, N2, N3, data):
    P = data.draw(st.integers(1, N1 * N2))
    xs = [oracle.box(N1, N2, N3, P, r)[0] for r in range(P)]
    xe = [oracle.box(N1, N2, N3, P, r)[1] for r in range(P)]
    assert xs[0] == 0 and xe[-1] == N1 * N2 * N3 - 1
    for r in range(P - 1):
        assert xs[r + 1] == xe[r] + 1                       # contiguous, in rank order
    unit = N2 * N3 if P <= N1 else N3                       # slabs (Eq. 2) or pencils (Eqs. 8-9)
    assert all(x % unit == 0 for x in xs)
    assert oracle.degree(N1, N2, P) == (1 if P <= N1 else 2)


@SETTINGS
@given(shape_and_p(), st.sampled_from(["abc->cab", "cab->cba", "cba->cab", "cab->abc"]))
def test_transposes_are_axis_permutations(sp, which):
    Na, Nb, Nc, P = sp
    src = (np.arange(Na * Nb * Nc) + 0.5j * np.arange(Na * Nb * Nc)[::-1]).astype(np.complex128)
    dst, C = oracle.redistribute(Na, Nb, Nc, P, which, src)
    assert np.array_equal(dst, _perm_target(Na, Nb, Nc, which, src))
    assert np.array_equal(C, _count_matrix_numpy(Na, Nb, Nc, P, which))


@SETTINGS
@given(shape_and_p())
def test_fft3d_matches_numpy(sp):
    Na, Nb, Nc, P = sp
    rng = np.random.default_rng(Na * 100 + Nb * 10 + Nc + P)
    x = rng.standard_normal((Na, Nb, Nc)) + 1j * rng.standard_normal((Na, Nb, Nc))
    y = oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)
    assert oracle.rel_l2(y, oracle.abc_to_cba(np.fft.fftn(x))) < 1e-14
    z = oracle.fft3d(y, Na, Nb, Nc, P, oracle.BACKWARD)
    assert oracle.rel_l2(z, x.reshape(-1)) < 1e-14


@SETTINGS
@given(shape_and_p(real=True))
def test_rfft3d_matches_numpy(sp):
    Na, Nb, Nc, P = sp
    rng = np.random.default_rng(Na * 100 + Nb * 10 + Nc + P + 7)
    x = rng.standard_normal((Na, Nb, Nc))
    X = oracle.rfft3d(x, Na, Nb, Nc, P)
    assert oracle.rel_l2(X, np.transpose(np.fft.rfftn(x), (2, 1, 0)).reshape(-1)) < 1e-14
    back = oracle.rfft3d(X, Na, Nb, Nc, P, oracle.BACKWARD)
    assert np.linalg.norm(back - x.reshape(-1)) <= 1e-14 * max(1.0, np.linalg.norm(x))
