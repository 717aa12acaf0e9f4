"""Pins of the oracle's D-dimensional transform (oracle.fftnd and its steps).

The paper cites 4-D and 5-D transforms under the same decomposition (Sec. 1)
without their transpose orders; the reading taken generalises Sec. 2's
abc -> cab -> cba: ordering s of A[N_1]...[N_D] is
(d_D, ..., d_{D-s+2}, d_1, ..., d_{D-s+1}), each ordering decomposed by
Eqs. 2-9 with (N1, N2, N3) = (first dim, second dim, product of the rest).
Everything here is checked against references that do not use the oracle:
numpy's fftn / ifftn, a direct O(N^2) DFT, numpy axis permutations, and
Eq. 2 written out in numpy.
"""
import itertools

import numpy as np
import pytest

import oracle


def _order(D, s):
    """Axes (0 = d_1) of ordering s, slowest first."""
    return [D - 1 - i for i in range(s - 1)] + list(range(D - s + 1))


def _eq2_boundaries(L, P):
    """Eq. 2 for dims L of an ordering (N3 = product of the rest)."""
    N1, N2 = L[0], L[1]
    N3 = int(np.prod(L[2:]))
    if P <= N1:
        f = [(N1 * r // P) * N2 * N3 for r in range(P + 1)]
    else:
        f = [(N1 * N2 * r // P) * N3 for r in range(P + 1)]
    return np.array(f, dtype=np.int64)


def _field(shape, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(-1, 1, shape) + 1j * rng.uniform(-1, 1, shape)


# P up to min over the orderings of N1 N2 (Eq. 2 is undefined beyond); slabs
# and pencils occur in different orderings of the same transform
CASES = [((4, 3, 5, 2), 2), ((4, 3, 5, 2), 8), ((6, 4, 2, 3), 5), ((2, 3, 2, 2, 3), 2),
         ((2, 3, 2, 2, 3), 6), ((3, 4, 2, 2, 5), 7), ((8, 8, 4, 4), 16), ((5, 6, 7, 2), 10)]


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("dims,P", CASES)
def test_forward_and_backward_against_numpy(dims, P):
    D = len(dims)
    x = _field(dims, sum(dims) + P)
    y = oracle.fftnd(x, dims, P, oracle.FORWARD)
    want = np.transpose(np.fft.fftn(x), tuple(range(D - 1, -1, -1))).reshape(-1)
    assert _rel(y, want) < 1e-14
    # backward takes ordering D (reversed axes) and returns the array as given, / N
    z = oracle.fftnd(want, dims, P, oracle.BACKWARD)
    assert _rel(z, x.reshape(-1)) < 1e-14
    zb = oracle.fftnd(x.transpose(tuple(range(D - 1, -1, -1))).reshape(-1), dims, P, oracle.BACKWARD)
    assert _rel(zb, np.fft.ifftn(x).reshape(-1)) < 1e-14


@pytest.mark.parametrize("dims", [(2, 3, 2, 2), (3, 2, 2, 2, 2), (2, 2, 3, 1)])
def test_tiny_shapes_against_direct_dft(dims):
    D = len(dims)
    x = _field(dims, 5)
    N = x.size
    pts = list(itertools.product(*[range(n) for n in dims]))
    X = np.zeros(dims, dtype=complex)
    for k in pts:
        acc = 0j
        for v in pts:
            # exact phase: sum of (v_i k_i mod n_i) / n_i
            ph = sum(((vi * ki) % ni) / ni for vi, ki, ni in zip(v, k, dims))
            acc += x[v] * np.exp(-2j * np.pi * ph)
        X[k] = acc
    got = oracle.fftnd(x, dims, 2, oracle.FORWARD)
    assert _rel(got, np.transpose(X, tuple(range(D - 1, -1, -1))).reshape(-1)) < 1e-13
    assert N == len(pts)


def test_rank_counts_beyond_eq2_are_refused():
    with pytest.raises(ValueError):
        oracle.fftnd(_field((4, 3, 5, 2), 1), (4, 3, 5, 2), 9, oracle.FORWARD)


def test_three_dims_is_the_3d_transform():
    x = _field((6, 5, 4), 8)
    for P in (3, 12, 20):
        a = oracle.fftnd(x, (6, 5, 4), P, oracle.FORWARD)
        b = oracle.fft3d(x, 6, 5, 4, P, oracle.FORWARD)
        assert np.array_equal(a.view(np.uint64), b.view(np.uint64))


def test_delta_and_plane_wave():
    dims = (4, 6, 3, 5)
    D = len(dims)
    N = int(np.prod(dims))
    x = np.zeros(dims, complex)
    x[0, 0, 0, 0] = 1.0
    assert np.allclose(oracle.fftnd(x, dims, 5, oracle.FORWARD), 1.0, atol=0, rtol=1e-15)
    k0 = (1, 4, 2, 3)
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    ph = sum(((g * k) % n) / n for g, k, n in zip(grids, k0, dims))
    pw = np.exp(2j * np.pi * ph)
    y = oracle.fftnd(pw, dims, 7, oracle.FORWARD).reshape(tuple(reversed(dims)))
    exact = np.zeros(tuple(reversed(dims)), complex)
    exact[tuple(reversed(k0))] = N
    assert np.linalg.norm(y - exact) / (N * np.sqrt(N)) < 1e-14


@pytest.mark.parametrize("dims,P", CASES)
def test_boundaries_are_eq2(dims, P):
    D = len(dims)
    for s in range(1, D + 1):
        L = [dims[a] for a in _order(D, s)]
        assert np.array_equal(oracle.nd_boundaries(dims, P, s), _eq2_boundaries(L, P)), s


@pytest.mark.parametrize("dims,P", CASES)
def test_transposes_are_axis_permutations_with_their_counts(dims, P):
    D = len(dims)
    N = int(np.prod(dims))
    src = _field((N,), N + 3 * P)
    for s in range(1, D):
        for forward in (True, False):
            a, b = (s, s + 1) if forward else (s + 1, s)
            oa, ob = _order(D, a), _order(D, b)
            # the array in ordering a, as an array indexed by original axes
            A = src.reshape([dims[i] for i in oa])
            perm = [oa.index(i) for i in ob]               # axes of ordering b in A
            want = np.ascontiguousarray(np.transpose(A, perm)).reshape(-1)
            got, C = oracle.nd_redistribute(dims, P, s, forward, src)
            assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (s, forward)
            # counts: element at position x of ordering a goes to position y of ordering b
            xa = np.arange(N).reshape([dims[i] for i in oa])
            yb = np.empty(N, np.int64)
            yb[np.transpose(xa, perm).reshape(-1)] = np.arange(N)
            ba = _eq2_boundaries([dims[i] for i in oa], P)
            bb = _eq2_boundaries([dims[i] for i in ob], P)
            r_of = np.searchsorted(ba, np.arange(N), side="right") - 1
            s_of = np.searchsorted(bb, yb, side="right") - 1
            want_C = np.zeros((P, P), np.int64)
            np.add.at(want_C, (r_of, s_of), 1)
            assert np.array_equal(C, want_C), (s, forward)
