"""Pins of the FP64 oracle against things other than itself.

Each test ties one oracle function to the paper (hand-worked values of Eqs.
2-7, the degree switch of Sec. 4.1), to the mathematics (brute-force DFT,
closed forms, Parseval, linearity, the inverse), or to an independent library
routine (numpy.fft, numpy transposes).  A dropped term, a wrong sign, a wrong
index or a transposed operand in the oracle fails at least one of them.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if line and not line.startswith("#"):
                yield [int(t) for t in line.split()]


# ----------------------------------------------------------- Eqs. 2-9 --

def test_boxes_match_hand_worked_eq2_to_eq7():
    for N1, N2, N3, Np, myid, xs, xe, a_s, b_s, c_s, a_e, b_e, c_e in _rows("eq2_to_eq7_boxes_4x3x2.txt"):
        got = oracle.box(N1, N2, N3, Np, myid)
        assert got == (xs, xe, (a_s, b_s, c_s), (a_e, b_e, c_e))


def test_degree_switch_at_256_cubed():
    for N1, N2, Np, deg in _rows("sec4_degree_switch_256.txt"):
        assert oracle.degree(N1, N2, Np) == deg


def test_f_undefined_beyond_n1n2():
    assert oracle.f(4, 3, 2, 12, 5) >= 0
    assert oracle.f(4, 3, 2, 13, 5) == -1


@pytest.mark.parametrize("N1,N2,N3", [(4, 3, 2), (7, 5, 3), (16, 9, 4), (1, 6, 5)])
def test_boxes_tile_the_array(N1, N2, N3):
    """Boxes are disjoint, ascending, cover [0, N) and hold whole rows of N3."""
    for Np in range(1, N1 * N2 + 1):
        xs = oracle.boundaries(N1, N2, N3, Np)
        assert xs[0] == 0 and xs[-1] == N1 * N2 * N3
        assert np.all(np.diff(xs) >= 0)
        assert np.all(xs % N3 == 0)
        if Np <= N1:
            assert np.all(xs % (N2 * N3) == 0)      # slabs: whole ab-planes... of the ordering
            assert np.all(np.diff(xs) > 0)


# ------------------------------------------------------------- 1-D FFT --

@pytest.mark.parametrize("n", list(range(1, 65)) + [96, 100, 108, 120, 144, 160, 256, 512, 49, 77])
def test_fft1d_matches_brute_force_dft(n):
    x = synth.complex_field((n,), seed=1000 + n)
    for sign in (-1, 1):
        y = oracle.fft1d(x, sign)
        assert oracle.rel_l2(y, oracle.dft1d_brute(x, sign)) < 1e-14


def test_brute_dft1d_matches_numpy():
    for n in (1, 2, 3, 7, 16, 30):
        x = synth.complex_field((n,), seed=7 + n)
        assert oracle.rel_l2(oracle.dft1d_brute(x, -1), np.fft.fft(x)) < 1e-14
        assert oracle.rel_l2(oracle.dft1d_brute(x, 1), np.fft.ifft(x) * n) < 1e-14


def test_fft1d_delta_and_constant():
    n = 60
    d = np.zeros(n, complex)
    d[0] = 1.0
    assert np.max(np.abs(oracle.fft1d(d) - 1.0)) < 1e-15
    assert abs(oracle.fft1d(np.ones(n))[0] - n) < 1e-12
    assert np.max(np.abs(oracle.fft1d(np.ones(n))[1:])) < 1e-12


# ------------------------------------------------------ 3-D brute force --

def test_dft3d_brute_matches_numpy():
    for shape in [(2, 3, 5), (4, 1, 6), (3, 3, 3)]:
        A = synth.complex_field(shape, seed=11)
        assert oracle.rel_l2(oracle.dft3d_brute(A, -1), np.fft.fftn(A)) < 1e-14
        assert oracle.rel_l2(oracle.dft3d_brute(A, 1), np.fft.ifftn(A) * A.size) < 1e-14


def _valid_ps(Na, Nb, Nc):
    pmax = min(Na * Nb, Nc * Na, Nc * Nb)
    return sorted({1, 2, 3, max(1, pmax // 2), pmax} & set(range(1, pmax + 1)))


SMALL_DIMS = (1, 2, 3, 4, 5, 6, 8)


@pytest.mark.parametrize("Na", SMALL_DIMS)
def test_fft3d_matches_brute_force_on_small_shapes(Na):
    for Nb, Nc in itertools.product(SMALL_DIMS, SMALL_DIMS):
        A = synth.complex_field((Na, Nb, Nc), seed=Na * 100 + Nb * 10 + Nc)
        ref = oracle.abc_to_cba(oracle.dft3d_brute(A, -1))
        for P in _valid_ps(Na, Nb, Nc):
            got = oracle.fft3d(A, Na, Nb, Nc, P, -1)
            assert oracle.rel_l2(got, ref) < 1e-14, (Na, Nb, Nc, P)


@pytest.mark.parametrize("shape", [(2, 3, 5), (4, 6, 5), (8, 3, 5), (5, 4, 3)])
def test_fft3d_backward_matches_brute_force(shape):
    Na, Nb, Nc = shape
    X = synth.complex_field(shape, seed=99)      # spectrum in [ka][kb][kc]
    ref = oracle.dft3d_brute(X, 1).reshape(-1) / X.size
    for P in _valid_ps(Na, Nb, Nc):
        got = oracle.fft3d(oracle.abc_to_cba(X), Na, Nb, Nc, P, 1)
        assert oracle.rel_l2(got, ref) < 1e-14


def test_dft3d_line_matches_brute_force():
    A = synth.complex_field((6, 5, 4), seed=5)
    X = oracle.dft3d_brute(A, -1)
    for kb, kc in [(0, 0), (2, 3), (4, 1)]:
        assert oracle.rel_l2(oracle.dft3d_line(A, kb, kc, -1), X[:, kb, kc]) < 1e-14
    Xi = oracle.dft3d_brute(A, 1)
    assert oracle.rel_l2(oracle.dft3d_line(A, 3, 2, 1), Xi[:, 3, 2]) < 1e-14


# --------------------------------------------------------- closed forms --

SHAPES = [(8, 6, 10), (12, 10, 9), (16, 16, 16)]


@pytest.mark.parametrize("shape", SHAPES)
def test_delta_at_origin_gives_ones(shape):
    Na, Nb, Nc = shape
    A = np.zeros(shape, complex)
    A[0, 0, 0] = 1.0
    y = oracle.fft3d(A, Na, Nb, Nc, 4, -1)
    assert np.max(np.abs(y - 1.0)) < 1e-15


@pytest.mark.parametrize("shape", SHAPES)
def test_shifted_delta_gives_plane_wave(shape):
    Na, Nb, Nc = shape
    a0, b0, c0 = 3, 5, 7
    A = np.zeros(shape, complex)
    A[a0 % Na, b0 % Nb, c0 % Nc] = 1.0
    y = oracle.fft3d(A, Na, Nb, Nc, 3, -1)
    # X[ka,kb,kc] = exp(-2 pi i (a0 ka/Na + b0 kb/Nb + c0 kc/Nc)) = conj(plane wave at k0=(a0,b0,c0))
    exact = np.conj(synth.plane_wave(Na, Nb, Nc, (a0 % Na, b0 % Nb, c0 % Nc)))
    assert np.max(np.abs(y - oracle.abc_to_cba(exact))) < 1e-14


@pytest.mark.parametrize("k0", [(0, 0, 0), (1, 2, 3), (11, 9, 8)])
def test_plane_wave_gives_single_bin(k0):
    Na, Nb, Nc = 12, 10, 9
    N = Na * Nb * Nc
    A = synth.plane_wave(Na, Nb, Nc, k0)
    y = oracle.fft3d(A, Na, Nb, Nc, 8, -1)
    exact = np.zeros((Na, Nb, Nc), complex)
    exact[k0] = N
    err = np.linalg.norm(y - oracle.abc_to_cba(exact)) / (N * np.sqrt(N))
    assert err < 1e-15


def test_parseval_and_linearity():
    Na, Nb, Nc = 12, 10, 16
    x = synth.complex_field((Na, Nb, Nc), seed=3)
    z = synth.complex_field((Na, Nb, Nc), seed=4)
    X = oracle.fft3d(x, Na, Nb, Nc, 6, -1)
    Z = oracle.fft3d(z, Na, Nb, Nc, 6, -1)
    N = x.size
    e_x = np.sum(np.abs(x) ** 2)
    assert abs(np.sum(np.abs(X) ** 2) - N * e_x) / (N * e_x) < 1e-13
    al, be = 0.7 - 0.2j, -1.3 + 0.5j
    XZ = oracle.fft3d(al * x + be * z, Na, Nb, Nc, 6, -1)
    assert oracle.rel_l2(XZ, al * X + be * Z) < 1e-14


@pytest.mark.parametrize("shape,P", [((16, 16, 16), 4), ((12, 10, 9), 30), ((8, 6, 10), 48)])
def test_round_trip_is_identity(shape, P):
    Na, Nb, Nc = shape
    x = synth.complex_field(shape, seed=8)
    X = oracle.fft3d(x, Na, Nb, Nc, P, -1)
    back = oracle.fft3d(X, Na, Nb, Nc, P, 1)
    assert oracle.rel_l2(back, x.reshape(-1)) < 1e-14


def test_fft3d_matches_numpy_fftn_medium():
    Na, Nb, Nc = 20, 18, 15
    x = synth.complex_field((Na, Nb, Nc), seed=21, dist="normal")
    y = oracle.fft3d(x, Na, Nb, Nc, 7, -1)
    assert oracle.rel_l2(y, oracle.abc_to_cba(np.fft.fftn(x))) < 1e-14


# -------------------------------------------------------- redistribution --

def _perm_target(Na, Nb, Nc, which, src):
    """Independent statement of each transpose with numpy axis permutations."""
    if which == "abc->cab":
        return np.transpose(src.reshape(Na, Nb, Nc), (2, 0, 1)).reshape(-1)
    if which == "cab->cba":
        return np.transpose(src.reshape(Nc, Na, Nb), (0, 2, 1)).reshape(-1)
    if which == "cba->cab":
        return np.transpose(src.reshape(Nc, Nb, Na), (0, 2, 1)).reshape(-1)
    if which == "cab->abc":
        return np.transpose(src.reshape(Nc, Na, Nb), (1, 2, 0)).reshape(-1)
    raise ValueError(which)


_DIMS_OF = {"abc": lambda n: (n[0], n[1], n[2]), "cab": lambda n: (n[2], n[0], n[1]),
            "cba": lambda n: (n[2], n[1], n[0])}


def _count_matrix_numpy(Na, Nb, Nc, P, which):
    """Count matrix by numpy: owners via searchsorted on Eq. 2 boundaries."""
    src_l, dst_l = which.split("->")
    n = (Na, Nb, Nc)
    D_s, D_d = _DIMS_OF[src_l](n), _DIMS_OF[dst_l](n)
    xs_s = np.array([oracle.f(*D_s, P, i) for i in range(P + 1)])
    xs_d = np.array([oracle.f(*D_d, P, i) for i in range(P + 1)])
    N = Na * Nb * Nc
    dest_of_src = _perm_target(Na, Nb, Nc, which, np.arange(N))  # value at dst pos = src index
    inv = np.empty(N, dtype=np.int64)
    inv[dest_of_src] = np.arange(N)                                  # src index -> dst pos
    own_s = np.searchsorted(xs_s, np.arange(N), side="right") - 1
    own_d = np.searchsorted(xs_d, inv, side="right") - 1
    C = np.zeros((P, P), dtype=np.int64)
    np.add.at(C, (own_s, own_d), 1)
    return C


REDIST_CASES = [((4, 3, 2), 3), ((4, 3, 2), 6), ((8, 6, 10), 5), ((8, 6, 10), 40), ((12, 10, 9), 30),
                ((5, 7, 3), 15), ((16, 16, 16), 16), ((6, 4, 8), 24)]


@pytest.mark.parametrize("shape,P", REDIST_CASES)
@pytest.mark.parametrize("which", ["abc->cab", "cab->cba", "cba->cab", "cab->abc"])
def test_redistribution_is_the_axis_permutation(shape, P, which):
    Na, Nb, Nc = shape
    src = (np.arange(Na * Nb * Nc) + 1j * np.arange(Na * Nb * Nc)[::-1]).astype(np.complex128)
    dst, C = oracle.redistribute(Na, Nb, Nc, P, which, src)
    assert np.array_equal(dst, _perm_target(Na, Nb, Nc, which, src))
    assert np.array_equal(C, _count_matrix_numpy(Na, Nb, Nc, P, which))


@pytest.mark.parametrize("shape,P", [((16, 16, 16), 4), ((12, 10, 9), 3), ((32, 32, 32), 8), ((20, 6, 10), 5)])
def test_count_matrix_closed_form_slabs(shape, P):
    """1-D slabs everywhere (P <= Na, Nc): C1[r][s] = nA(r)*Nb*nC(s); C2 diagonal."""
    Na, Nb, Nc = shape
    x = np.zeros(shape, complex)
    _, C1, C2 = oracle.fft3d(x, Na, Nb, Nc, P, -1, counts=True)
    nA = np.diff([(Na * r) // P for r in range(P + 1)])
    nC = np.diff([(Nc * s) // P for s in range(P + 1)])
    assert np.array_equal(C1, np.outer(nA, nC) * Nb)
    assert np.array_equal(C2, np.diag(np.diag(C2)))
    assert np.array_equal(np.diag(C2), nC * Na * Nb)
    N = Na * Nb * Nc
    if Na % P == 0 and Nc % P == 0:
        assert C1.sum() - np.trace(C1) == N - N // P      # sent volume N(1 - 1/P)


def test_count_matrix_2d_cab_to_cba_half_local():
    """In 2-D (P = 2*Nc), each cab pencil of rank r overlaps the cba pencil of the
    same rank by half of its elements (transpose-order awareness, Sec. 2)."""
    Na = Nb = Nc = 8
    P = 16
    x = np.zeros((Na, Nb, Nc), complex)
    _, C1, C2 = oracle.fft3d(x, Na, Nb, Nc, P, -1, counts=True)
    box = Na * Nb * Nc // P
    assert np.all(np.diag(C2) == box // 2)
    assert C2.sum() == Na * Nb * Nc


# ------------------------------------------------- real transforms (R2C) --
# The half spectrum kc <= Nc/2 of a real input, with the complex stages
# decomposed over (Na, Nb, Nc//2 + 1).  Pinned to numpy's rfftn / irfftn (the
# special case of a library routine), to brute-force DFTs on tiny shapes, to
# the complex oracle and to the round trip.

R2C_SHAPES = [((4, 6, 8), 3), ((5, 3, 7), 2), ((8, 8, 8), 8), ((6, 5, 4), 5), ((3, 10, 9), 15),
              ((16, 12, 10), 48), ((7, 7, 2), 14), ((2, 3, 1), 2)]


def _half_cba(X_abc_half):
    """[Na][Nb][Nch] -> flat cba-half order (index (kc*Nb + kb)*Na + ka)."""
    return np.ascontiguousarray(np.transpose(X_abc_half, (2, 1, 0))).reshape(-1)


@pytest.mark.parametrize("shape,P", R2C_SHAPES)
def test_rfft3d_matches_numpy_rfftn(shape, P):
    Na, Nb, Nc = shape
    x = synth.uniform_pm1(synth.config_seed(11) + Na * Nb * Nc, Na * Nb * Nc).reshape(shape)
    X = oracle.rfft3d(x, Na, Nb, Nc, P)
    assert X.size == Na * Nb * (Nc // 2 + 1)
    assert oracle.rel_l2(X, _half_cba(np.fft.rfftn(x))) < 1e-14


@pytest.mark.parametrize("shape,P", R2C_SHAPES)
def test_irfft3d_matches_numpy_irfftn_on_any_half_spectrum(shape, P):
    """Inverse of an arbitrary (not Hermitian-consistent) half spectrum: the real
    part of the inverse DFT of its Hermitian extension along c, which drops the
    imaginary parts of kc = 0 and (even Nc) kc = Nc/2: numpy's convention."""
    Na, Nb, Nc = shape
    Nch = Nc // 2 + 1
    H = synth.complex_field((Nch, Nb, Na), seed=synth.config_seed(12) + Nc).reshape(-1)
    x = oracle.rfft3d(H, Na, Nb, Nc, P, oracle.BACKWARD)
    ref = np.fft.irfftn(np.transpose(H.reshape(Nch, Nb, Na), (2, 1, 0)), s=(Na, Nb, Nc), axes=(0, 1, 2))
    assert np.linalg.norm(x - ref.reshape(-1)) <= 1e-14 * np.linalg.norm(ref)


@pytest.mark.parametrize("shape", [(2, 3, 4), (3, 2, 5), (4, 4, 1), (1, 5, 6), (3, 3, 3)])
def test_rfft3d_brute_force(shape):
    Na, Nb, Nc = shape
    x = synth.uniform_pm1(synth.config_seed(13), Na * Nb * Nc).reshape(shape)
    full = oracle.dft3d_brute(x.astype(np.complex128), oracle.FORWARD).reshape(shape)
    for P in (1, 2, min(Na * Nb, (Nc // 2 + 1) * min(Na, Nb))):
        X = oracle.rfft3d(x, Na, Nb, Nc, P)
        assert oracle.rel_l2(X, _half_cba(full[:, :, : Nc // 2 + 1])) < 1e-14


@pytest.mark.parametrize("shape,P", R2C_SHAPES[:5])
def test_rfft3d_is_the_half_of_the_complex_transform(shape, P):
    Na, Nb, Nc = shape
    x = synth.uniform_pm1(synth.config_seed(14), Na * Nb * Nc).reshape(shape)
    Y = oracle.fft3d(x.astype(np.complex128), Na, Nb, Nc, min(P, Nc * min(Na, Nb)), oracle.FORWARD)
    Y = Y.reshape(Nc, Nb, Na)[: Nc // 2 + 1].reshape(-1)
    assert oracle.rel_l2(oracle.rfft3d(x, Na, Nb, Nc, P), Y) < 1e-14


@pytest.mark.parametrize("shape,P", R2C_SHAPES)
def test_rfft3d_round_trip_and_hermitian_columns(shape, P):
    Na, Nb, Nc = shape
    x = synth.normal(synth.config_seed(15), Na * Nb * Nc).reshape(shape)
    X = oracle.rfft3d(x, Na, Nb, Nc, P)
    back = oracle.rfft3d(X, Na, Nb, Nc, P, oracle.BACKWARD)
    assert np.linalg.norm(back - x.reshape(-1)) <= 1e-14 * np.linalg.norm(x)
    # kc = 0 (and kc = Nc/2 for even Nc) is the 2-D DFT of a real array: Hermitian in (ka, kb)
    Xh = X.reshape(Nc // 2 + 1, Nb, Na)
    for kc in ([0, Nc // 2] if Nc % 2 == 0 else [0]):
        col = Xh[kc]
        mirror = np.conj(col[(-np.arange(Nb))[:, None] % Nb, (-np.arange(Na))[None, :] % Na])
        assert np.max(np.abs(col - mirror)) <= 1e-13 * max(1.0, np.max(np.abs(col)))


def test_rfft3d_counts_are_those_of_the_half_array():
    Na, Nb, Nc, P = 12, 10, 16, 6
    x = synth.uniform_pm1(synth.config_seed(16), Na * Nb * Nc)
    _, C1, C2 = oracle.rfft3d(x, Na, Nb, Nc, P, counts=True)
    _, D1, D2 = oracle.fft3d(np.zeros(Na * Nb * (Nc // 2 + 1), complex), Na, Nb, Nc // 2 + 1, P,
                             oracle.FORWARD, counts=True)
    assert np.array_equal(C1, D1) and np.array_equal(C2, D2)
    assert C1.sum() == C2.sum() == Na * Nb * (Nc // 2 + 1)


def test_rfft3d_rejects_p_beyond_the_half_orderings():
    with pytest.raises(ValueError):
        oracle.rfft3d(np.zeros(3 * 4 * 5), 3, 4, 5, 12)       # cab-half (3, 3, 4): 9 < 12
