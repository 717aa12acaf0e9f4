"""Host-side checks of the C ABI (no GPU needed).

- the shared library loads and exports every function include/openfft_gb.h
  declares;
- the closed-form decomposition of the library (boxes, degrees, count
  matrices) equals the oracle's literal enumeration bit for bit;
- argument errors are reported with the documented status codes.
"""
import ctypes
import itertools
import os
import re

import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import openfft as of

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1501_07350_gb300 import _build
    _build.build()
    return of.load()


def _declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for fn in os.listdir(inc):
        if fn.endswith(".h"):
            text = open(os.path.join(inc, fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(openfft_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported():
    declared = _declared_functions()
    assert declared, "no declarations found"
    lib = ctypes.CDLL(of.library_path())
    for name in sorted(declared):
        assert hasattr(lib, name), name
    assert declared == set(of.EXPORTS)


def test_checked_build_compiles_and_exports_the_same_abi():
    """The bounds-checked library (-DOPENFFT_CHECKED) builds for sm_103a,
    exports every declared function and says which build it is; the normal
    one refuses the bounds-status query.  Neither call touches a GPU."""
    from paper_1501_07350_gb300 import _build
    path = _build.build(checked=True)
    chk = ctypes.CDLL(path)
    for name in sorted(_declared_functions()):
        assert hasattr(chk, name), name
    assert chk.openfft_checked_build() == 1
    assert not of.openfft_checked_build()
    with pytest.raises(of.OpenFFTError) as e:
        of.openfft_debug_bounds_status()
    assert e.value.status == of.ERR_UNSUPPORTED


ORDER_DIMS = {of.LAYOUT_ABC: lambda a, b, c: (a, b, c), of.LAYOUT_CAB: lambda a, b, c: (c, a, b),
              of.LAYOUT_CBA: lambda a, b, c: (c, b, a)}

SHAPES = [(4, 3, 2), (8, 6, 10), (12, 10, 9), (32, 32, 32), (120, 144, 160), (5, 7, 3), (1, 6, 4),
          (100, 108, 120), (256, 256, 256), (512, 512, 512)]


def _ps(shape):
    Na, Nb, Nc = shape
    pmax = min(Na * Nb, Nc * Na, Nc * Nb)
    cand = {1, 2, 3, 4, 5, 7, 8, 16, 32, 33, 64, 100, 128, 256, 512, 1024, pmax, max(1, pmax - 1)}
    return sorted(p for p in cand if 1 <= p <= pmax and p <= 1024)


@pytest.mark.parametrize("shape", SHAPES)
def test_boxes_and_degree_match_oracle(shape):
    Na, Nb, Nc = shape
    for P in _ps(shape):
        for layout, dims in ORDER_DIMS.items():
            D = dims(Na, Nb, Nc)
            assert of.openfft_decomp_degree(Na, Nb, Nc, P, layout) == oracle.degree(D[0], D[1], P)
            ranks = range(P) if P <= 64 else list(range(0, P, max(1, P // 37))) + [P - 1]
            for r in ranks:
                s3, e3, off, cnt = of.openfft_decomp_box(Na, Nb, Nc, P, layout, r)
                xs, xe, os3, oe3 = oracle.box(D[0], D[1], D[2], P, r)
                assert (s3, e3, off, cnt) == (os3, oe3, xs, xe - xs + 1)


COUNT_CASES = [((4, 3, 2), 3), ((4, 3, 2), 6), ((8, 6, 10), 5), ((8, 6, 10), 40), ((12, 10, 9), 30),
               ((5, 7, 3), 15), ((16, 16, 16), 16), ((6, 4, 8), 24), ((16, 16, 16), 64), ((8, 8, 8), 16),
               ((12, 10, 16), 100), ((20, 18, 15), 7), ((7, 1, 5), 5)]


@pytest.mark.parametrize("shape,P", COUNT_CASES)
def test_count_matrices_match_oracle_enumeration(shape, P):
    Na, Nb, Nc = shape
    src = np.zeros(Na * Nb * Nc, complex)
    for which, code in [("abc->cab", 1), ("cab->cba", 2), ("cba->cab", -2), ("cab->abc", -1)]:
        _, C_ref = oracle.redistribute(Na, Nb, Nc, P, which, src)
        assert np.array_equal(of.openfft_decomp_counts(Na, Nb, Nc, P, code), C_ref), which


def test_count_matrix_256_cubed_slabs_closed_form():
    """Sec. 4.1 at 256^3: slabs up to P = 256; the total volume sent by R1 is N(1 - 1/P)."""
    N = 256 ** 3
    for P in (16, 64, 256):
        C1 = of.openfft_decomp_counts(256, 256, 256, P, 1)
        assert C1.sum() == N
        assert C1.sum() - np.trace(C1) == N - N // P
        C2 = of.openfft_decomp_counts(256, 256, 256, P, 2)
        assert np.array_equal(C2, np.diag(np.diag(C2)))            # cab -> cba stays local
    C2 = of.openfft_decomp_counts(256, 256, 256, 512, 2)
    assert np.all(np.diag(C2) == N // 512 // 2)                     # pencils: half local


def test_count_matrix_512_cubed_p1024_half_local():
    C2 = of.openfft_decomp_counts(512, 512, 512, 1024, 2)
    box = 512 ** 3 // 1024
    assert np.all(np.diag(C2) == box // 2)
    assert C2.sum() == 512 ** 3


def test_errors_are_reported():
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_decomp_counts(4, 3, 2, 13, 1)
    assert ei.value.status == of.ERR_P_TOO_LARGE
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_decomp_box(0, 3, 2, 1, 0, 0)
    assert ei.value.status == of.ERR_INVALID_ARG
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_decomp_counts(4, 3, 2, 2, 3)
    assert ei.value.status == of.ERR_INVALID_ARG
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_decomp_box(4, 3, 2, 2, 0, 2)
    assert ei.value.status == of.ERR_INVALID_ARG
    assert of.openfft_decomp_degree(4, 3, 2, 13, 0) == -1
    # P_TOO_LARGE uses the smallest leading product over the three orderings
    with pytest.raises(of.OpenFFTError) as ei:
        of.openfft_decomp_counts(8, 8, 1, 9, 1)      # cab / cba lead with Nc*Na = 8
    assert ei.value.status == of.ERR_P_TOO_LARGE


def test_null_plan_is_rejected():
    lib = of.load()
    assert lib.openfft_exec_c2c(None, None, None, -1) == of.ERR_INVALID_ARG
    assert lib.openfft_set_tuning(None, 0, 0) == of.ERR_INVALID_ARG
    lib.openfft_destroy(None)      # NULL-safe


def test_committed_learned_data_is_consistent():
    """The committed timing dataset covers the held-out benchmark problems and the
    committed cost model has the library's feature count."""
    import json
    from paper_1501_07350_gb300 import learned
    rows = learned.load_rows()
    train_rows, test_rows = learned.split(rows)
    assert len(test_rows) == len(learned.HELD_OUT) and len(train_rows) > 50
    for r in rows:
        assert len(r["ms"]) == len(r["features"]) == len(r["candidates"])
        assert all(len(f) == of.openfft_num_features() for f in r["features"])
    with open(learned.MODEL_FILE) as fh:
        model = json.load(fh)
    assert model["d"] == of.openfft_num_features()
    assert all(len(p) == of.openfft_mlp_num_params(model["d"], model["hidden"]) for p in model["params"])
    assert model["held_out"]["mean_regret"] <= 0.05
