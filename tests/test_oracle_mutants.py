"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of oracle/oracle.c: a sign, a dropped
term, an index, a transposed operand, an off-by-one in the decomposition or
in the real transform. It compiles the copy and runs a battery of checks
against references independent of the oracle: numpy's FFTs, the hand-worked
Eq. 2-7 boxes and numpy axis permutations. Every mutant must fail at least
one check, and the unmodified oracle must pass them all.
"""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1501_07350_gb300 import synth

SRC = os.path.join(os.path.dirname(oracle.__file__), "oracle.c")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "eq2_to_eq7_boxes_4x3x2.txt")

MUTANTS = {
    "twiddle sign": ("W[e].im = (double)((long double)sign * sinl(ang));",
                     "W[e].im = (double)(-(long double)sign * sinl(ang));"),
    "dropped product term": ("r.re = a.re * b.re - a.im * b.im;", "r.re = a.re * b.re;"),
    "twiddle index off by one": ("t[j] = cmul(y[j * m + k], W[((j * k) % n) * step]);",
                                 "t[j] = cmul(y[j * m + k], W[((j * (k + 1)) % n) * step]);"),
    "output index transposed": ("for (int64_t q = 0; q < r; ++q) y[k + q * m] = z[q];",
                                "for (int64_t q = 0; q < r; ++q) y[k * r + q] = z[q];"),
    "table stride dropped": ("cplx t = cmul(x[j * stride], W[((j * k) % n) * step]);",
                             "cplx t = cmul(x[j * stride], W[((j * k) % n)]);"),
    "Eq. 2 rounds up": ("if (Np <= N1) return ((N1 * id) / Np) * N2 * N3;",
                        "if (Np <= N1) return ((N1 * id + Np - 1) / Np) * N2 * N3;"),
    "Eq. 9 wrong factor": ("if (Np <= N1 * N2) return ((N1 * N2 * id) / Np) * N3;",
                           "if (Np <= N1 * N2) return ((N1 * N2 * id) / Np) * N2;"),
    "Eqs. 5-7 wrong divisor": ("int64_t b = (x - a * N2 * N3) / N3;", "int64_t b = (x - a * N2 * N3) / N2;"),
    "cab ordering transposed": ("static const int tab[3][3] = {{0, 1, 2}, {2, 0, 1}, {2, 1, 0}};",
                                "static const int tab[3][3] = {{0, 1, 2}, {1, 0, 2}, {2, 1, 0}};"),
    "owner bisection off by one": ("if (xs[mid] <= y) lo = mid; else hi = mid - 1;",
                                   "if (xs[mid] < y) lo = mid; else hi = mid - 1;"),
    "one stage with the wrong sign": ("rc |= transform_stage(1, n, Np, t1, -1);             /* along b in cab */",
                                      "rc |= transform_stage(1, n, Np, t1, 1);             /* along b in cab */"),
    "backward normalisation half dropped": ("out[i].re = t0[i].re / (double)N;", "out[i].re = t0[i].re;"),
    "Hermitian extension without conjugate": ("buf[k].im = -half[l * Nch + Nc - k].im;",
                                              "buf[k].im = half[l * Nch + Nc - k].im;"),
    "inverse real transform keeps Im": ("for (int64_t i = 0; i < Nc; ++i) x[xx + i] = res[i].re;",
                                        "for (int64_t i = 0; i < Nc; ++i) x[xx + i] = res[i].im;"),
    "real stage keeps one frequency too few": ("memcpy(half + l * Nch, res, sizeof(cplx) * (size_t)Nch);",
                                               "memcpy(half + l * Nch, res, sizeof(cplx) * (size_t)(Nch - 1));"),
    "D-dimensional ordering keeps the moved axes in forward order": (
        "for (int i = 0; i < s - 1; ++i) axes[k++] = D - 1 - i;",
        "for (int i = 0; i < s - 1; ++i) axes[k++] = D - s + 1 + i;"),
    "D-dimensional decomposition drops the trailing product": (
        "for (int j = 2; j < D; ++j) rest *= n[axes[j]];",
        "for (int j = 2; j < 3; ++j) rest *= n[axes[j]];"),
}


def _close(a, b, tol=1e-12):
    a = np.asarray(a).reshape(-1)
    b = np.asarray(b).reshape(-1)
    return a.shape == b.shape and np.all(np.isfinite(a)) and np.linalg.norm(a - b) <= tol * max(1.0, np.linalg.norm(b))


def _checks():
    """name -> bool: each compares the loaded oracle with an independent reference."""
    out = {}
    # 1-D engine vs numpy, both signs, composite and prime lengths
    ok = True
    for n in list(range(1, 17)) + [30, 49, 77]:
        x = synth.complex_field((n,), seed=n)
        ok &= _close(oracle.fft1d(x, oracle.FORWARD), np.fft.fft(x))
        ok &= _close(oracle.fft1d(x, oracle.BACKWARD), np.fft.ifft(x) * n)
    out["fft1d vs numpy"] = bool(ok)
    # 3-D forward and backward vs numpy (slabs and pencils)
    ok = True
    for shape, P in [((4, 6, 5), 3), ((6, 4, 8), 10), ((5, 6, 7), 2), ((8, 8, 8), 16)]:
        Na, Nb, Nc = shape
        x = synth.complex_field(shape, seed=sum(shape) + P)
        try:
            y = oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)
            z = oracle.fft3d(x.reshape(-1), Na, Nb, Nc, P, oracle.BACKWARD)
        except ValueError:
            ok = False
            continue
        ok &= _close(y, oracle.abc_to_cba(np.fft.fftn(x)))
        X_cba = x.reshape(Nc, Nb, Na)          # the input read as a cba spectrum
        ok &= _close(z, np.fft.ifftn(np.transpose(X_cba, (2, 1, 0))).reshape(-1))
    out["fft3d vs numpy"] = bool(ok)
    # boxes vs the hand-worked Eq. 2-7 table
    ok = True
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(t) for t in line.split()]
        N1, N2, N3, Np, i = v[:5]
        try:
            xs, xe, s3, e3 = oracle.box(N1, N2, N3, Np, i)
        except ValueError:
            ok = False
            continue
        ok &= (xs, xe, tuple(s3), tuple(e3)) == (v[5], v[6], tuple(v[7:10]), tuple(v[10:13]))
    out["boxes vs hand-worked table"] = bool(ok)
    # transposes vs numpy axis permutations
    ok = True
    for shape, P in [((4, 3, 2), 3), ((4, 3, 2), 6), ((8, 6, 10), 40), ((5, 7, 3), 15)]:
        Na, Nb, Nc = shape
        a = synth.complex_field(shape, seed=P)
        try:
            cab, _ = oracle.redistribute(Na, Nb, Nc, P, "abc->cab", a.reshape(-1))
            cba, _ = oracle.redistribute(Na, Nb, Nc, P, "cab->cba", cab)
        except ValueError:
            ok = False
            continue
        ok &= np.array_equal(cab, np.transpose(a, (2, 0, 1)).reshape(-1))
        ok &= np.array_equal(cba, np.transpose(a, (2, 1, 0)).reshape(-1))
    out["transposes vs axis permutations"] = bool(ok)
    # real transforms vs numpy rfftn / irfftn
    ok = True
    for shape, P in [((4, 6, 8), 3), ((5, 3, 7), 2), ((6, 5, 4), 5)]:
        Na, Nb, Nc = shape
        Nch = Nc // 2 + 1
        x = synth.uniform_pm1(Nc, Na * Nb * Nc).reshape(shape)
        H = synth.complex_field((Nch, Nb, Na), seed=Nc + 1).reshape(-1)
        try:
            X = oracle.rfft3d(x, Na, Nb, Nc, P)
            xb = oracle.rfft3d(H, Na, Nb, Nc, P, oracle.BACKWARD)
        except ValueError:
            ok = False
            continue
        ok &= _close(X, np.transpose(np.fft.rfftn(x), (2, 1, 0)).reshape(-1))
        ref = np.fft.irfftn(np.transpose(H.reshape(Nch, Nb, Na), (2, 1, 0)), s=(Na, Nb, Nc), axes=(0, 1, 2))
        ok &= _close(xb, ref.reshape(-1))
    out["real transforms vs numpy"] = bool(ok)
    # D-dimensional transforms vs numpy fftn (result in the reversed axes)
    ok = True
    for dims, P in [((4, 3, 5, 2), 8), ((2, 3, 2, 2, 3), 6), ((3, 4, 2, 2, 5), 2)]:
        x = synth.complex_field(dims, seed=sum(dims) + P)
        rev = tuple(range(len(dims) - 1, -1, -1))
        try:
            y = oracle.fftnd(x, dims, P, oracle.FORWARD)
        except ValueError:
            ok = False
            continue
        ok &= _close(y, np.transpose(np.fft.fftn(x), rev))
    out["D-dimensional transforms vs numpy"] = bool(ok)
    return out


def _run_checks(so_path):
    """Checks of the library at so_path, in a child process (a planted mistake
    may also crash the oracle, e.g. an index past an array: that counts as
    caught).  Returns the dict of results, or None if the child failed."""
    import json
    import sys
    code = ("import json, ctypes, sys; sys.path[:0] = %r; import oracle; "
            "import tests.test_oracle_mutants as m; "
            "oracle._lib = oracle._configure(ctypes.CDLL(%r)); print(json.dumps(m._checks()))"
            % ([os.path.dirname(os.path.dirname(os.path.abspath(__file__)))], so_path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=300)
    if r.returncode != 0:
        return None
    return json.loads(r.stdout.strip().splitlines()[-1])


def _build(src_text, tmp_path, name):
    c = tmp_path / (name + ".c")
    so = tmp_path / (name + ".so")
    c.write_text(src_text)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-o", str(so), str(c), "-lm"])
    return str(so)


def test_unmodified_oracle_passes_every_check(tmp_path):
    res = _run_checks(_build(open(SRC).read(), tmp_path, "clean"))
    assert res is not None and all(res.values()), res


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "the mutation site must exist exactly once"
    res = _run_checks(_build(src.replace(old, new), tmp_path, "mutant"))
    assert res is None or not all(res.values()), "no check caught: " + name
