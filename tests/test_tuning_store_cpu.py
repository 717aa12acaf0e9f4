"""Persisted tuning choices (the paper's "User-select" reuse of a tuned method,
Sec. 3.2.3) on the host: the table's text file round trip, merging, lookup and
the rejection of malformed files.  No GPU: these calls never touch one."""
import os

import pytest

from paper_1501_07350_gb300 import openfft as of


@pytest.fixture(autouse=True)
def library():
    from paper_1501_07350_gb300 import _build
    _build.build()
    of.load()
    of.openfft_tuning_clear()
    yield
    of.openfft_tuning_clear()


def _write(path, text):
    with open(path, "w") as fh:
        fh.write(text)


def test_load_lookup_save_round_trip(tmp_path):
    src = tmp_path / "choices.txt"
    _write(src, "# comment\n512 512 512 64 0 2 1 4 0\n\n120 144 160 32 1 2 0 16 2\n")
    of.openfft_tuning_load(str(src))
    assert of.openfft_tuning_lookup(512, 512, 512, 64, of.C2C_F64) == (2, 1, 4, 0)
    assert of.openfft_tuning_lookup(120, 144, 160, 32, of.C2C_F32) == (2, 0, 16, 2)
    assert of.openfft_tuning_lookup(512, 512, 512, 256, of.C2C_F64) is None
    out = tmp_path / "saved.txt"
    of.openfft_tuning_save(str(out))
    lines = [l for l in open(out).read().splitlines() if not l.startswith("#")]
    assert sorted(lines) == sorted(["512 512 512 64 0 2 1 4 0", "120 144 160 32 1 2 0 16 2"])
    of.openfft_tuning_clear()
    assert of.openfft_tuning_lookup(512, 512, 512, 64, of.C2C_F64) is None
    of.openfft_tuning_load(str(out))
    assert of.openfft_tuning_lookup(512, 512, 512, 64, of.C2C_F64) == (2, 1, 4, 0)


def test_a_later_file_replaces_entries_of_the_same_problem(tmp_path):
    a, b = tmp_path / "a.txt", tmp_path / "b.txt"
    _write(a, "64 64 64 8 0 2 1 8 0\n32 32 32 4 0 2 1 4 2\n")
    _write(b, "64 64 64 8 0 1 1 8 0\n")
    of.openfft_tuning_load(str(a))
    of.openfft_tuning_load(str(b))
    assert of.openfft_tuning_lookup(64, 64, 64, 8, of.C2C_F64) == (1, 1, 8, 0)
    assert of.openfft_tuning_lookup(32, 32, 32, 4, of.C2C_F64) == (2, 1, 4, 2)


@pytest.mark.parametrize("bad", ["64 64 64 8 0 2 1 8\n", "64 64 64 8 0 2 1 8 0 7\n", "0 64 64 8 0 2 1 8 0\n",
                                 "64 64 64 0 0 2 1 8 0\n", "64 64 64 8 99 2 1 8 0\n", "64 64 x 8 0 2 1 8 0\n"])
def test_malformed_lines_are_refused_and_leave_the_table(tmp_path, bad):
    good = tmp_path / "good.txt"
    _write(good, "16 16 16 2 0 2 1 4 0\n")
    of.openfft_tuning_load(str(good))
    path = tmp_path / "bad.txt"
    _write(path, "32 32 32 4 0 2 1 4 2\n" + bad)
    with pytest.raises(of.OpenFFTError) as e:
        of.openfft_tuning_load(str(path))
    assert e.value.status == of.ERR_INVALID_ARG
    assert "line 2" in str(e.value)
    assert of.openfft_tuning_lookup(32, 32, 32, 4, of.C2C_F64) is None     # nothing of the file merged
    assert of.openfft_tuning_lookup(16, 16, 16, 2, of.C2C_F64) == (2, 1, 4, 0)


def test_missing_files_are_reported(tmp_path):
    with pytest.raises(of.OpenFFTError) as e:
        of.openfft_tuning_load(str(tmp_path / "absent.txt"))
    assert e.value.status == of.ERR_INVALID_ARG
    with pytest.raises(of.OpenFFTError):
        of.openfft_tuning_save(os.path.join(str(tmp_path), "no", "such", "dir.txt"))
