"""Persisted tuning choices on the GPU: tuning records its choice, a saved
choice is selected without timing runs (a deliberately slow candidate, which
exhaustive tuning would never pick, proves that the table decided), and a
problem without an entry falls back to exhaustive tuning and is recorded.
The transform with the selected candidate matches the oracle (1e-12)."""
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


def _describe(plan, index):
    c = of.openfft_candidate(plan, index)
    return (c["variant"], c["arith"], c["lines_per_cta"], c["kernel"])


def test_saved_choice_is_selected_and_tuning_records(torch, tmp_path):
    Na, Nb, Nc, P = 48, 40, 64, 8
    of.openfft_tuning_clear()
    try:
        plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
        try:
            # the explicit pack / exchange / unpack method: never the fastest
            slow = [i for i in range(of.openfft_num_candidates(plan))
                    if of.openfft_candidate(plan, i)["variant"] == of.VARIANT_PACK_EXCHANGE_UNPACK][0]
            d = _describe(plan, slow)
        finally:
            of.openfft_destroy(plan)
        path = tmp_path / "choices.txt"
        path.write_text("%d %d %d %d %d %d %d %d %d\n" % ((Na, Nb, Nc, P, of.C2C_F64) + d))
        of.openfft_tuning_load(str(path))
        x = synth.complex_field((Na, Nb, Nc), seed=31)
        ref = oracle.fft3d(x, Na, Nb, Nc, P, oracle.FORWARD)
        plan = of.openfft_plan(Na, Nb, Nc, P, of.C2C_F64)
        try:
            of.openfft_set_stream(plan, torch.cuda.current_stream())
            of.openfft_set_tuning(plan, of.TUNE_SAVED)
            assert _describe(plan, of.openfft_current_candidate(plan)) == d
            xd = torch.from_numpy(x.reshape(-1).copy()).cuda()
            yd = torch.empty_like(xd)
            of.openfft_exec_c2c(plan, xd, yd, of.FORWARD)
            of.openfft_sync(plan)
            assert oracle.rel_l2(yd.cpu().numpy(), ref) < 1e-12
            # exhaustive tuning replaces the entry with its own (faster) choice
            of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
            best = _describe(plan, of.openfft_current_candidate(plan))
            assert best != d
            assert of.openfft_tuning_lookup(Na, Nb, Nc, P, of.C2C_F64) == best
        finally:
            of.openfft_destroy(plan)
        # a problem without an entry: SAVED runs exhaustive tuning and records it
        plan = of.openfft_plan(Na, Nb, Nc, 4, of.C2C_F64)
        try:
            of.openfft_set_stream(plan, torch.cuda.current_stream())
            assert of.openfft_tuning_lookup(Na, Nb, Nc, 4, of.C2C_F64) is None
            of.openfft_set_tuning(plan, of.TUNE_SAVED)
            assert of.openfft_tuning_lookup(Na, Nb, Nc, 4, of.C2C_F64) == \
                _describe(plan, of.openfft_current_candidate(plan))
        finally:
            of.openfft_destroy(plan)
        # save and reload: the same table
        out = tmp_path / "saved.txt"
        of.openfft_tuning_save(str(out))
        of.openfft_tuning_clear()
        of.openfft_tuning_load(str(out))
        assert of.openfft_tuning_lookup(Na, Nb, Nc, P, of.C2C_F64) == best
    finally:
        of.openfft_tuning_clear()
