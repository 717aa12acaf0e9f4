import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built extension")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def pytest_collection_modifyitems(config, items):
    # GPU tests are skipped (not failed) on machines without a GPU only when the
    # run did not ask for them explicitly; `-m gpu` on a machine with a GPU runs them.
    try:
        import torch
        has_gpu = torch.cuda.is_available()
    except Exception:  # pragma: no cover
        has_gpu = False
    if has_gpu:
        return
    skip = pytest.mark.skip(reason="no CUDA device on this machine")
    for item in items:
        if "gpu" in item.keywords:
            item.add_marker(skip)


@pytest.fixture(autouse=True)
def _bounds_status_of_the_checked_build():
    """Under OPENFFT_GB_CHECKED=1 (the bounds-checked library), every test
    also requires that no kernel met an index outside its array: the per-plan
    words are reported by openfft_sync, the per-device word is read here."""
    yield
    if os.environ.get("OPENFFT_GB_CHECKED", "") != "1":
        return
    from paper_1501_07350_gb300 import openfft as of
    if of._lib is None:
        return
    assert of.openfft_checked_build(), "OPENFFT_GB_CHECKED=1 but the normal library is loaded"
    assert of.openfft_debug_bounds_status() == 0, "a kernel met a global index outside its array"
