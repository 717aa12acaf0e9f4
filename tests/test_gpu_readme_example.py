"""The basic usage sequence of the library (plan, stream, tuning, forward,
backward, box query, destroy) runs on the GPU, and its round trip gives back
the input (FP64 bound 1e-12).  The calls are the ones a user's first program
makes; the same sequence is shown as the usage example of the package."""
import pytest

pytestmark = pytest.mark.gpu


def test_usage_sequence_round_trip():
    import torch
    from paper_1501_07350_gb300 import _build, openfft as of

    _build.build()
    torch.manual_seed(5)
    n, P = 256, 64
    x = torch.randn(n ** 3, dtype=torch.complex128, device="cuda")    # abc order [Na][Nb][Nc]
    x0 = x.clone()
    y = torch.empty_like(x)
    plan = of.openfft_plan(n, n, n, P, of.C2C_F64)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        of.openfft_set_tuning(plan, of.TUNE_EXHAUSTIVE)
        of.openfft_exec_c2c(plan, x, y, of.FORWARD)      # y: cba order [Nc][Nb][Na]
        of.openfft_exec_c2c(plan, y, x, of.BACKWARD)     # back to abc, divided by N
        of.openfft_sync(plan)
        assert float(torch.linalg.vector_norm(x - x0) / torch.linalg.vector_norm(x0)) < 1e-12
        start, end, offset, count = of.openfft_box(plan, 1, 3)   # rank 3's output box
        assert count > 0 and offset >= 0
    finally:
        of.openfft_destroy(plan)
