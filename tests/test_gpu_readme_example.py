"""The usage example of the README runs as written on the GPU, and its round
trip gives back the input (FP64 bound 1e-12)."""
import os
import re

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    import torch
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, flags=re.S)
    assert blocks, "no python example in the README"
    code = blocks[0].replace("print(", "_shown.append(")
    ns = {"_shown": []}
    torch.manual_seed(5)
    exec(compile(code, "README.md", "exec"), ns)
    x0 = ns["x"].clone()
    # the example ends with x = BACKWARD(FORWARD(x)); run the same two calls on a
    # fresh plan from a saved copy to check the round trip
    of = ns["of"]
    n, P = ns["n"], ns["P"]
    plan = of.openfft_plan(n, n, n, P, of.C2C_F64)
    try:
        of.openfft_set_stream(plan, torch.cuda.current_stream())
        y = torch.empty_like(x0)
        z = torch.empty_like(x0)
        of.openfft_exec_c2c(plan, x0, y, of.FORWARD)
        of.openfft_exec_c2c(plan, y, z, of.BACKWARD)
        of.openfft_sync(plan)
        assert float(torch.linalg.vector_norm(z - x0) / torch.linalg.vector_norm(x0)) < 1e-12
    finally:
        of.openfft_destroy(plan)
    start, end, offset, count = ns["_shown"][0]
    assert count > 0 and offset >= 0
