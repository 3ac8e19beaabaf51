"""The usage example in README.md runs as written (pair sum, rod stepping, Parareal, serving)."""
import os
import re

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    from paper_2604_12083_gb300 import build as B
    B.build()
    text = open(os.path.join(ROOT, "README.md")).read()
    blocks = re.findall(r"```python\n(.*?)```", text, re.S)
    assert blocks, "README.md has no python example"
    env = {}
    for code in blocks:
        exec(compile(code, "README.md", "exec"), env)
    torch.cuda.synchronize()
    assert env["done"] and env["latency_s"] > 0
    assert env["st"].final_incr < 1e-11
    assert torch.isfinite(env["u"]).all() and torch.isfinite(env["Xr"]).all()
    env["ctx"].close()
