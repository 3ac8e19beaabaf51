"""The usage example (examples/usage.py: pair sum, rod stepping, Parareal, serving) runs and its
results are finite and converged."""
import importlib.util
import os

import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_usage_example_runs():
    from paper_2604_12083_gb300 import build as B
    B.build()
    spec = importlib.util.spec_from_file_location("usage", os.path.join(ROOT, "examples", "usage.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    env = mod.run()
    torch.cuda.synchronize()
    assert env["done"] and env["latency_s"] > 0
    assert env["st"].final_incr < 1e-11
    assert torch.isfinite(env["u"]).all() and torch.isfinite(env["Xr"]).all()
    env["ctx"].close()
