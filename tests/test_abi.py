"""The C-ABI library builds, loads and exports every symbol include/*.h declares (no GPU)."""
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        for m in re.finditer(r"MRS_API\s+[A-Za-z_][A-Za-z0-9_ \*]*?\b([A-Za-z_][A-Za-z0-9_]*)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2604_12083_gb300 import build as B
    return B.build()


def test_library_exports_every_declared_symbol(libpath):
    decl = declared_symbols()
    assert len(decl) >= 15
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True).stdout
    exported = {ln.split()[-1] for ln in out.splitlines() if " T " in ln}
    missing = decl - exported
    assert not missing, missing
    # nothing but the declared ABI is exported
    assert exported - decl == set(), exported - decl


def test_library_loads_and_binding_lists_match(libpath):
    from paper_2604_12083_gb300 import mrs
    L = mrs.lib()
    assert L.mrs_version().decode().startswith("mrs_gb300")
    assert set(mrs.EXPORTS) == declared_symbols()
    for name in mrs.EXPORTS:
        assert hasattr(L, name)
    assert L.mrs_plan_config_count() >= 1


def test_errors_without_gpu_are_reported_not_fatal(libpath):
    """With no usable device, context creation fails with a status and a message."""
    import ctypes
    import torch
    from paper_2604_12083_gb300 import mrs
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = mrs.lib().mrs_ctx_create(ctypes.byref(h), 0)
    assert st in (mrs.MRS_EINVAL, mrs.MRS_ECUDA)
    assert len(mrs.lib().mrs_last_error()) > 0


def test_config_table_host_queries(libpath):
    """The configuration table answers without a device: the persistent ordered
    configurations 0..16, the symmetric ones (each unordered pair evaluated once) 17..26, then
    the ordered cluster ones; out-of-range ids are rejected."""
    from paper_2604_12083_gb300 import mrs
    n = mrs.plan_config_count()
    flags = [mrs.plan_config_symmetric(c) for c in range(n)]
    assert n == 29 and not any(flags[:17]) and all(flags[17:27]) and not any(flags[27:])
    assert mrs.lib().mrs_plan_config_symmetric(n) == -1
    assert mrs.lib().mrs_plan_config_symmetric(-1) == -1
    with pytest.raises(mrs.MrsError):
        mrs.plan_config_symmetric(n)
