"""The debug build's index checks (paper_2604_12083_gb300/csrc/mrs_checks.h), on the host: each
predicate accepts a valid work tile or rod node entry and rejects every copy with one planted
mistake (an extent past the tile size or the point arrays, unit or diagonal counts that do not
match the extent, units outside the pass's column buffer, row segments outside the row buffer,
a node index outside its rod, a rod outside the node range).  The debug library builds for
sm_103a and exports the same symbols as the release library."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_12083_gb300", "csrc")


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    from paper_2604_12083_gb300 import build as B
    exe = str(tmp_path_factory.mktemp("checks") / "checks_driver")
    cmd = [B.nvcc(), "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "checks_driver.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_valid_entries_accepted(results):
    assert results["sym_valid"] == 1 and results["ordered_valid"] == 1 and results["node_valid"] == 1


def test_planted_mistakes_rejected(results):
    bad = {k: v for k, v in results.items() if not k.endswith("_valid")}
    assert len(bad) == 21
    assert all(v == 0 for v in bad.values()), {k: v for k, v in bad.items() if v}


def test_debug_library_builds_with_the_same_exports():
    from paper_2604_12083_gb300 import build as B
    rel, dbg = B.build(), B.build(debug=True)

    def exports(path):
        out = subprocess.run(["nm", "-D", "--defined-only", path], check=True, capture_output=True,
                             text=True).stdout
        return {l.split()[-1] for l in out.splitlines() if " T " in l}

    assert exports(rel) == exports(dbg) and len(exports(rel)) > 30
