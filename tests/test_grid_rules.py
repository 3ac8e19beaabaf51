"""Host logic of the pair-sum plans (paper_2604_12083_gb300/csrc/mrs_internal.h), on the CPU:
the persistent grid of an ordered plan on one system of 3072 / 4096 / 6144 / 8192 points with
256-thread CTAs (one CTA per SM while the full grid would give each fewer than 12 units, the
full grid above), the per-tile split cap alone for 64- and 128-thread CTAs, fewer units than
SMs, and the tile size of the cluster and symmetric configurations."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2604_12083_gb300", "csrc")


@pytest.fixture(scope="module")
def results(tmp_path_factory):
    from paper_2604_12083_gb300 import build as B
    exe = str(tmp_path_factory.mktemp("grid") / "grid_driver")
    cmd = [B.nvcc(), "-std=c++17", "-O1", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "grid_driver.cu"), "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return {k: int(v) for k, v in (line.split() for line in out.splitlines())}


def test_one_cta_per_sm_when_little_work(results):
    # 3072 points: 12 tiles x 96 units, capped at 16 CTAs per tile (192), then one per SM
    assert results["p256_3072"] == 152
    # 4096 and 6144 points: 4.5 and 10 units per CTA of the full grid of 456 -> one per SM
    assert results["p256_4096"] == 152 and results["p256_6144"] == 152
    # 8192 points: 18 units per CTA -> the full grid
    assert results["p256_8192"] == 456


def test_small_ctas_keep_the_cap(results):
    # 10 tiles x 80 units = 800 units: 16 CTAs per tile, tile-aligned ranges kept
    assert results["p64_2560"] == 160
    # 16 tiles x 64 units: the full grid of 912 would give ~1 unit each -> 16 per tile
    assert results["p128_2048"] == 256


def test_fewer_units_than_sms(results):
    # 2 tiles x 10 units: one unit per CTA
    assert results["p256_300"] == 20


def test_tile_sizes(results):
    assert results["tm_cluster8"] == 32 and results["tm_cluster4"] == 64 and results["tm_sym"] == 384
