"""CPU check of the row passes' plan (csrc/rows_plan.h, compiled for the
host): which lattices the row-staged and fused passes take, the tile
enumeration (single-row tiles skip the face rows of a non-periodic axis 1,
whose nodes the face pass steps; every other row is in exactly one tile),
and a shared-memory layout that is aligned, non-overlapping and within the
opt-in limit."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1803_07822_gb300", "csrc")
MAX_SMEM = 232448  # 227 KB opt-in per block


@pytest.fixture(scope="module")
def plan_exe(tmp_path_factory):
    exe = tmp_path_factory.mktemp("plan") / "plan"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-I" + CSRC, os.path.join(ROOT, "tests", "rows_plan_check.cpp"),
                           "-o", str(exe)])
    return exe


def plan(exe, n, yper, zper, sb, max_smem=MAX_SMEM):
    out = subprocess.check_output([str(exe), *map(str, n), str(int(yper)), str(int(zper)), str(sb), str(max_smem)])
    return {k: int(v) for k, v in (kv.split("=") for kv in out.decode().split())}


def tile_rows(p, n1):
    """Rows of a plane covered by the tiles, with multiplicity."""
    rows = []
    for yb in range(p["nyb"]):
        y0 = p["y1"] + yb * p["TR"]
        rows += [y for y in range(y0, y0 + p["TR"]) if y < n1]
    return rows


@pytest.mark.parametrize("n,yper,zper,sb", [
    ((256, 256, 256), False, False, 4), ((256, 256, 64), False, False, 2), ((256, 24, 12), False, False, 4),
    ((256, 16, 10), True, False, 4), ((100, 24, 10), True, False, 4), ((64, 16, 9), False, False, 4),
    ((20, 29, 13), False, False, 4), ((32, 32, 16), True, True, 4), ((96, 37, 9), False, False, 2)])
def test_tiles_cover_the_rows_the_row_passes_step(plan_exe, n, yper, zper, sb):
    p = plan(plan_exe, n, yper, zper, sb)
    assert p["ok"] == 1
    n0, n1, n2 = n
    assert p["TR"] * n0 <= 256 and p["TR"] >= 1
    rows = tile_rows(p, n1)
    if p["TR"] == 1 and not yper:
        assert p["y1"] == 1 and sorted(rows) == list(range(1, n1 - 1))
    else:
        assert p["y1"] == 0 and sorted(rows) == list(range(n1))
    planes = n2 if zper else n2 - 2
    assert p["z0"] == (0 if zper else 1) and p["ntiles"] == p["nyb"] * planes


@pytest.mark.parametrize("n,sb", [((256, 256, 256), 4), ((256, 256, 256), 2), ((128, 64, 32), 4), ((20, 29, 13), 4)])
def test_shared_memory_layout(plan_exe, n, sb):
    p = plan(plan_exe, n, False, False, sb)
    assert p["ok"] == 1 and p["fused_ok"] == 1
    # one stage: populations [19][256], rho u [3][JS] of 16 bytes, geometry [25][256], history [10][256]
    for k in ("off_jf", "off_geo", "off_hist", "stage", "off_m", "off_sg", "off_h4", "off_js"):
        assert p[k] % 128 == 0 or k in ("off_h4",), k
    assert p["off_jf"] >= 19 * 256 * sb
    assert p["off_geo"] >= p["off_jf"] + 3 * p["JS"] * 16
    assert p["off_hist"] == p["off_geo"] + 25 * 256 * 4
    assert p["stage"] >= p["off_hist"] + 10 * 256 * 4
    assert p["JS"] >= (p["TR"] + 2) * n[0] and p["JL"] * p["JR"] == (p["TR"] + 2) * 4 * n[0]
    # the fused pass: two step stages, the momentum stage, two rho u tiles and ten barriers
    assert p["off_m"] == 2 * p["stage"] and p["off_js"] >= p["off_m"] + p["off_h4"] + 4 * 256 * 4
    assert p["fused"] == p["off_js"] + 2 * 256 * 16 + 80 <= MAX_SMEM


@pytest.mark.parametrize("n,yper,zper,sb", [
    ((300, 16, 16), False, False, 4),   # rows longer than a tile
    ((30, 16, 16), False, False, 4),    # rows not a whole number of 4 nodes
    ((100, 16, 16), False, False, 2),   # FP16 rows not a whole number of 16-byte chunks
    ((256, 2, 16), False, False, 4),    # a non-periodic axis 1 with fewer than 3 rows
    ((256, 16, 2), False, False, 4),    # a non-periodic axis 2 with fewer than 3 planes
    ((8, 4, 4), True, True, 4),         # fewer nodes than a tile
])
def test_lattices_the_row_passes_refuse(plan_exe, n, yper, zper, sb):
    assert plan(plan_exe, n, yper, zper, sb)["ok"] == 0


def test_stages_that_do_not_fit_are_refused(plan_exe):
    assert plan(plan_exe, (256, 256, 256), False, False, 4, max_smem=100000)["ok"] == 0
