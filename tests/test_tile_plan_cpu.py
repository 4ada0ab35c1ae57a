"""The pipelined volume kernel's tile schedule on the host (csrc/tile_plan.h, compiled alone with g++): the tiles of
every plan cover the elements once each and in order, the counter schedule is taken only where it is allowed and
every CTA has two full tiles, and at the sizes measured on a GB300 (p = 3 FP64: 4 elements per tile, 304 resident
CTAs on 152 SMs, meshes of 16 x 16 x k elements) the plan picks the schedule that ran faster there (volume kernel
time, round-robin / counter, us: k = 12: 138.6 / 131.0, 14: 139.1 / 141.2, 15: 159.8 / 151.9, 16: 159.9 / 163.7,
17: 182.2 / 174.0, 18: 182.3 / 184.4, 19: 182.3 / 185.8, 20: 202.8 / 195.7, 24: 246.2 / 238.0, 32: 313.3 /
305.3)."""
import json
import os
import random
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2112_10517_gb300", "csrc")


@pytest.fixture(scope="module")
def plan(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if not cxx:
        pytest.skip("no C++ compiler")
    exe = str(tmp_path_factory.mktemp("tile_plan") / "tile_plan_check")
    subprocess.run([cxx, "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(ROOT, "tests", "tile_plan_check.cpp"), "-o", exe], check=True)

    def run(cases):
        text = "".join("%d %d %d %d %d\n" % c for c in cases)
        out = subprocess.run([exe], input=text, capture_output=True, text=True, check=True).stdout
        return [json.loads(line) for line in out.splitlines()]
    return run


MEASURED = {12: "counter", 14: "rr", 15: "counter", 16: "rr", 17: "counter", 18: "rr", 19: "rr", 20: "counter",
            24: "counter", 32: "counter"}


def test_plan_picks_the_faster_schedule_at_the_measured_sizes(plan):
    res = plan([(256 * k, 4, 304, 152, 1) for k in sorted(MEASURED)])
    for k, r in zip(sorted(MEASURED), res):
        assert ("counter" if r["counter"] else "rr") == MEASURED[k], (k, r)
        assert r["once"] and r["in_order"] and r["sizes_ok"] and r["first_full"], r


def test_plan_keeps_round_robin_where_it_is_balanced_or_not_allowed(plan):
    res = plan([(32 ** 3, 4, 304, 152, 1),      # 53.9 tiles per SM: balanced either way
                (16 ** 3, 4, 304, 152, 0),      # not allowed (FP32, or half tiles that leave lanes idle)
                (256 * 17, 1, 304, 152, 1),     # one element per tile: no half tiles
                (256 * 17, 4, 600, 152, 1),     # fewer than two full tiles per CTA
                (0, 4, 304, 152, 1), (3, 4, 1, 152, 1)])
    for r in res:
        assert not r["counter"] and r["nfull"] == r["ntiles"], r
        assert r["once"] and r["in_order"] and r["sizes_ok"], r


def test_every_plan_covers_its_elements_once(plan):
    rng = random.Random(7)
    cases = []
    for _ in range(400):
        epb = rng.choice([1, 2, 3, 4, 7, 8, 16])
        sms = rng.choice([1, 7, 76, 152])
        grid = rng.randint(1, 3 * sms)
        elems = rng.randint(1, 40000)
        cases.append((elems, epb, grid, sms, rng.randint(0, 1)))
    res = plan(cases)
    assert len(res) == len(cases)
    for r in res:
        assert r["once"] and r["in_order"] and r["sizes_ok"] and r["first_full"], r
        if r["counter"]:
            assert r["allowed"] and r["epb"] >= 2 and r["elems"] // r["epb"] >= 2 * r["grid"], r
            assert r["grid"] <= r["nfull"] < r["ntiles"], r
    assert any(r["counter"] for r in res) and not all(r["counter"] for r in res)
