"""bench.py's host-side bookkeeping, on the CPU: the pair-pipeline byte model
behind `roofline` (32 B per grid point per unique pair, plus the Phi read and
the W write), the roofline fields built from it, the peak it divides by, the
scaling of the profiled DRAM traffic from one captured batch to a build, and
the gate that reports that traffic only for the default schedule."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _system(name):
    return bench.SINGLE[name][1]


def test_pair_model_bytes_closed_form():
    s48, s96 = _system(bench.SI64), _system(bench.LARGE)
    assert (s48.ng, s48.n_occ, s96.ng, s96.n_occ) == (48 ** 3, 128, 96 ** 3, 1024)
    # unique pairs N(N+1)/2: 8256 and 524,800
    assert bench.unique_pairs(128) == 8256 and bench.unique_pairs(1024) == 524800
    assert bench.pair_model_bytes(s48) == 32 * 110592 * 8256 + 2 * 128 * 110592 * 8 == 29_444_014_080
    assert bench.pair_model_bytes(s96) == 32 * 884736 * 524800 + 2 * 1024 * 884736 * 8
    assert bench.pair_model_bytes(s96) == pytest.approx(14.87e12, rel=1e-3)


def test_peak_is_the_measured_copy_bandwidth():
    hbm, kind = bench.peaks()
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            assert (hbm, kind) == (float(json.load(f)["hbm_gbs"]), "measured")
    else:
        assert (hbm, kind) == (6800.0, "fallback")


def test_roofline_fields():
    s = _system(bench.SI64)
    hbm, _ = bench.peaks()
    r = bench.roofline(s, 8.8, None)
    achieved = 29_444_014_080 / 8.8e-3 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["peak"] == hbm
    assert r["achieved"] == pytest.approx(achieved)
    assert r["frac"] == pytest.approx(achieved / hbm)
    assert r["alg_bytes_per_launch"] == 29_444_014_080 and r["ms_per_launch"] == 8.8
    assert r["traffic"] is None and "traffic_source" not in r
    r = bench.roofline(s, 8.8, (12.0e9, "a capture"))
    assert r["traffic"] == 12.0e9 and r["traffic_source"] == "a capture"


def test_profiled_traffic_scaled_by_batch_equivalents():
    # one off-diagonal batch holds 64 pairs; a build is unique_pairs / 64 such batches
    for name, per_batch_mb in ((bench.LARGE, 3146.0), (bench.SI64, 93.5)):
        s = _system(name)
        batches = bench.unique_pairs(s.n_occ) / 64
        total, source = bench.TRAFFIC[name]
        assert f"x {batches:.0f} batch equivalents" in source
        assert f"({per_batch_mb:g} MB" in source
        assert total == pytest.approx(per_batch_mb * 1e6 * batches, rel=2e-3)


@pytest.mark.parametrize("flags", [["--max-pairs", "36"], ["--tile", "4"], ["--lanes", "2"], ["--eager"],
                                   ["--engine"], ["--no-pdl"], ["--no-overlap"], ["--radix", "1"]])
def test_traffic_reported_for_the_default_schedule_only(flags):
    assert bench.default_schedule(bench.parse([]))
    assert not bench.default_schedule(bench.parse(flags))
