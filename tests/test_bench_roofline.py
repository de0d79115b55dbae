"""Host arithmetic of the bench's roofline entry: the dominant stage, its
algorithmic bandwidth from the per-stage times, and the committed DRAM
traffic record scaled to the timed launch (no GPU)."""
import hashlib
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _prof(sort_ms=0.17, radix_calls=0):
    calls = 4
    per_hull = {"extremes": 0.04, "witness": 0.01, "filter": 0.10, "scatter": 0.09, "split": 0.12,
                "sort": sort_ms, "-6": 0.0, "regions": 0.01, "final": 0.035}
    return {"calls": calls, "radix_calls": radix_calls, "points": 20_000_000 * calls,
            "survivors": 0, "witness_survivors": 8_000_000 * calls, "second_round": 300_000 * calls,
            "ms": {k: v * calls for k, v in per_hull.items()}}


def test_dominant_stage_and_its_bandwidth():
    r = bench.roofline_of(_prof(), 6000.0, "measured")
    assert r["kernel"] == "k3_bucket"
    b = 12.0 * 8_000_000 + 12.0 * 300_000
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(b)
    assert r["achieved"] == pytest.approx(b / 0.17e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6000.0)
    assert set(r["stages"]) == set(bench.STAGE_KERNELS)
    assert "-6" not in r["stage_ms_per_hull"]
    # the pipeline figure: all stages' algorithmic bytes over their summed time
    tot_b = sum(k["algorithmic_bytes"] for k in r["stages"].values())
    tot_ms = sum(r["stage_ms_per_hull"].values())
    assert r["pipeline_gbs"] == pytest.approx(tot_b / (tot_ms / 1e3) / 1e9)


def test_another_stage_can_dominate():
    r = bench.roofline_of(_prof(sort_ms=0.05), 6000.0, "measured")
    assert r["kernel"].startswith("k3_split")
    # the fused filter's bytes: one read of the points and the pairs it writes
    assert r["stages"]["filter"]["algorithmic_bytes"] == pytest.approx(8.0 * 20_000_000 + 12.0 * 8_000_000)
    assert r["stages"]["filter"]["units"] == pytest.approx(20_000_000)


def test_rerun_on_radix_passes_reports_no_single_kernel():
    r = bench.roofline_of(_prof(radix_calls=1), 6000.0, "measured")
    assert r["achieved"] is None and r["frac"] is None and r["traffic"] is None


def test_traffic_record_scaled_and_invalidated(tmp_path, monkeypatch):
    src = tmp_path / "k.cu"
    src.write_bytes(b"kernel source")
    (tmp_path / "profiles").mkdir()
    rec = {"sources": {"k.cu": hashlib.sha256(b"kernel source").hexdigest()},
           "dram_bytes_read": 1000, "dram_bytes_write": 200, "units": 100}
    (tmp_path / "profiles" / "kx_traffic.json").write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.kernel_traffic("kx", 50) == pytest.approx(600.0)
    assert bench.kernel_traffic("missing", 50) is None
    src.write_bytes(b"kernel source, changed")
    assert bench.kernel_traffic("kx", 50) is None



def test_single_read_front_stage_bytes():
    """Calls on the single-read front: the extremes stage reads every point
    once and writes the raw survivors; the polygon stage reads the sample
    polygon's 1/1024 sample; the witnesses read the raw survivors' points;
    the fused filter reads the raw survivors and writes the pairs, its
    units being the raw survivors."""
    p = _prof()
    calls = p["calls"]
    p["raw_survivors"] = 200_000 * calls
    p["single_read_calls"] = calls
    p["ms"]["extremes"] = 0.2 * calls            # the dominant stage
    p["ms"]["polygon"] = 0.01 * calls
    r = bench.roofline_of(p, 6000.0, "measured")
    n, q, s = 20_000_000, 200_000, 8_000_000
    assert r["front"] == "single-read" and r["raw_survivors_per_hull"] == pytest.approx(q)
    assert r["kernel"] == "k1_poly"
    b = 8.0 * n + 12.0 * q
    assert r["algorithmic_bytes_per_launch"] == pytest.approx(b)
    assert r["stages"]["witness"]["algorithmic_bytes"] == pytest.approx(8.0 * q)
    assert r["stages"]["polygon"]["algorithmic_bytes"] == pytest.approx(8.0 * n / 1024)
    assert r["stages"]["polygon"]["gbs"] == pytest.approx(8.0 * n / 1024 / 0.01e-3 / 1e9)
    assert r["stages"]["filter"]["algorithmic_bytes"] == pytest.approx(12.0 * q + 12.0 * s)
    assert r["stages"]["filter"]["units"] == pytest.approx(q)
    # a profile that mixes both fronts is read with the two-read table
    p["single_read_calls"] = calls - 1
    assert bench.roofline_of(p, 6000.0, "measured")["front"] == "two-read"
