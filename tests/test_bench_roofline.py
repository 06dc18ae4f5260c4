"""Host-side arithmetic of the bench line's roofline entry (no GPU): achieved
bandwidth from the algorithmic bytes of one launch over its event-timed
duration, the fraction of the peak, and the ncu DRAM bytes taken from the
committed record only for the launch shape and kernel sources they were
measured on."""
import json
import os

import bench

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_achieved_and_fraction():
    cells = 256 ** 3
    # 20 launches of the moment kernel taking 18.4 ms in all: 0.92 ms each
    r = bench.roofline_entry("bme", {"bme": 18.4}, 20, cells, 4, "mixed", None)
    alg = bench.ALG_WORDS["bme"] * 4 * cells
    assert bench.ALG_WORDS["bme"] == 33 and bench.ALG_WORDS["gas"] == 13   # words read + written per cell
    assert r["alg_bytes_per_launch"] == alg
    assert abs(r["avg_launch_ms"] - 0.92) < 1e-12
    assert abs(r["achieved"] - alg / 0.92e-3 / 1e9) < 1e-6
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-12
    assert r["bound"] == "hbm" and r["unit"] == "GB/s" and r["traffic"] is None


def test_traffic_only_for_the_recorded_shape_and_sources(monkeypatch):
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    monkeypatch.setattr(bench, "traffic_key_hash", lambda: rec["sha256_16"])
    hit = bench.roofline_entry("bme", {"bme": 18.4}, 20, 256 ** 3, 4, "mixed", 256, cand=0)
    assert hit["traffic"] == rec["bme-mixed-256-shape0"]
    assert bench.roofline_entry("bme", {"bme": 18.4}, 20, 256 ** 3, 4, "mixed", 256, cand=1)["traffic"] is None
    assert bench.roofline_entry("bme", {"bme": 18.4}, 20, 128 ** 3, 4, "mixed", 128, cand=0)["traffic"] is None
    monkeypatch.setattr(bench, "traffic_key_hash", lambda: "0" * 16)
    assert bench.roofline_entry("bme", {"bme": 18.4}, 20, 256 ** 3, 4, "mixed", 256, cand=0)["traffic"] is None


def test_traffic_record_covers_the_kernel_sources():
    rec = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    assert tuple(rec["sources"]) == bench.TRAFFIC_SOURCES
    for rel in rec["sources"]:
        assert os.path.exists(os.path.join(ROOT, rel))
    # DRAM bytes per launch are near the compulsory bytes of the 256^3 launches
    for kern in ("bme", "gas"):
        alg = bench.ALG_WORDS[kern] * 4 * 256 ** 3
        assert 1.0 <= rec[f"{kern}-mixed-256-shape0"] / alg < 1.5
