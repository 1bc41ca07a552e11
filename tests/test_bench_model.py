"""Host-side parts of the benchmark (no GPU): the byte model of the stages and
the DRAM traffic figures it reads from profiles/traffic.json."""
from __future__ import annotations

import bench

COUNTS = {"clusters": 1_000_000, "tl_hits": 1_650_000, "tracklets": 38_000, "st_hits": 870_000,
          "sector_tracks": 21_000, "fit_hits": 860_000, "fit_tracks": 9_000,
          "fit_stations": 870_000, "re_hits": 0, "re_tracklets": 0, "seed_iters": 1}


def test_every_stage_has_a_byte_model():
    stages = ("grid", "links", "starts", "tracklets", "select", "sector_refit", "merge", "fit12",
              "ambiguity2", "fit3", "output")
    for s in stages:
        assert bench.stage_bytes(s, COUNTS) > 0, s
    # the later seeding iterations move nothing when they are off
    assert bench.stage_bytes("reseed", COUNTS) == 0
    more = dict(COUNTS, seed_iters=2, re_hits=100_000, re_tracklets=5_000)
    assert bench.stage_bytes("reseed", more) > 53 * COUNTS["clusters"]


def test_traffic_figures_come_from_the_committed_json():
    for stage in ("tracklets", "fit12", "fit3", "sector_refit", "links"):
        t, src = bench.measured_traffic(stage, COUNTS)
        assert t is not None and src, stage
        # DRAM bytes per cluster: above the stage's algorithmic bytes (re-reads),
        # below a few hundred bytes
        per = t / COUNTS["clusters"]
        assert 0.5 * bench.stage_bytes(stage, COUNTS) / COUNTS["clusters"] < per < 400.0, stage
    assert bench.measured_traffic("no_such_stage", COUNTS) == (None, None)


def test_whole_chain_traffic_is_at_least_the_algorithmic_bytes():
    t, src = bench.measured_traffic("chain", COUNTS)
    if t is None:  # no whole-chain capture committed, or marked stale
        return
    assert bench.CHAIN_BYTES_PER_CLUSTER * COUNTS["clusters"] < t < 2000 * COUNTS["clusters"]


def test_stale_figures_are_not_reported(tmp_path, monkeypatch):
    import json

    table = {"tracklets": {"bytes_per_cluster": 200.0, "kernels": "k", "workload": "w",
                           "stale": True}}
    monkeypatch.setattr(bench, "_traffic_table", lambda: table)
    assert bench.measured_traffic("tracklets", COUNTS) == (None, None)
    table["tracklets"].pop("stale")
    assert bench.measured_traffic("tracklets", COUNTS)[0] == 200.0 * COUNTS["clusters"]
    json.dumps(table)
