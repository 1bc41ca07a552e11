"""The configuration and definitions the paper fixes with printed numbers
(tests/golden/paper_values.txt, each with its section) against the library's
defaults, the generator's time-frame preset and the truth-matching helper."""
from __future__ import annotations

import inspect
import os

import numpy as np

from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests import helpers

HERE = os.path.dirname(os.path.abspath(__file__))


def paper_values():
    out = {}
    for line in open(os.path.join(HERE, "golden", "paper_values.txt")):
        if line.strip() and not line.startswith("#"):
            key, val = line.split()[:2]
            out[key] = float(val)
    return out


def test_paper_numbers_are_consistent():
    v = paper_values()
    # 50 kHz over a 100 us drift time is the stated average of 5 collisions
    assert v["collision_rate_khz"] * 1e3 * v["drift_time_us"] * 1e-6 == v["collisions_per_drift"]


def test_tracker_defaults_follow_the_paper():
    v = paper_values()
    o = TrackerOptions()
    assert o.n_sectors == v["tpc_halves"] * v["sectors_per_half"]
    assert o.shared_frac == v["shared_fraction_default"]
    assert o.inner_rows == v["inner_region_rows"]
    q = inspect.signature(helpers.quality).parameters
    assert q["min_findable"].default == v["findable_min_hits"]


def test_time_frame_preset_follows_the_paper():
    """The time-frame workload: collisions at 50 kHz over 2.8 ms, i.e. 140 on
    average, their times spread over the frame."""
    v = paper_values()
    f = synth.generate("timeframe", frame=0)
    t0 = np.unique(f.particles["t0"])
    mean = v["collision_rate_khz"] * 1e3 * v["time_frame_ms"] * 1e-3
    assert mean == 140.0
    assert abs(len(t0) - mean) < 4.5 * np.sqrt(mean)  # Poisson count of collisions
    assert t0.min() >= 0.0 and t0.max() < v["time_frame_ms"] * 1e3
