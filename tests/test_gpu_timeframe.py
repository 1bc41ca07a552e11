"""The benchmark's workload through the whole chain: one 2.8 ms, 50 kHz Pb-Pb
time frame (frame 0 of the `timeframe` preset, about 2e7 clusters, Poisson(140)
collisions spread over the frame in z, per-sector occupancy varying about 10x).

* strict mode: links, start hits, accepted tracklets, sector tracks and merge
  links, Phase II candidates and assignments, every output track and attach[]
  bit-exact against the oracle run on the whole frame;
* fast mode (the benchmark's mode): efficiency, fake rate and attached
  fraction within 0.2 points of the oracle, and the decision-by-decision
  comparison with strict mode of tests/fast_compare.py.

The oracle (single thread, about a minute) runs in a spawned process while the
GPU tracks the frame.
"""
from __future__ import annotations

import multiprocessing
from concurrent.futures import ProcessPoolExecutor

import numpy as np
import pytest

from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import quality

pytestmark = pytest.mark.gpu

RX = synth.row_x()


def _oracle_run(cols, opts):
    import oracle
    from tests.chain_compare import oracle_subset

    y, z, row, sec = cols
    return oracle_subset(oracle.track(y, z, row, sec, synth.row_x(), opts, full=True))


@pytest.fixture(scope="module")
def frame_and_oracle():
    f = synth.generate("timeframe", frame=0)
    opts = TrackerOptions().as_dict()
    ex = ProcessPoolExecutor(1, mp_context=multiprocessing.get_context("spawn"))
    fut = ex.submit(_oracle_run, (f.y, f.z, f.row, f.sector), opts)
    yield f, opts, fut
    ex.shutdown(wait=True, cancel_futures=True)


@pytest.fixture(scope="module")
def strict_run(frame_and_oracle):
    from paper_2601_20569_gb300 import tpc
    from tests import chain_compare as cc
    from tests import fast_compare as fc

    f, opts, _ = frame_and_oracle
    tr = tpc.Tracker(RX, opts, mode=0, cap_clusters=f.n)
    tr.track(*tr.to_device(f.y, f.z, f.q, f.row, f.sector))
    out = cc.gpu_state(tr)
    out["snap"] = fc.snapshot(tr)
    tr.close()
    return out


def test_full_timeframe_strict_bit_exact(frame_and_oracle, strict_run):
    from tests import chain_compare as cc

    f, opts, fut = frame_and_oracle
    info = cc.assert_chain_equal(strict_run, fut.result(), f.n, opts)
    print(f"time frame, strict mode bit-exact: {info}")


def test_full_timeframe_fast_mode(frame_and_oracle, strict_run):
    from paper_2601_20569_gb300 import tpc
    from tests import fast_compare as fc

    f, opts, fut = frame_and_oracle
    tr = tpc.Tracker(RX, opts, mode=1, cap_clusters=f.n)
    tr.track(*tr.to_device(f.y, f.z, f.q, f.row, f.sector))
    df = fc.snapshot(tr)
    tr.close()
    r = df["res"]
    off, ids = r["cl_offset"], r["cl_ids"]
    hits = [ids[off[i]:off[i + 1]] for i in range(len(r["key"]))]
    ref = fut.result()
    roff, rids = ref["trk_offset"], ref["trk_ids"]
    rhits = [rids[roff[i]:roff[i + 1]] for i in range(len(ref["trk_key"]))]
    qg = quality(f.label, hits, r["attach"])
    qr = quality(f.label, rhits, ref["attach"])
    print("fast", qg, "\noracle", qr)
    for k in ("eff", "fake_rate", "attached"):
        assert abs(qg[k] - qr[k]) <= 0.002, (k, qg, qr)
    c = fc.compare(strict_run["snap"], df)
    print(fc.summary(c))
    assert len(c["matched"]) >= 0.95 * c["n_common"], c["first"]
    rel, pull = c["rel"], c["pull"]
    assert (np.median(rel, axis=0) < 1e-4).all()
    # in units of the track's own uncertainty: tiny for almost every track; the
    # tail is short, poorly constrained tracks whose nonlinear fit amplifies
    # the rounding differences of its first steps
    worst = pull.max(axis=1)
    assert np.quantile(worst, 0.99) < 0.05 and np.quantile(worst, 0.999) < 0.3
    assert worst.max() < 2.0
