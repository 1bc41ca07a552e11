"""Sector-tracking iterations on leftover clusters (Sec. 3, Phase III
seeding) on the GPU against the oracle, strict FP32: bit-exact links of the
last iteration, tracklets of every iteration, selection and sector owners,
and the full chain after them; batched frames equal frames tracked alone."""
from __future__ import annotations

import numpy as np
import pytest

from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.test_gpu_batch import host, single_tracks, tracks_by_frame
from tests.test_gpu_fit import compare_full, run_gpu
from tests.test_gpu_sector import _run, compare_sector

pytestmark = pytest.mark.gpu

RX = synth.row_x()


@pytest.mark.parametrize("iters", [2, 3])
def test_seeding_iterations_sector_bit_exact(iters):
    f = synth.generate("central_event", n_primaries=2500, seed=31)
    opts = TrackerOptions(seed_iters=iters).as_dict()
    tr = _run(f.y, f.z, f.row, f.sector, opts)
    ref = compare_sector(tr, f.y, f.z, f.row, f.sector, opts)
    later = ref["tl_iter"] > 0
    assert later.any() and ref["tl_accept"][later].sum() > 0
    # taken clusters: exactly those kept by, or starting, an accepted tracklet
    # of an iteration before the last
    R = 152
    used = np.zeros(f.n, bool)
    for i in np.nonzero(ref["tl_accept"] & (ref["tl_iter"] < iters - 1))[0]:
        k = ref["tl_kept"][i * R:(i + 1) * R]
        used[k[k >= 0]] = True
        used[ref["tl_start"][i]] = True
    sid = tr.debug("sid")
    assert np.array_equal(tr.debug("sused")[np.argsort(sid)].astype(bool), used)


def test_seeding_iterations_full_chain_bit_exact():
    f = synth.generate("central_event", n_primaries=2500, seed=31)
    opts = TrackerOptions(seed_iters=2).as_dict()
    tr = run_gpu(f, opts)
    compare_full(tr, f, opts)


def test_seeding_iterations_batch_equals_frames_alone():
    from paper_2601_20569_gb300 import tpc

    frames = [synth.generate("central_event", n_primaries=1200, seed=41),
              synth.generate("central_event", n_primaries=700, seed=42)]
    ntot = sum(f.n for f in frames)
    opts = TrackerOptions(seed_iters=2).as_dict()
    tb = tpc.Tracker(RX, opts, mode=0, cap_clusters=ntot, max_frames=2, use_graphs=True)
    dev = [tb.to_device(f.y, f.z, f.q, f.row, f.sector) for f in frames]
    offsets = np.concatenate([[0], np.cumsum([f.n for f in frames])])
    for _ in range(2):  # capture, then replay
        tb.track_batch(dev)
        batch = tracks_by_frame(host(tb), offsets)
    ts = tpc.Tracker(RX, opts, mode=0, cap_clusters=max(f.n for f in frames))
    for i in range(len(frames)):
        ts.track(*dev[i])
        assert batch.get(i, {}) == single_tracks(host(ts)), i


def test_seed_iters_out_of_range_rejected():
    from paper_2601_20569_gb300 import tpc

    for bad in (-1, 5):
        with pytest.raises(tpc.TpcError):
            tpc.Tracker(RX, TrackerOptions(seed_iters=bad).as_dict(), cap_clusters=1024)


@pytest.mark.parametrize("lanes", [4, 8, 32])
def test_seeding_iterations_links_on_lane_groups(lanes):
    """The later iteration's neighbour search (taken clusters skipped) gives the
    same links, tracklets, owners and attachments on lane groups and staged per
    warp as on one lane per cluster."""
    from paper_2601_20569_gb300 import tpc

    f = synth.generate("central_event", n_primaries=1500, seed=33)
    opts = TrackerOptions(seed_iters=2).as_dict()
    names = ("lup", "ldn", "starts", "tl_n", "tl_par", "sec_owner", "attach")
    res = {}
    for ln in (1, lanes):
        tr = tpc.Tracker(RX, opts, mode=0, cap_clusters=f.n)
        cfg = tr.launch_config()
        tr.set_launch_config(cfg[:5] + [dict(cfg[5], lanes=ln)])
        assert tr.launch_config()[5]["lanes"] == ln
        tr.track(*tr.to_device(f.y, f.z, f.q, f.row, f.sector))
        res[ln] = {k: tr.debug(k) for k in names}
        tr.close()
    for k in names:
        assert np.array_equal(res[1][k].view(np.uint8), res[lanes][k].view(np.uint8)), (k, lanes)
