"""Online cluster removal (Sec. 4) on the GPU against the oracle, strict
FP32: per-cluster flags, track classes and looper-leg parents bit-exact, with
and without protection 2, after one and two seeding iterations; a batch gives
each frame's flags as tracked alone; call order and option errors."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions

pytestmark = pytest.mark.gpu

RX = synth.row_x()


def looper_event(n=3000, seed=7):
    return synth.generate("central_event", n_primaries=n, looper_frac=0.2, seed=seed)


def by_key(res, rem):
    """Class and parent key of every track, keyed by track key."""
    key = res["key"].cpu().numpy()
    cls = rem["track_class"].cpu().numpy()
    par = rem["leg_parent"].cpu().numpy()
    pk = np.where(par >= 0, key[np.maximum(par, 0)], -1)
    return {int(k): (int(c), int(p)) for k, c, p in zip(key, cls, pk)}


@pytest.mark.parametrize("mode,iters", [(1, 1), (2, 1), (2, 2)])
def test_removal_bit_exact(mode, iters):
    from paper_2601_20569_gb300 import tpc

    f = looper_event()
    opts = TrackerOptions(cr_mode=mode, seed_iters=iters).as_dict()
    tr = tpc.Tracker(RX, opts, mode=0, cap_clusters=f.n)
    tr.track(*tr.to_device(f.y, f.z, f.q, f.row, f.sector))
    rem = tr.cluster_removal(opts)
    ref = oracle.track(f.y, f.z, f.row, f.sector, RX, opts, full=True)
    flags = rem["flags"].cpu().numpy().astype(np.int32)
    assert np.array_equal(flags, ref["cr_flags"]), np.nonzero(flags != ref["cr_flags"])[0][:10]
    assert rem["n_removed"] == int(((ref["cr_flags"] & 8) != 0).sum()) > 0
    rk = ref["trk_key"]
    want = {int(k): (int(c), int(rk[p]) if p >= 0 else -1)
            for k, c, p in zip(rk, ref["cr_class"], ref["cr_parent"])}
    got = by_key(tr.result(), rem)
    assert got == want
    assert sum(c == 2 for c, _ in got.values()) > 100


def test_removal_batch_equals_frames_alone():
    from paper_2601_20569_gb300 import tpc

    frames = [looper_event(1500, 21), looper_event(900, 22)]
    ntot = sum(f.n for f in frames)
    opts = TrackerOptions(cr_mode=2).as_dict()
    tb = tpc.Tracker(RX, opts, mode=0, cap_clusters=ntot, max_frames=2)
    dev = [tb.to_device(f.y, f.z, f.q, f.row, f.sector) for f in frames]
    tb.track_batch(dev)
    fb = tb.cluster_removal(opts)["flags"].cpu().numpy()
    offsets = np.concatenate([[0], np.cumsum([f.n for f in frames])])
    ts = tpc.Tracker(RX, opts, mode=0, cap_clusters=max(f.n for f in frames))
    for i in range(len(frames)):
        ts.track(*dev[i])
        fa = ts.cluster_removal(opts)["flags"].cpu().numpy()
        assert np.array_equal(fb[offsets[i]:offsets[i + 1]], fa), i


def test_removal_call_order_and_options():
    from paper_2601_20569_gb300 import tpc

    f = looper_event(300, 5)
    opts = TrackerOptions(cr_mode=1).as_dict()
    tr = tpc.Tracker(RX, opts, mode=0, cap_clusters=f.n)
    with pytest.raises(tpc.TpcError) as e:
        tr.cluster_removal(opts)
    assert e.value.status == 7  # TPC_ERR_STATE: nothing tracked yet
    dev = tr.to_device(f.y, f.z, f.q, f.row, f.sector)
    tr.track(*dev)
    for bad in ({"cr_leg_dc": 0.0}, {"cr_protect": -1.0}, {"cr_qpt": 0.0}):
        o = dict(opts, **bad)
        with pytest.raises(tpc.TpcError) as e:
            tr.cluster_removal(o)
        assert e.value.status == 1
    with pytest.raises(tpc.TpcError):
        tr.cluster_removal(opts, mode=3)
    assert tr.cluster_removal(opts)["flags"].shape[0] == f.n
