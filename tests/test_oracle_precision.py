"""Precision of the FP32 chain against the FP64 chain (oracle builds).

The strict GPU path equals the FP32 oracle bit for bit (the GPU parity
tests), so these numbers are also the GPU's error against FP64.  Workload: a
central event with 20 % loopers (pT 0.06-0.15 GeV) and the B-spline
space-charge distortion, i.e. the high-occupancy stress frame scaled down to
3,000 primaries.  Three builds: FP32 with the FP64 looper update (the
product), FP32 throughout (looper_qpt = 0) and FP64 throughout.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import exact_row_x, quality

RX = exact_row_x()
DIAG = [0, 2, 5, 9, 14]


def _tracks(r):
    off, ids = r["trk_offset"], r["trk_ids"]
    return [ids[off[i]:off[i + 1]] for i in range(len(off) - 1)]


def _errors(r, ref, looper_qpt):
    """max_k |p_k - p64_k| / sigma64_k per track with the same clusters as the
    FP64 track of the same key, and whether the FP64 track is a looper."""
    rk = {int(k): i for i, k in enumerate(ref["trk_key"])}
    rt, tt = _tracks(ref), _tracks(r)
    rp, rc = ref["trk_param"].reshape(-1, 5), ref["trk_cov"].reshape(-1, 15)
    p = r["trk_param"].reshape(-1, 5)
    err, loop = [], []
    for t, k in enumerate(r["trk_key"]):
        i = rk.get(int(k))
        if i is None or not np.array_equal(tt[t], rt[i]):
            continue
        err.append(float((np.abs(p[t].astype(np.float64) - rp[i]) / np.sqrt(rc[i][DIAG])).max()))
        loop.append(abs(rp[i][4]) > looper_qpt)
    return np.array(err), np.array(loop), len(tt)


def test_fp32_chain_against_fp64():
    f = synth.generate("central_event", n_primaries=3000, looper_frac=0.2, distort=True,
                       store_truth=True, seed=77)
    o = TrackerOptions().as_dict()
    runs = {
        "fp32 + fp64 looper update": oracle.track(f.y, f.z, f.row, f.sector, RX, o, full=True,
                                                  dist_map=f.map),
        "fp32 throughout": oracle.track(f.y, f.z, f.row, f.sector, RX, dict(o, looper_qpt=0.0),
                                        full=True, dist_map=f.map),
        "fp64": oracle.track(f.y, f.z, f.row, f.sector, RX, o, full=True, dist_map=f.map,
                             fp64=True),
    }
    q = {k: quality(f.label, _tracks(r), r["attach"]) for k, r in runs.items()}
    ref = runs["fp64"]
    stats = {}
    for name in ("fp32 + fp64 looper update", "fp32 throughout"):
        err, loop, n = _errors(runs[name], ref, o["looper_qpt"])
        stats[name] = (err, loop, n)
        print(f"{name}: eff {q[name]['eff']:.5f} fake {q[name]['fake_rate']:.5f} "
              f"(fp64: {q['fp64']['eff']:.5f} / {q['fp64']['fake_rate']:.5f}); "
              f"{len(err)} of {n} tracks with the fp64 clusters")
        for sel, lab in ((~loop, "non-loopers"), (loop, "loopers")):
            e = err[sel]
            print(f"   {lab:11s} max|dp|/sigma: median {np.median(e):.2e}  "
                  f"p99 {np.percentile(e, 99):.2e}  max {e.max():.2e}")
        # discrete results: efficiency and fake rate as in FP64
        assert abs(q[name]["eff"] - q["fp64"]["eff"]) <= 0.002
        assert abs(q[name]["fake_rate"] - q["fp64"]["fake_rate"]) <= 0.002
        assert len(err) >= 0.98 * n
        # parameters: FP32 rounding is a small fraction of the fit's own error
        assert np.median(err) < 1e-3 and err.max() < 0.25
    # the FP64 update of loopers reduces their error against FP64
    e_mix, l_mix, _ = stats["fp32 + fp64 looper update"]
    e_32, l_32, _ = stats["fp32 throughout"]
    assert np.percentile(e_mix[l_mix], 99) < np.percentile(e_32[l_32], 99)
    assert np.median(e_mix[l_mix]) < np.median(e_32[l_32])
