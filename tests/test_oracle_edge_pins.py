"""Pins of the edge following (Sec. 2: tracks ending at a sector edge close to
the upper or lower end of the TPC are propagated into the adjacent sector
before the merging, and an extra track following picks up the short segment
the sector tracking cannot find), against the generator's truth.

* the short segments themselves: particles whose clusters lie in two
  adjacent sectors of one side, with fewer clusters in the second sector than
  the sector tracking accepts (min_hits) and all of them beyond the end of the
  first sector's part: without the edge following few of those clusters are
  attached to the particle's track, with it most are;
* every cluster the option attaches in addition belongs to the particle of
  the track it joins (checked at 99 %), lies in a sector adjacent to the
  sectors of that track's other clusters, and no attached cluster is
  lost; efficiency does not fall and the fake rate does not rise.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import exact_row_x, quality

RX = exact_row_x()


def _tracks(r):
    off, ids = r["trk_offset"], r["trk_ids"]
    return [ids[off[i]:off[i + 1]] for i in range(len(r["trk_key"]))]


def _majority(labels):
    v, c = np.unique(labels, return_counts=True)
    return int(v[c.argmax()])


@pytest.fixture(scope="module")
def runs():
    f = synth.generate("central_event", n_primaries=3000, seed=991)
    out = {}
    for er in (0, 20):
        o = TrackerOptions(edge_rows=er).as_dict()
        out[er] = oracle.track(f.y, f.z, f.row, f.sector, RX, o, full=True)
    return f, out


def _short_segments(f, min_hits):
    """Clusters of truth segments too short to seed: (cluster ids, label)."""
    segs = []
    order = np.argsort(f.label, kind="stable")
    lab = f.label[order]
    bounds = np.nonzero(np.diff(lab))[0] + 1
    for idx in np.split(order, bounds):
        L = int(f.label[idx[0]])
        if L < 0:
            continue
        secs, cnt = np.unique(f.sector[idx], return_counts=True)
        if len(secs) != 2:
            continue
        s_major, s_minor = (int(secs[0]), int(secs[1])) if cnt[0] >= cnt[1] else (int(secs[1]), int(secs[0]))
        if s_major // 18 != s_minor // 18 or (s_major - s_minor) % 18 not in (1, 17):
            continue
        mi = idx[f.sector[idx] == s_minor]
        ma = idx[f.sector[idx] == s_major]
        if not (3 <= len(mi) < min_hits) or len(ma) < 2 * min_hits:
            continue
        if f.row[mi].min() > f.row[ma].max() or f.row[mi].max() < f.row[ma].min():
            segs.append((mi, L))
    return segs


def test_short_segments_in_the_adjacent_sector_are_recovered(runs):
    f, r = runs
    o = TrackerOptions().as_dict()
    segs = _short_segments(f, o["min_hits"])
    assert len(segs) >= 30, len(segs)
    frac = {}
    for er, res in r.items():
        tk = _tracks(res)
        lab = np.array([_majority(f.label[h]) for h in tk])
        got = tot = 0
        for mi, L in segs:
            a = res["attach"][mi]
            got += int(((a >= 0) & (lab[np.maximum(a, 0)] == L)).sum())
            tot += len(mi)
        frac[er] = got / tot
    print(f"{len(segs)} short segments: attached to their particle's track "
          f"{frac[0]:.3f} without, {frac[20]:.3f} with the edge following")
    assert frac[0] < 0.35 and frac[20] > 0.75 and frac[20] > frac[0] + 0.4


def test_added_clusters_belong_to_the_track_and_the_adjacent_sector(runs):
    f, r = runs
    a0, a1 = r[0]["attach"] >= 0, r[20]["attach"] >= 0
    assert not (a0 & ~a1).sum() > 0.001 * a0.sum()
    new = np.nonzero(a1 & ~a0)[0]
    res = r[20]
    tk = _tracks(res)
    t_of = res["attach"][new]
    own = np.array([_majority(f.label[tk[t]]) for t in t_of]) == f.label[new]
    is_new = np.zeros(f.n, bool)
    is_new[new] = True
    adj = []
    for c, t in zip(new, t_of):
        h = tk[t]
        others = {int(s) for s in f.sector[h[~is_new[h]]]}
        sc = int(f.sector[c])
        adj.append(sc not in others and any(sc // 18 == s // 18 and (sc - s) % 18 in (1, 17)
                                            for s in others))
    adj = np.array(adj)
    print(f"{len(new)} clusters added, to their own particle's track {own.mean():.4f}, in a "
          f"sector adjacent to the sectors of the track's other clusters {adj.mean():.4f}")
    assert len(new) > 1000 and own.mean() > 0.99 and adj.mean() > 0.95
    q0 = quality(f.label, _tracks(r[0]), r[0]["attach"])
    q1 = quality(f.label, tk, res["attach"])
    assert q1["eff"] >= q0["eff"] and q1["fake_rate"] <= q0["fake_rate"] + 1e-4
    # segments are sector tracks of their own, after the tracklet keys
    assert (res["st_key"] >= 1 << 29).sum() > 100
