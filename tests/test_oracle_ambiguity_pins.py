"""Pins of the oracle's ranking decisions: the tracklet key of the first
ambiguity solving (Sec. 3 Phase I: smaller global chi2 gets priority), the
cluster pick of the track following (Sec. 2: the Kalman following takes the
best-fitting cluster of a row), and the second ambiguity solving over several
candidates per (track, row) (Sec. 3 Phase II).

Each pin fixes the decision from its definition, not from the oracle's own
outputs: keys recomputed from (n, chi2, ndf, start) and checked against which
tracklet actually owns shared clusters; a frame built by hand where a decoy
cluster lies inside the search window next to the true one; hand-made
candidate lists with known assignments, and a sequential restatement of the
K rounds over Python tuples on a full event.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import exact_row_x

RX = exact_row_x()
R = 152


def opts(**kw):
    o = TrackerOptions().as_dict()
    o.update(kw)
    return o


def ordered_bits(f32):
    u = np.asarray(f32, dtype=np.float32).view(np.uint32).astype(np.uint64)
    return np.where(u & 0x80000000, (~u) & 0xFFFFFFFF, u | 0x80000000)


# ------------------------------------------------------------- a6 tracklet key
def test_tracklet_key_follows_its_definition_and_prefers_small_chi2():
    """key = (ordered bits of the FP32 score n - w*chi2/ndf) << 32 | ~start;
    of two tracklets of equal length sharing a cluster, the one with the
    smaller chi2/ndf owns it."""
    f = synth.generate("central_event", n_primaries=3000)
    o = opts()
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), o)
    valid = np.nonzero(r["tl_n"] > 0)[0]
    n = r["tl_n"][valid].astype(np.float32)
    chi2 = r["tl_chi2"][valid].astype(np.float32)
    ndf = r["tl_ndf"][valid].astype(np.float32)
    assert np.array_equal(r["tl_ndf"][valid], 2 * r["tl_n"][valid] - 5)
    score = n - np.float32(o["score_w"]) * (chi2 / ndf)
    start = r["tl_start"][valid].astype(np.uint64)
    key = (ordered_bits(score) << np.uint64(32)) | (np.uint64(0xFFFFFFFF) - start)
    assert np.array_equal(key, r["tl_key"][valid].astype(np.uint64))

    # which tracklet owns a shared cluster: the accepted owner's start is
    # sector_owner; every other tracklet holding the cluster must rank lower
    score64 = n.astype(np.float64) - o["score_w"] * (chi2.astype(np.float64) / ndf)
    holders = {}
    for j, i in enumerate(valid):
        h = r["tl_hits"][i * R:(i + 1) * R]
        for c in h[h >= 0]:
            holders.setdefault(int(c), []).append(j)
    idx_of_start = {int(s): j for j, s in enumerate(r["tl_start"][valid])}
    own = r["sector_owner"]
    n_equal_len = n_checked = 0
    for c, js in holders.items():
        if len(js) < 2 or own[c] < 0:
            continue
        w = idx_of_start[int(own[c])]
        assert w in js
        for j in js:
            if j == w:
                continue
            n_checked += 1
            assert score64[j] <= score64[w] + 1e-4
            if n[j] == n[w] and abs(chi2[j] / ndf[j] - chi2[w] / ndf[w]) > 1e-3:
                n_equal_len += 1
                assert chi2[w] / ndf[w] < chi2[j] / ndf[j]
    assert n_checked > 1000 and n_equal_len > 50


# ------------------------------------------------------------- a5 pick-up
def _stiff_track_frame():
    """One stiff noise-free track in sector 0 with rows 50 and 51 emptied (the
    cellular automaton links adjacent rows only, so the track falls into two
    chains and the following has to bridge the gap), and a decoy beside the
    true cluster on rows 30-40 and 60-70: 0.15 cm off in y, inside the 3-sigma
    window (chi2 about 2 of the cut 9), farther than the true cluster."""
    g = synth.generate("one_sector", n_primaries=1, pt_min=3.0, pt_max=3.0, eta_min=0.2,
                       eta_max=0.2, sigma=0.0, noise_frac=0.0, seed=4242)
    keep = ~np.isin(g.row, [50, 51]) & (g.sector == 0)
    y, z, row, sec = g.y[keep], g.z[keep], g.row[keep], g.sector[keep]
    assert len(np.unique(row)) == len(row) and len(row) > 140
    dec = np.isin(row, list(range(30, 41)) + list(range(60, 71)))
    yy = np.concatenate([y, y[dec] + np.float32(0.15)]).astype(np.float32)
    zz = np.concatenate([z, z[dec]]).astype(np.float32)
    rr = np.concatenate([row, row[dec]]).astype(np.uint8)
    ss = np.concatenate([sec, sec[dec]]).astype(np.uint8)
    n_true = len(y)
    return yy, zz, rr, ss, n_true


def test_following_picks_the_best_cluster_of_the_window():
    yy, zz, rr, ss, n_true = _stiff_track_frame()
    o = opts(ms_theta=0.0)
    r = oracle.track(yy, zz, rr, ss, RX.astype(np.float32), o)
    valid = np.nonzero(r["tl_n"] > 0)[0]
    starts = r["tl_start"][valid]
    # the track's two chains start below and above the gap (the decoys of a
    # run of rows chain up among themselves and seed tracklets of their own)
    true_starts = [int(s) for s in starts if s < n_true]
    assert len(true_starts) == 2
    assert rr[min(true_starts, key=lambda s: rr[s])] < 30 and max(rr[true_starts]) > 51
    for s in true_starts:
        i = valid[list(starts).index(s)]
        h = r["tl_hits"][i * R:(i + 1) * R]
        h = h[h >= 0]
        # the following crossed the gap and covered the decoy rows ...
        rows = set(rr[h].tolist())
        assert rows >= set(range(30, 41)) | set(range(60, 71)), sorted(rows)
        # ... and took the true cluster on every one of them
        assert (h < n_true).all(), h[h >= n_true]


# --------------------------------------------------------- a10 second ambiguity
def _amb(tracks, K=4):
    """tracks: list of (key, [slot candidates as [(cluster, chi2), ...]])."""
    T = len(tracks)
    S = max(len(sl) for _, sl in tracks)
    key = np.array([k for k, _ in tracks], np.int32)
    ncand = np.zeros((T, S), np.int32)
    cand = np.full((T, S, K), -1, np.int32)
    chi2 = np.zeros((T, S, K), np.float32)
    for t, (_, slots) in enumerate(tracks):
        for s, cs in enumerate(slots):
            ncand[t, s] = len(cs)
            for k, (c, x2) in enumerate(cs):
                cand[t, s, k] = c
                chi2[t, s, k] = x2
    return oracle.second_ambiguity(key, ncand, cand, chi2)


def test_second_ambiguity_hand_made_cases():
    # a shared first choice goes to the smaller chi2; the loser takes its
    # second choice in the next round
    a = _amb([(10, [[(100, 2.0), (101, 3.0)]]), (20, [[(100, 1.0)]])])
    assert a.tolist() == [[101], [100]]
    # equal chi2: the smaller track key wins
    a = _amb([(20, [[(100, 1.0)]]), (10, [[(100, 1.0)]])])
    assert a.tolist() == [[-1], [100]]
    # rounds go by rank before chi2: a cluster given away as someone's first
    # choice in round 1 is not reassigned to a better second choice in round 2
    a = _amb([(1, [[(200, 5.0)]]),
              (2, [[(300, 0.7), (200, 0.1)]]),
              (3, [[(300, 0.5)]])])
    assert a.tolist() == [[200], [-1], [300]]
    # a slot served in an early round takes nothing later; one slot per row of
    # a track, several rows per track
    a = _amb([(1, [[(1, 0.5), (2, 0.6)], [(3, 0.4)]]),
              (2, [[(1, 0.2), (2, 0.3)], [(3, 0.9), (4, 1.0)]])])
    assert a.tolist() == [[2, 3], [1, 4]]
    # nothing offered, nothing assigned
    a = _amb([(5, [[]]), (6, [[(7, 1.0)]])])
    assert a.tolist() == [[-1], [7]]


def _sequential_restatement(slots, K):
    """slots: list of (track key, [(cluster, chi2 as float32), ...] best first).
    Round k: among slots still empty whose k-th candidate is still free, each
    such cluster goes to the lexicographically smallest (chi2, track key)."""
    assigned = [-1] * len(slots)
    taken = set()
    for k in range(K):
        best = {}
        for s, (tkey, cs) in enumerate(slots):
            if assigned[s] >= 0 or len(cs) <= k:
                continue
            c, x2 = cs[k]
            if c in taken:
                continue
            bid = (float(x2), tkey)
            if c not in best or bid < best[c][0]:
                best[c] = (bid, s)
        for c, (_, s) in best.items():
            assigned[s] = c
        taken |= set(best)
    return assigned


def test_second_ambiguity_equals_sequential_restatement_on_an_event():
    f = synth.generate("central_event", n_primaries=3000)
    o = opts()
    K = o["cand_k"]
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), o, full=True)
    ids = r["cand_ids"].reshape(-1, K)
    x2 = r["cand_chi2"].reshape(-1, K).astype(np.float32)
    slots = [(int(r["cand_key"][s]), [(int(ids[s, k]), x2[s, k]) for k in range(r["cand_n"][s])])
             for s in range(len(r["cand_n"]))]
    exp = _sequential_restatement(slots, K)
    assert np.array_equal(np.array(exp), r["cand_assigned"])
    # the event exercises contention: some clusters are offered by several tracks
    offered = {}
    for key, cs in slots:
        for c, _ in cs:
            offered.setdefault(c, set()).add(key)
    assert sum(len(v) > 1 for v in offered.values()) > 20
    assert sum(e >= 0 for e in exp) > 1000
