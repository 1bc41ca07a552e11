"""Pins of the oracle's online cluster removal (Sec. 4: protective tubes
around physics tracks, removal tubes around secondary looper legs and very
low-pT tracks, protection of the seeding history, protection 2).

What fixes it independently of its own code: the generator's truth (which
leg of which particle a track follows), an all-pairs search for the tube
contents, set relations between the protection settings, and invariants of
the flag definition."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions

RX = synth.row_x()
TAN10 = np.float32(np.tan(np.deg2rad(10.0)))


def opts(**kw):
    o = TrackerOptions(cr_mode=1).as_dict()
    o.update(kw)
    return o


def looper_event(n=3000, seed=7):
    return synth.generate("central_event", n_primaries=n, looper_frac=0.2, seed=seed,
                          store_truth=True)


def majority(lab):
    lab = lab[lab >= 0]
    return int(np.bincount(lab).argmax()) if len(lab) else -1


def tracks(r):
    off, ids = r["trk_offset"], r["trk_ids"]
    return [ids[off[t]:off[t + 1]] for t in range(len(off) - 1)]


def test_secondary_legs_follow_generator_truth():
    f = looper_event()
    r = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(), full=True)
    hits = tracks(r)
    cls, par = r["cr_class"], r["cr_parent"]
    sec = np.nonzero(cls == 2)[0]
    assert len(sec) > 300
    good = 0
    for t in sec:
        a, b = majority(f.label[hits[t]]), majority(f.label[hits[par[t]]])
        good += a >= 0 and a // 2 == b // 2 and a % 2 == 1 and b % 2 == 0
    assert good >= 0.95 * len(sec), (good, len(sec))
    # parents come first: they are not secondary legs of the same link
    assert np.all(par[sec] != sec)
    # very low pT class = |q/pT| above the cut at the output parameters
    q = np.abs(r["trk_param"].reshape(-1, 5)[:, 4])
    low = q > np.float32(opts()["cr_qpt"])
    assert np.array_equal(cls == 1, low & (cls != 2))


def _brute_flags(f, r, o):
    """Flags by an all-pairs scan of every tube centre against every cluster."""
    y, z, row, sec = f.y, f.z, f.row.astype(np.int64), f.sector.astype(np.int64)
    flags = np.zeros(f.n, np.int64)
    cls = r["cr_class"]
    key = sec * 152 + row
    for t, h in enumerate(tracks(r)):
        protect = cls[t] == 0
        cents = []
        for i, c in enumerate(h):
            cents.append((sec[c], row[c], y[c], z[c]))
            if i + 1 == len(h):
                break
            d = h[i + 1]
            if sec[d] != sec[c]:
                continue
            lo, hi = (c, d) if row[c] < row[d] else (d, c)
            for rr in range(row[lo] + 1, row[hi]):
                fr = np.float32(rr - row[lo]) / np.float32(row[hi] - row[lo])
                cents.append((sec[c], rr, np.float32(y[lo] + (y[hi] - y[lo]) * fr),
                              np.float32(z[lo] + (z[hi] - z[lo]) * fr)))
        for s, rr, yc, zc in cents:
            on = key == s * 152 + rr
            h0 = np.float32(o["cr_protect"] if protect else o["cr_remove"])
            if o["cr_mode"] >= 2:
                w = np.float32(o["cr_occ_w"])
                occ = np.sum(on & (np.abs(y - yc) <= w) & (np.abs(z - zc) <= w))
                edge = np.abs(yc) > np.float32(RX[rr]) * TAN10 - np.float32(o["cr_edge"])
                if rr < o["inner_rows"] or edge or occ > o["cr_occ_max"]:
                    h0 = np.float32(h0 * np.float32(o["cr_p2_grow"] if protect else o["cr_p2_shrink"]))
            m = on & (np.abs(y - yc) <= h0) & (np.abs(z - zc) <= h0)
            flags[m] |= 1 if protect else 4
    return flags


@pytest.mark.parametrize("mode", [1, 2])
def test_tubes_equal_all_pairs_scan(mode):
    f = looper_event(n=250, seed=3)
    o = opts(cr_mode=mode)
    r = oracle.track(f.y, f.z, f.row, f.sector, RX, o, full=True)
    assert (r["cr_class"] > 0).any() and (r["cr_class"] == 0).any()
    got = r["cr_flags"] & 5
    want = _brute_flags(f, r, o)
    assert np.array_equal(got, want), np.nonzero(got != want)[0][:10]


def test_flag_invariants():
    f = looper_event(n=1500, seed=11)
    r = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(), full=True)
    fl = r["cr_flags"]
    rem = (fl & 8) != 0
    assert np.array_equal(rem, ((fl & 4) != 0) & ((fl & 3) == 0))
    cls = r["cr_class"]
    for t, h in enumerate(tracks(r)):
        assert np.all(fl[h] & (1 if cls[t] == 0 else 4)), t  # own clusters lie in own tube
    att = r["attach"]
    phys = (att >= 0) & (cls[np.maximum(att, 0)] == 0)
    assert not rem[phys].any()
    # seeding history: a subset of the clusters of accepted tracklets
    acc = np.nonzero(r["tl_accept"])[0]
    hits = r["tl_hits"].reshape(-1, 152)[acc]
    assert np.all(np.isin(np.nonzero(fl & 2)[0], hits[hits >= 0]))


def test_protection_settings_only_shrink_the_removed_set():
    f = looper_event(n=1500, seed=11)
    base = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(), full=True)["cr_flags"] & 8
    for kw in ({"cr_mode": 2}, {"cr_protect": 3.0}, {"cr_remove": 0.4}):
        other = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(**kw), full=True)["cr_flags"] & 8
        assert not np.any(other & ~base), kw
        assert other.sum() < base.sum(), kw


def test_removal_spares_physics_clusters_against_truth():
    f = looper_event()
    lab = f.label
    pt = f.particles["pt"]
    leg0 = (lab >= 0) & (lab % 2 == 0)
    phys = leg0 & (pt[np.maximum(lab // 2, 0)] >= 0.1)
    leg1 = (lab >= 0) & (lab % 2 == 1)
    for mode in (1, 2):
        fl = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(cr_mode=mode), full=True)["cr_flags"]
        rem = (fl & 8) != 0
        print(mode, rem[phys].mean(), rem[leg1].mean())
        assert rem[phys].mean() < 0.003 and rem[leg1].mean() > 0.25
