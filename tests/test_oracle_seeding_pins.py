"""Pins of the oracle's seeding iterations on leftover clusters (Sec. 3,
Phase III: the sector tracking's seeding runs again on the clusters left over
after the ambiguity solving).

The definition is checked directly: a later iteration must give exactly what
the single-iteration sector tracking gives on a frame that holds only the
leftover clusters (same order, ids renumbered), and it must leave the earlier
iterations' results untouched."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import exact_row_x, quality

RX = exact_row_x().astype(np.float32)
R = 152
TL_KEYS = ("tl_start", "tl_n", "tl_ndf", "tl_accept", "tl_nkept")
TL_ROWS = ("tl_hits", "tl_kept")
TL_BITS = ("tl_param", "tl_cov", "tl_chi2", "tl_x")


def opts(**kw):
    o = TrackerOptions().as_dict()
    o.update(kw)
    return o


def frame():
    # dense enough that first-pass ambiguities leave seedable clusters behind
    return synth.generate("central_event", n_primaries=2500, seed=31)


def taken_by(r, n, iters=(0,)):
    """Clusters kept by, or starting, an accepted tracklet of the given iterations."""
    used = np.zeros(n, bool)
    it = r["tl_iter"] if "tl_iter" in r else np.zeros(len(r["tl_start"]), np.int32)
    for i in np.nonzero(r["tl_accept"])[0]:
        if it[i] not in iters:
            continue
        k = r["tl_kept"][i * R:(i + 1) * R]
        used[k[k >= 0]] = True
        used[r["tl_start"][i]] = True
    return used


def test_first_iteration_unchanged_by_later_ones():
    f = frame()
    one = oracle.track(f.y, f.z, f.row, f.sector, RX, opts())
    two = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(seed_iters=2))
    m = two["tl_iter"] == 0
    assert m.sum() == len(one["tl_start"]) and (two["tl_iter"][m.sum():] == 1).all()
    for k in TL_KEYS:
        assert np.array_equal(two[k][m], one[k]), k
    for k in TL_ROWS:
        assert np.array_equal(two[k].reshape(-1, R)[m], one[k].reshape(-1, R)), k
    for k in TL_BITS:
        a = two[k].reshape(len(m), -1)[m]
        assert np.array_equal(a.view(np.uint32), one[k].reshape(len(a), -1).view(np.uint32)), k


def test_second_iteration_equals_tracking_the_leftover_clusters():
    f = frame()
    two = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(seed_iters=2))
    used = taken_by(two, f.n, iters=(0,))
    assert 0 < used.sum() < f.n
    keep = np.nonzero(~used)[0]  # leftover clusters, original order
    sub = oracle.track(f.y[keep], f.z[keep], f.row[keep], f.sector[keep], RX, opts())
    m = two["tl_iter"] == 1
    assert m.sum() == len(sub["tl_start"]) > 0
    # the later iteration's links are those of the leftover frame, -1 on taken clusters
    for k in ("link_up", "link_dn", "clean_up", "clean_dn"):
        want = np.full(f.n, -1, np.int32)
        s = sub[k]
        want[keep] = np.where(s >= 0, keep[np.maximum(s, 0)], -1)
        assert np.array_equal(two[k], want), k
    assert np.array_equal(two["tl_start"][m], keep[sub["tl_start"]])
    for k in ("tl_n", "tl_ndf", "tl_accept", "tl_nkept"):
        assert np.array_equal(two[k][m], sub[k]), k
    for k in TL_ROWS:
        a = two[k].reshape(-1, R)[m]
        b = sub[k].reshape(-1, R)
        assert np.array_equal(a, np.where(b >= 0, keep[np.maximum(b, 0)], -1)), k
    for k in TL_BITS:
        a = two[k].reshape(len(m), -1)[m]
        assert np.array_equal(a.view(np.uint32), sub[k].reshape(len(a), -1).view(np.uint32)), k
    # sector-level owners: the first iteration's on taken clusters, the
    # leftover frame's (mapped back) on the others
    one = oracle.track(f.y, f.z, f.row, f.sector, RX, opts())
    so = sub["sector_owner"]
    assert np.array_equal(two["sector_owner"][used], one["sector_owner"][used])
    assert np.array_equal(two["sector_owner"][keep], np.where(so >= 0, keep[np.maximum(so, 0)], -1))


def test_iterations_never_share_a_kept_cluster():
    f = frame()
    r = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(seed_iters=3))
    owner_iter = np.full(f.n, -1)
    for i in np.nonzero(r["tl_accept"])[0]:
        k = r["tl_kept"][i * R:(i + 1) * R]
        k = k[k >= 0]
        it = r["tl_iter"][i]
        assert np.all((owner_iter[k] == -1) | (owner_iter[k] == it))
        owner_iter[k] = it
    for it in (1, 2):
        prev = taken_by(r, f.n, iters=tuple(range(it)))
        for i in np.nonzero(r["tl_iter"] == it)[0]:
            h = r["tl_hits"][i * R:(i + 1) * R]
            assert not prev[h[h >= 0]].any()


def test_seeding_iterations_keep_quality():
    """Against generator truth the second iteration adds tracks and attached
    clusters without losing efficiency or raising the fake rate beyond the
    statistical noise of this event."""
    f = synth.generate("central_event", n_primaries=2500, seed=31)
    q = []
    for it in (1, 2):
        r = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(seed_iters=it), full=True)
        off, ids = r["trk_offset"], r["trk_ids"]
        q.append(quality(f.label, [ids[off[i]:off[i + 1]] for i in range(len(off) - 1)],
                         r["attach"]))
    print(q)
    assert q[1]["eff"] >= q[0]["eff"]
    assert q[1]["attached"] >= q[0]["attached"]
    assert q[1]["fake_rate"] < 0.005
