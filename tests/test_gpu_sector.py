"""GPU sector tracking vs the CPU oracle (strict FP32: bit-exact).

Covers the grid build, CA neighbour finding and cleaning, start hits, the
Kalman tracklet constructor and the ambiguity solving on frames that span many
grid bins and rows with ragged occupancy, an empty frame, a frame with
adversarial clusters on window edges, and input-error handling.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions

pytestmark = pytest.mark.gpu

RX = synth.row_x()


def _tracker(n, **kw):
    from paper_2601_20569_gb300 import tpc

    return tpc.Tracker(RX, kw.pop("opts", TrackerOptions().as_dict()), cap_clusters=max(n, 1024),
                       **kw)


def _run(y, z, row, sec, opts=None, mode=0, **kw):
    opts = opts or TrackerOptions().as_dict()
    tr = _tracker(len(y), opts=opts, mode=mode, **kw)
    dev = tr.to_device(y, z, np.zeros(len(y), np.uint16), row, sec)
    tr.track(*dev)
    return tr


def _to_id(sid, a):
    """Map a sorted-index array (values sorted indices or -1) to input-id space."""
    out = np.full(len(sid), -1, np.int64)
    out[sid] = np.where(a >= 0, sid[np.maximum(a, 0)], -1)
    return out


def compare_sector(tr, y, z, row, sec, opts, R=152):
    ref = oracle.track(y, z, row, sec, RX, opts)
    n = len(y)
    sid = tr.debug("sid")
    # a1: the sorted layout is a permutation grouped by (sector,row), bins in order
    assert np.array_equal(np.sort(sid), np.arange(n))
    srow = tr.debug("srow").astype(np.int64)
    assert np.array_equal(srow, sec[sid].astype(np.int64) * 152 + row[sid])
    assert np.all(np.diff(srow) >= 0)
    rows = tr.debug("rows")
    bf = tr.debug("bin_first")
    syz = tr.debug("syz")
    sy, sz = syz[0::2], syz[1::2]
    assert np.array_equal(sy, y[sid]) and np.array_equal(sz, z[sid])
    cl0 = np.concatenate([[0], np.cumsum(rows["ncl"].astype(np.int64))])
    for rr in np.nonzero(rows["ncl"])[0][:400]:
        g = rows[rr]
        k = np.arange(cl0[rr], cl0[rr] + g["ncl"])
        iy = np.clip(np.floor((sy[k] - g["y0"]) * g["invDy"]).astype(np.int64), 0, g["nY"] - 1)
        iz = np.clip(np.floor((sz[k] - g["z0"]) * g["invDz"]).astype(np.int64), 0, g["nZ"] - 1)
        b = g["bin0"] + iz * g["nY"] + iy
        assert np.all(bf[b] <= k) and np.all(k < bf[b + 1])
    # a2/a3: links by input id, exact
    for name, refname in (("lup", "link_up"), ("ldn", "link_dn"), ("cup", "clean_up"),
                          ("cdn", "clean_dn")):
        assert np.array_equal(_to_id(sid, tr.debug(name)), ref[refname]), name
    # a4
    starts = tr.debug("starts")
    st_id = sid[starts]
    assert np.array_equal(np.sort(st_id), np.sort(ref["start"]))
    # a5: tracklets keyed by (sector-tracking iteration, start id), bit-exact
    it_g = np.zeros(len(starts), np.int64)
    if opts.get("seed_iters", 1) > 1:
        ps = tr.debug("pass_start")[:opts["seed_iters"]]
        it_g = np.searchsorted(ps, np.arange(len(starts)), side="right") - 1
    order = {(int(i), int(s)): j for j, (i, s) in enumerate(zip(ref["tl_iter"], ref["tl_start"]))}
    tl_n = tr.debug("tl_n")
    par, cov = tr.debug("tl_par").reshape(-1, 5), tr.debug("tl_cov").reshape(-1, 15)
    chi2, x = tr.debug("tl_chi2"), tr.debug("tl_x")
    rlo, rhi = tr.debug("tl_rlo"), tr.debug("tl_rhi")
    hits = tr.debug("tl_hits").reshape(-1, 160)
    acc, nk = tr.debug("tl_acc"), tr.debug("tl_nkept")
    kept = tr.debug("tl_kept").reshape(-1, 160)
    rpar, rcov = ref["tl_param"].reshape(-1, 5), ref["tl_cov"].reshape(-1, 15)
    rhits, rkept = ref["tl_hits"].reshape(-1, R), ref["tl_kept"].reshape(-1, R)
    for gi, s in enumerate(st_id):
        oi = order[(int(it_g[gi]), int(s))]
        assert tl_n[gi] == ref["tl_n"][oi], (s, tl_n[gi], ref["tl_n"][oi])
        if tl_n[gi] == 0:
            continue
        assert np.array_equal(par[gi].view(np.uint32), rpar[oi].view(np.uint32)), s
        assert np.array_equal(cov[gi].view(np.uint32), rcov[oi].view(np.uint32)), s
        assert chi2[gi].view(np.uint32) == ref["tl_chi2"][oi].view(np.uint32)
        assert x[gi] == ref["tl_x"][oi]
        h = hits[gi, rlo[gi]:rhi[gi] + 1][::-1]
        h = sid[h[h >= 0]]
        rh = rhits[oi][rhits[oi] >= 0]
        assert np.array_equal(h, rh), s
        # a6
        assert acc[gi] == ref["tl_accept"][oi]
        assert nk[gi] == ref["tl_nkept"][oi]
        if acc[gi]:
            assert np.array_equal(sid[kept[gi, :nk[gi]]], rkept[oi][:nk[gi]])
    owner = tr.debug("sec_owner")
    own_id = np.full(n, -1, np.int64)
    own_id[sid] = np.where(owner >= 0, st_id[np.maximum(owner, 0)], -1)
    assert np.array_equal(own_id, ref["sector_owner"])
    return ref


@pytest.mark.parametrize("workload,kw", [
    ("one_sector", {}),
    ("one_sector", {"shuffle": True, "seed": 3}),
    ("central_event", {"n_primaries": 2500}),
])
def test_sector_tracking_bit_exact(workload, kw):
    f = synth.generate(workload, **kw)
    opts = TrackerOptions().as_dict()
    if workload == "one_sector":
        opts["ms_theta"] = 0.0
    tr = _run(f.y, f.z, f.row, f.sector, opts)
    compare_sector(tr, f.y, f.z, f.row, f.sector, opts)


def test_sector_tracking_bit_exact_full_central_event():
    f = synth.generate("central_event")
    opts = TrackerOptions().as_dict()
    tr = _run(f.y, f.z, f.row, f.sector, opts)
    compare_sector(tr, f.y, f.z, f.row, f.sector, opts)


def test_adversarial_edges_and_small_rows():
    from tests.test_oracle_pins import _tiny_frame

    y, z, row, sec = _tiny_frame(7)
    opts = TrackerOptions().as_dict()
    tr = _run(y, z, row, sec, opts)
    compare_sector(tr, y, z, row, sec, opts)


def test_empty_frame():
    opts = TrackerOptions().as_dict()
    e = np.zeros(0, np.float32)
    tr = _run(e, e, np.zeros(0, np.uint8), np.zeros(0, np.uint8), opts)
    assert tr.debug("starts").size == 0


def test_deterministic_rerun():
    f = synth.generate("central_event", n_primaries=1500, shuffle=True)
    opts = TrackerOptions().as_dict()
    a = _run(f.y, f.z, f.row, f.sector, opts)
    b = _run(f.y, f.z, f.row, f.sector, opts)
    for name in ("sid", "lup", "starts", "tl_par", "tl_cov", "tl_hits", "tl_kept", "sec_owner"):
        x, y_ = a.debug(name), b.debug(name)
        if name == "tl_hits" or name == "tl_kept":
            continue  # rows outside a tracklet's range are not written
        assert np.array_equal(x.view(np.uint8), y_.view(np.uint8)), name


def test_invalid_input_rejected():
    from paper_2601_20569_gb300 import tpc

    f = synth.generate("one_sector", n_primaries=20)
    y = f.y.copy()
    y[5] = np.nan
    with pytest.raises(tpc.TpcError) as e:
        _run(y, f.z, f.row, f.sector)
    assert e.value.status == 2
    row = f.row.copy()
    row[3] = 200
    with pytest.raises(tpc.TpcError) as e:
        _run(f.y, f.z, row, f.sector)
    assert e.value.status == 2


def test_capacity_errors_report_needed_size():
    from paper_2601_20569_gb300 import tpc

    f = synth.generate("one_sector")
    tr = tpc.Tracker(RX, TrackerOptions(), cap_clusters=1024)
    dev = tr.to_device(f.y, f.z, f.q, f.row, f.sector)
    with pytest.raises(tpc.TpcError) as e:
        tr.track(*dev)
    assert e.value.status == 3 and e.value.needed == f.n
    tr2 = tpc.Tracker(RX, TrackerOptions(), cap_clusters=f.n, cap_tracklets=5)
    with pytest.raises(tpc.TpcError) as e:
        tr2.track(*tr2.to_device(f.y, f.z, f.q, f.row, f.sector))
    assert e.value.status == 3 and e.value.needed > 5


def test_clusters_piled_on_one_point_rejected():
    """Thousands of clusters at one point of a row cannot come from the
    detector; the grid build rejects the frame instead of ordering one huge
    bin."""
    from paper_2601_20569_gb300 import tpc

    f = synth.generate("one_sector", n_primaries=20)
    n = 5000
    y = np.concatenate([f.y, np.full(n, 1.5, np.float32)])
    z = np.concatenate([f.z, np.full(n, 10.0, np.float32)])
    row = np.concatenate([f.row, np.full(n, 30, np.uint8)])
    sec = np.concatenate([f.sector, np.full(n, f.sector[0], np.uint8)])
    with pytest.raises(tpc.TpcError) as e:
        _run(y, z, row, sec)
    assert e.value.status == 2
