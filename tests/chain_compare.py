"""Whole-chain strict parity of a GPU run against an oracle run (test helper,
vectorised for frames of millions of clusters): links, start hits, accepted
tracklets, sector tracks and merge links, Phase II candidates and
assignments, output tracks with their cluster lists, and attach[]."""
from __future__ import annotations

import numpy as np

DEBUG = ("sid", "lup", "ldn", "starts", "tl_acc", "st_key", "st_ok", "st_ie", "st_oe", "st_next",
         "ft_key", "ft_ok", "ft_nst", "ft_st_rs", "ft_ncand", "ft_cand", "ft_cchi", "ft_assigned")
ORACLE_KEYS = ("link_up", "link_dn", "start", "tl_accept", "st_key", "st_ie", "st_oe", "st_next",
               "attach")


def gpu_state(tr) -> dict:
    g = {k: tr.debug(k) for k in DEBUG}
    g["res"] = {k: v.cpu().numpy() for k, v in tr.result().items()}
    return g


def oracle_subset(r) -> dict:
    """The oracle outputs the comparison reads (keeps a pickled result small)."""
    return {k: v for k, v in r.items() if k in ORACLE_KEYS or k.startswith(("cand_", "trk_"))}


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def _csr(off, ids, order):
    lens = (off[1:] - off[:-1])[order]
    starts = off[:-1][order]
    idx = np.repeat(starts - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens) + \
        np.arange(lens.sum())
    return lens, ids[idx]


def assert_chain_equal(g: dict, ref: dict, n: int, opts: dict) -> dict:
    sid = g["sid"]
    # a2-a4: links (input-id space) and start hits
    up = np.full(n, -1, np.int64)
    dn = np.full(n, -1, np.int64)
    up[sid] = np.where(g["lup"] >= 0, sid[np.maximum(g["lup"], 0)], -1)
    dn[sid] = np.where(g["ldn"] >= 0, sid[np.maximum(g["ldn"], 0)], -1)
    assert np.array_equal(up, ref["link_up"]) and np.array_equal(dn, ref["link_dn"])
    assert np.array_equal(np.sort(sid[g["starts"]]), np.sort(ref["start"]))
    assert int(g["tl_acc"].sum()) == int(ref["tl_accept"].sum())
    # a7: sector tracks, their end states and merge links
    good = g["st_ok"] == 1
    st_key = g["st_key"]
    assert np.array_equal(np.sort(st_key[good]), ref["st_key"])
    gi = np.nonzero(good)[0][np.argsort(st_key[good])]
    ie = g["st_ie"].reshape(-1, 22)
    oe = g["st_oe"].reshape(-1, 22)
    assert np.array_equal(bits(ie[gi, :5]), bits(ref["st_ie"].reshape(-1, 5)))
    assert np.array_equal(bits(oe[gi, :5]), bits(ref["st_oe"].reshape(-1, 5)))
    nxt = g["st_next"][gi]
    assert np.array_equal(np.where(nxt >= 0, st_key[np.maximum(nxt, 0)], -1), ref["st_next"])
    # a10: Phase II candidates and assignments per (track, inner row)
    K = opts["cand_k"]
    fk, fok, nst = g["ft_key"], g["ft_ok"], g["ft_nst"]
    nft = len(fk)
    rs = g["ft_st_rs"].reshape(nft, -1)
    ns = g["ft_ncand"].size // max(nft, 1)
    nc = g["ft_ncand"].reshape(nft, ns).astype(np.int64)[:, :32]
    cand = g["ft_cand"].reshape(nft, ns, 8)[:, :32, :K]
    cchi = g["ft_cchi"].reshape(nft, ns, 8)[:, :32, :K]
    asg = g["ft_assigned"].reshape(nft, ns)[:, :32]
    T = np.nonzero(fok == 1)[0]
    m = (np.arange(32)[None, :] < np.minimum(nst[T], 32)[:, None]) & \
        ((rs[T, :32] % 152) < opts["inner_rows"])
    tt, ks = np.nonzero(m)
    t = T[tt]
    valid = np.arange(K)[None, :] < nc[t, ks][:, None]
    gcand = np.where(valid, sid[np.maximum(cand[t, ks], 0)], -1)
    gchi = np.where(valid, bits(cchi[t, ks]), 0)
    gas = np.where(asg[t, ks] >= 0, sid[np.maximum(asg[t, ks], 0)], -1)
    go = np.lexsort((rs[t, ks] % 152, fk[t]))
    rn = ref["cand_n"].astype(np.int64)
    rvalid = np.arange(K)[None, :] < rn[:, None]
    rcand = np.where(rvalid, ref["cand_ids"].reshape(-1, K), -1)
    rchi = np.where(rvalid, bits(ref["cand_chi2"].reshape(-1, K)), 0)
    ro = np.lexsort((ref["cand_row"], ref["cand_key"]))
    assert np.array_equal(fk[t][go], ref["cand_key"][ro])
    assert np.array_equal((rs[t, ks] % 152)[go], ref["cand_row"][ro])
    assert np.array_equal(nc[t, ks][go], rn[ro])
    assert np.array_equal(gcand[go], rcand[ro]) and np.array_equal(gchi[go], rchi[ro])
    assert np.array_equal(gas[go], ref["cand_assigned"][ro])
    # a11: output tracks by key and their cluster lists, attach[] by owner key
    r = g["res"]
    o = np.argsort(r["key"])
    assert np.array_equal(r["key"][o], ref["trk_key"])
    assert np.array_equal(bits(r["params"][o]), bits(ref["trk_param"].reshape(-1, 5)))
    assert np.array_equal(bits(r["cov"][o]), bits(ref["trk_cov"].reshape(-1, 15)))
    assert np.array_equal(bits(r["chi2"][o]), bits(ref["trk_chi2"]))
    assert np.array_equal(bits(r["x"][o]), bits(ref["trk_x"]))
    assert np.array_equal(r["ndf"][o], ref["trk_ndf"])
    assert np.array_equal(r["n_clusters"][o], ref["trk_ncl"])
    assert np.array_equal(r["sector"][o], ref["trk_sector"])
    lens, ids = _csr(r["cl_offset"], r["cl_ids"], o)
    assert np.array_equal(np.concatenate([[0], np.cumsum(lens)]), ref["trk_offset"])
    assert np.array_equal(ids, ref["trk_ids"])
    ga = r["attach"]
    gkey = np.where(ga >= 0, r["key"][np.maximum(ga, 0)], -1)
    ra = ref["attach"]
    assert np.array_equal(gkey, np.where(ra >= 0, ref["trk_key"][np.maximum(ra, 0)], -1))
    return {"clusters": n, "tracks": len(r["key"]), "sector_tracks": int(good.sum()),
            "phase2_rows": len(t)}


def track_lists(off, ids, n):
    return [ids[off[i]:off[i + 1]] for i in range(n)]
