"""GPU merging, distortion-corrected three-iteration fit, Phase II attachment
and outputs vs the CPU oracle: bit-exact in strict mode; tolerances in fast
mode (parameters 1e-4 relative, efficiency and fake rate within 0.2 points)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import quality

pytestmark = pytest.mark.gpu

RX = synth.row_x()


def run_gpu(f, opts, mode=0, dist_map=None):
    import torch

    from paper_2601_20569_gb300 import tpc

    tr = tpc.Tracker(RX, opts, mode=mode, cap_clusters=max(f.n, 1024))
    if dist_map is not None:
        tr.set_map(torch.as_tensor(dist_map).cuda())
    tr.track(*tr.to_device(f.y, f.z, f.q, f.row, f.sector))
    torch.cuda.synchronize()
    return tr


def gpu_tracks(tr):
    res = {k: v.cpu().numpy() for k, v in tr.result().items()}
    off, ids = res["cl_offset"], res["cl_ids"]
    res["hits"] = [ids[off[i]:off[i + 1]] for i in range(len(res["key"]))]
    return res


def ref_tracks(r):
    off, ids = r["trk_offset"], r["trk_ids"]
    return [ids[off[i]:off[i + 1]] for i in range(len(r["trk_key"]))]


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)


def compare_full(tr, f, opts, dist_map=None):
    ref = oracle.track(f.y, f.z, f.row, f.sector, RX, opts, full=True, dist_map=dist_map)
    sid = tr.debug("sid")
    # a7: sector tracks, refit states and merge links
    st_key, st_ok = tr.debug("st_key"), tr.debug("st_ok")
    ie = tr.debug("st_ie").reshape(-1, 22)
    oe = tr.debug("st_oe").reshape(-1, 22)
    nxt = tr.debug("st_next")
    good = st_ok == 1
    assert np.array_equal(np.sort(st_key[good]), ref["st_key"])
    order = np.argsort(st_key[good])
    gi = np.nonzero(good)[0][order]
    assert np.array_equal(bits(ie[gi, :5]), bits(ref["st_ie"].reshape(-1, 5)))
    assert np.array_equal(bits(oe[gi, :5]), bits(ref["st_oe"].reshape(-1, 5)))
    nkey = np.where(nxt[gi] >= 0, st_key[np.maximum(nxt[gi], 0)], -1)
    assert np.array_equal(nkey, ref["st_next"])
    # a10: candidates and assignments per (track, inner row)
    fk = tr.debug("ft_key")
    fok = tr.debug("ft_ok")
    nst = tr.debug("ft_nst")
    rs = tr.debug("ft_st_rs").reshape(-1, 160)
    ns = 32 + 2 * opts.get("ext_rows", 0)  # inner-station slots, inward then outward rows
    nc = tr.debug("ft_ncand").reshape(-1, ns)
    cand = tr.debug("ft_cand").reshape(-1, ns, 8)
    cchi = tr.debug("ft_cchi").reshape(-1, ns, 8)
    asg = tr.debug("ft_assigned").reshape(-1, ns)
    K = opts["cand_k"]
    gpu_c = {}
    for t in np.nonzero(fok == 1)[0]:
        for k in range(min(nst[t], 32)):
            row = rs[t, k] % 152
            if row >= opts["inner_rows"]:
                continue
            ids = sid[cand[t, k, :nc[t, k]]]
            a = sid[asg[t, k]] if asg[t, k] >= 0 else -1
            gpu_c[(int(fk[t]), int(row))] = (ids.tolist(), bits(cchi[t, k, :nc[t, k]]).tolist(), a)
    ref_c = {}
    rc = ref["cand_ids"].reshape(-1, K)
    rx = ref["cand_chi2"].reshape(-1, K)
    for i in range(len(ref["cand_key"])):
        n = ref["cand_n"][i]
        ref_c[(int(ref["cand_key"][i]), int(ref["cand_row"][i]))] = (
            rc[i, :n].tolist(), bits(rx[i, :n]).tolist(), int(ref["cand_assigned"][i]))
    assert gpu_c == ref_c
    if opts.get("ext_rows", 0) > 0:
        # Phase III: rows extrapolated per track, candidates and assignments per row
        nxt = tr.debug("ft_next")
        nout = tr.debug("ft_nout")
        ok_ref = ref["fit_fail"] < 0
        assert np.array_equal(np.sort(nxt[fok == 1]), np.sort(ref["fit_next"][ok_ref]))
        assert np.array_equal(np.sort(nout[fok == 1]), np.sort(ref["fit_nout"][ok_ref]))
        E = opts["ext_rows"]
        xsec = tr.debug("ft_ext_sec").reshape(-1, 2 * E)
        gpu_e = {}
        for t in np.nonzero(fok == 1)[0]:
            r0 = rs[t, 0] % 152
            rl = rs[t, nst[t] - 1] % 152
            rows = [(32 + e, r0 - 1 - e, e) for e in range(nxt[t])] + \
                   [(32 + E + e, rl + 1 + e, E + e) for e in range(nout[t])]
            for s_, r_, j_ in rows:
                ids = sid[cand[t, s_, :nc[t, s_]]]
                a = sid[asg[t, s_]] if asg[t, s_] >= 0 else -1
                gpu_e[(int(fk[t]), int(r_))] = (int(xsec[t, j_]), ids.tolist(),
                                                bits(cchi[t, s_, :nc[t, s_]]).tolist(), a)
        ref_e = {}
        ec = ref["ext_ids"].reshape(-1, K)
        ex = ref["ext_chi2"].reshape(-1, K)
        for i in range(len(ref["ext_key"])):
            n = ref["ext_n"][i]
            ref_e[(int(ref["ext_key"][i]), int(ref["ext_row"][i]))] = (
                int(ref["ext_sector"][i]), ec[i, :n].tolist(), bits(ex[i, :n]).tolist(),
                int(ref["ext_assigned"][i]))
        assert gpu_e == ref_e
    # a11: output tracks by key, bit-exact
    g = gpu_tracks(tr)
    rk = ref["trk_key"]
    assert np.array_equal(np.sort(g["key"]), rk)
    o = np.argsort(g["key"])
    assert np.array_equal(bits(g["params"][o]), bits(ref["trk_param"].reshape(-1, 5)))
    assert np.array_equal(bits(g["cov"][o]), bits(ref["trk_cov"].reshape(-1, 15)))
    assert np.array_equal(bits(g["chi2"][o]), bits(ref["trk_chi2"]))
    assert np.array_equal(bits(g["x"][o]), bits(ref["trk_x"]))
    assert np.array_equal(g["ndf"][o], ref["trk_ndf"])
    assert np.array_equal(g["n_clusters"][o], ref["trk_ncl"])
    assert np.array_equal(g["sector"][o], ref["trk_sector"])
    rh = ref_tracks(ref)
    for j, t in enumerate(o):
        assert np.array_equal(g["hits"][t], rh[j])
    # attachments: owning track by key
    ga = g["attach"]
    gkey = np.where(ga >= 0, g["key"][np.maximum(ga, 0)], -1)
    ra = ref["attach"]
    rkey = np.where(ra >= 0, rk[np.maximum(ra, 0)], -1)
    assert np.array_equal(gkey, rkey)
    return ref, g


@pytest.mark.parametrize("workload,kw", [
    ("one_sector", {"ms_theta": 0.0}),
    ("central_event", {"n_primaries": 2500}),
])
def test_full_chain_bit_exact(workload, kw):
    f = synth.generate(workload, **{k: v for k, v in kw.items() if k != "ms_theta"})
    opts = TrackerOptions().as_dict()
    opts.update({k: v for k, v in kw.items() if k == "ms_theta"})
    tr = run_gpu(f, opts)
    compare_full(tr, f, opts)


def test_full_chain_bit_exact_with_distortion_map():
    """Space-charge distorted clusters corrected with the B-spline map (the
    differentiation workload's field), strict parity through fit and attachment."""
    f = synth.generate("central_event", n_primaries=2000, distort=True)
    opts = TrackerOptions().as_dict()
    tr = run_gpu(f, opts, dist_map=f.map)
    compare_full(tr, f, opts, dist_map=f.map)


def test_full_central_event_bit_exact():
    f = synth.generate("central_event")
    opts = TrackerOptions().as_dict()
    tr = run_gpu(f, opts)
    ref, g = compare_full(tr, f, opts)
    q = quality(f.label, g["hits"], g["attach"])
    assert q["eff"] > 0.99 and q["fake_rate"] < 0.01, q


def test_fast_mode_within_tolerance():
    """Fast mode (FMA contraction, hardware reciprocals) against strict mode on
    a central event, track by track: which discrete decision diverges first
    (merge links, fit stations, interpolation flags, Phase II assignments,
    final clusters), and for the tracks whose decisions all agree the parameter
    differences, relative (floors per component in tests/fast_compare.py) and
    in units of the track's own uncertainty; efficiency and fake rate within
    0.2 points of the oracle; and against the FP64 oracle, fast mode is as
    accurate as strict mode."""
    from tests import fast_compare as fc

    f = synth.generate("central_event", seed=808)
    opts = TrackerOptions().as_dict()
    ts = run_gpu(f, opts, mode=0)
    ds = fc.snapshot(ts)
    ts.close()
    tf = run_gpu(f, opts, mode=1)
    df = fc.snapshot(tf)
    g = gpu_tracks(tf)
    tf.close()
    c = fc.compare(ds, df)
    print(fc.summary(c))
    # decisions: most tracks take every decision alike; the rest part at a
    # merge link (chi2 values of candidates differ in the last bits)
    n_div = c["n_common"] - len(c["matched"])
    assert len(c["matched"]) >= 0.93 * c["n_common"], c["first"]
    assert c["first"].get("merge", 0) >= 0.8 * n_div
    rel, pull = c["rel"], c["pull"]
    assert (np.median(rel, axis=0) < 1e-5).all()
    assert np.mean((rel <= 1e-4).all(axis=1)) >= 0.95
    worst = pull.max(axis=1)
    assert np.quantile(worst, 0.99) < 0.05 and np.quantile(worst, 0.999) < 0.3
    assert worst.max() < 2.0
    # efficiency and fake rate against the strict oracle
    ref = oracle.track(f.y, f.z, f.row, f.sector, RX, opts, full=True)
    qg = quality(f.label, g["hits"], g["attach"])
    qr = quality(f.label, ref_tracks(ref), ref["attach"])
    assert abs(qg["eff"] - qr["eff"]) <= 0.002, (qg, qr)
    assert abs(qg["fake_rate"] - qr["fake_rate"]) <= 0.002, (qg, qr)
    # accuracy against the FP64 oracle on tracks with the same clusters in all
    # three: fast mode's errors are no larger than strict mode's
    r64 = oracle.track(f.y, f.z, f.row, f.sector, RX, opts, full=True, fp64=True)
    h64 = ref_tracks(r64)
    p64 = r64["trk_param"].reshape(-1, 5)
    k64 = {int(k): i for i, k in enumerate(r64["trk_key"])}
    es, ef = [], []
    for k in c["matched"]:
        i = k64.get(k)
        if i is None or tuple(h64[i].tolist()) != c["strict"][k]["hits"]:
            continue
        sig = np.sqrt(c["strict"][k]["cov"][fc.DIAG])
        es.append(np.abs(c["strict"][k]["par"] - p64[i]) / sig)
        ef.append(np.abs(c["fast"][k]["par"] - p64[i]) / sig)
    es, ef = np.array(es), np.array(ef)
    print(f"vs FP64 ({len(es)} tracks), |dp|/sigma median strict {np.median(es, 0)} fast "
          f"{np.median(ef, 0)}; p99 strict {np.quantile(es, .99, 0)} fast {np.quantile(ef, .99, 0)}")
    assert len(es) > 0.8 * len(c["matched"])
    assert (np.median(ef, 0) <= 1.5 * np.median(es, 0) + 1e-6).all()
    assert (np.quantile(ef, .99, 0) <= 1.5 * np.quantile(es, .99, 0) + 1e-4).all()


@pytest.mark.parametrize("kw", [{"n_primaries": 2500},
                                {"n_primaries": 3000, "looper_frac": 0.2, "distort": True}])
def test_edge_following_bit_exact(kw):
    """Edge following (Sec. 2): segments found in the adjacent sector beyond
    track ends at a sector edge, linked before the merging; the whole chain
    bit-exact against the oracle, with and without the distortion map."""
    f = synth.generate("central_event", **kw)
    opts = TrackerOptions(edge_rows=20).as_dict()
    dm = f.map if kw.get("distort") else None
    tr = run_gpu(f, opts, dist_map=dm)
    ref, g = compare_full(tr, f, opts, dist_map=dm)
    nseg = int((ref["st_key"] >= 1 << 29).sum())
    print(f"edge following: {nseg} segments")
    assert nseg > 100


class _Cut:
    """A frame without the clusters of rows lo..hi (generator arrays only)."""

    def __init__(self, f, lo, hi):
        keep = (f.row < lo) | (f.row > hi)
        self.y, self.z, self.q = f.y[keep], f.z[keep], f.q[keep]
        self.row, self.sector, self.label = f.row[keep], f.sector[keep], f.label[keep]
        self.n = int(keep.sum())


@pytest.mark.parametrize("workload,kw,cut", [
    ("one_sector", {"n_primaries": 150, "noise_frac": 0.0}, (8, 19)),
    ("one_sector", {"n_primaries": 150, "noise_frac": 0.0}, (132, 143)),
    ("central_event", {"n_primaries": 2500}, (8, 19)),
    ("central_event", {"n_primaries": 2500}, None),
])
def test_inward_extrapolation_bit_exact(workload, kw, cut):
    """Phase III: inward and outward extrapolation over 20 rows, their
    candidates, their assignment by the second ambiguity and the extended
    third iteration, strict parity (on frames with rows 8-19 or 132-143
    emptied, where the extrapolation has segments to find, and on a complete
    event)."""
    f = synth.generate(workload, **kw)
    if cut is not None:
        f = _Cut(f, *cut)
    opts = TrackerOptions(ext_rows=20).as_dict()
    tr = run_gpu(f, opts)
    ref, g = compare_full(tr, f, opts)
    if cut is not None:
        assert np.count_nonzero(ref["ext_assigned"] >= 0) > 0


def test_inward_extrapolation_bit_exact_with_distortion_map():
    f = synth.generate("central_event", n_primaries=1500, distort=True)
    opts = TrackerOptions(ext_rows=20).as_dict()
    tr = run_gpu(f, opts, dist_map=f.map)
    compare_full(tr, f, opts, dist_map=f.map)


@pytest.mark.parametrize("workload,kw", [
    ("central_event", {"n_primaries": 3000, "seed": 9, "vz_sigma": 10.0}),
    ("timeframe", {"mean_collisions": 4, "vz_sigma": 10.0}),
])
def test_central_electrode_merging_bit_exact(workload, kw):
    """Merging across the central electrode (collisions spread along z, so
    that some particles cross it): links, fits, attachments and the far
    side's z shift, strict parity; in continuous readout (the time-frame case)
    the shift carries the collision time."""
    f = synth.generate(workload, **kw)
    opts = TrackerOptions(ac_merge=1).as_dict()
    tr = run_gpu(f, opts)
    ref, g = compare_full(tr, f, opts)
    o = np.argsort(g["key"])
    assert np.array_equal(bits(g["z_shift"][o]), bits(ref["trk_zshift"]))
    assert np.count_nonzero(ref["trk_zshift"]) >= 2
