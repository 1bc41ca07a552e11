"""Fast against strict mode, track by track (test helper, no tracking
arithmetic): which discrete decision of the chain diverges first, and the
parameter differences of the tracks whose decisions all agree."""
from __future__ import annotations

import numpy as np

NAMES = ("y", "z", "snp", "tgl", "qpt")
# Relative differences |dp| / max(|p|, floor): below the floor a parameter is
# compared absolutely.  y and z are positions (cm) measured with 0.1 cm
# resolution, so 1e-4 of 1 cm is 1e-3 of the resolution; sin(phi) and
# tan(lambda) cross zero and are known to about 1e-3, so their floor is 0.01;
# q/pT's floor of 0.1 /GeV is pT = 10 GeV, the top of the spectrum.
FLOORS = np.array([1.0, 1.0, 0.01, 0.01, 0.1])
DIAG = [0, 2, 5, 9, 14]


def snapshot(tr) -> dict:
    """The per-track decisions and outputs of the last tracking call."""
    d = {k: tr.debug(k) for k in ("sid", "st_key", "st_ok", "st_next", "st_bestB", "st_bestchi",
                                  "ft_key", "ft_ok", "ft_nst", "ft_st_cl", "ft_flag",
                                  "ft_assigned")}
    d["res"] = {k: v.cpu().numpy() for k, v in tr.result().items()}
    return d


def per_track(d: dict) -> dict:
    sid = d["sid"]
    fk, nst = d["ft_key"], d["ft_nst"]
    nft = len(fk)
    cl = d["ft_st_cl"].reshape(nft, -1)
    fl = d["ft_flag"].reshape(nft, -1)
    asg = d["ft_assigned"].reshape(nft, -1)
    stk, nxt = d["st_key"], d["st_next"]
    idx = {int(k): i for i, k in enumerate(stk)}
    out = {}
    for t in range(nft):
        chain, s = [], idx.get(int(fk[t]), -1)
        while s >= 0 and len(chain) < 64:
            chain.append(int(stk[s]))
            s = int(nxt[s])
        n = int(nst[t])
        a = asg[t]
        out[int(fk[t])] = {"ok": int(d["ft_ok"][t]), "merge": tuple(chain),
                           "stations": tuple(np.where(cl[t, :n] >= 0, sid[np.maximum(cl[t, :n], 0)],
                                                      -1).tolist()),
                           "flags": tuple(fl[t, :n].tolist()),
                           "phase2": tuple(np.where(a >= 0, sid[np.maximum(a, 0)], -1).tolist())}
    r = d["res"]
    off, ids = r["cl_offset"], r["cl_ids"]
    for i, k in enumerate(r["key"]):
        o = out.setdefault(int(k), {})
        o["hits"] = tuple(ids[off[i]:off[i + 1]].tolist())
        o["par"] = r["params"][i].astype(np.float64)
        o["cov"] = r["cov"][i].astype(np.float64)
    return out


def merge_margin(ds: dict, df: dict, key: int, si: dict, fi: dict) -> dict:
    """At the first sector track of a chain whose merge link differs: the two
    modes' best partners and chi2 values (the cut is 30).  si / fi: sector
    track index by key in the strict and the fast snapshot."""
    a_s, a_f = si.get(key, -1), fi.get(key, -1)
    while a_s >= 0 and a_f >= 0:
        ns, nf = int(ds["st_next"][a_s]), int(df["st_next"][a_f])
        ks = int(ds["st_key"][ns]) if ns >= 0 else -1
        kf = int(df["st_key"][nf]) if nf >= 0 else -1
        if ks != kf:
            bs, bf = int(ds["st_bestB"][a_s]), int(df["st_bestB"][a_f])
            return {"best_same": (int(ds["st_key"][bs]) if bs >= 0 else -1) ==
                    (int(df["st_key"][bf]) if bf >= 0 else -1),
                    "chi2": (float(ds["st_bestchi"][a_s]), float(df["st_bestchi"][a_f]))}
        a_s = ns
        a_f = fi.get(ks, -1) if ks >= 0 else -1
    return {"best_same": True, "chi2": (0.0, 0.0)}


def compare(ds: dict, df: dict) -> dict:
    """Per-track comparison of a strict (ds) and a fast (df) snapshot."""
    S, F = per_track(ds), per_track(df)
    common = sorted(set(S) & set(F))
    si = {int(k): i for i, k in enumerate(ds["st_key"])}
    fi = {int(k): i for i, k in enumerate(df["st_key"])}
    first = {}
    matched, margins = [], []
    for k in common:
        a, b = S[k], F[k]
        why = next((n for n in ("ok", "merge", "stations", "flags", "phase2", "hits")
                    if a.get(n) != b.get(n)), None)
        first[why] = first.get(why, 0) + 1
        if why == "merge":
            margins.append(merge_margin(ds, df, k, si, fi))
        if why is None and "par" in a and "par" in b:
            matched.append(k)
    P = np.array([S[k]["par"] for k in matched]).reshape(-1, 5)
    Q = np.array([F[k]["par"] for k in matched]).reshape(-1, 5)
    C = np.array([S[k]["cov"] for k in matched]).reshape(-1, 15)
    D = np.abs(P - Q)
    rel = D / np.maximum(np.abs(P), FLOORS)
    pull = D / np.sqrt(C[:, DIAG])
    return {"n_strict": len(S), "n_fast": len(F), "n_common": len(common), "first": first,
            "matched": matched, "rel": rel, "pull": pull, "margins": margins,
            "strict": S, "fast": F}


def summary(c: dict) -> str:
    rel, pull = c["rel"], c["pull"]
    lines = [f"fit tracks: strict {c['n_strict']}, fast {c['n_fast']}, common {c['n_common']}; "
             f"first diverging decision: {c['first']}"]
    m = c["margins"]
    if m:
        same = sum(x["best_same"] for x in m)
        dchi = np.array([abs(x["chi2"][0] - x["chi2"][1]) for x in m])
        lines.append(f"merge divergences: {len(m)}, same best candidate in both modes {same} "
                     f"(a mutual-best pairing flipped by a neighbour), median |chi2_strict - "
                     f"chi2_fast| of the first differing link {np.median(dchi):.3g}")
    for j, nm in enumerate(NAMES):
        r = rel[:, j]
        lines.append(f"{nm:4s} rel median {np.median(r):.2e} p99 {np.quantile(r, .99):.2e} "
                     f"max {r.max():.2e} within 1e-4 {np.mean(r <= 1e-4):.4f}; pull p99 "
                     f"{np.quantile(pull[:, j], .99):.2e} max {pull[:, j].max():.2e}")
    lines.append(f"decision-matched tracks {len(c['matched'])}, all components within 1e-4: "
                 f"{np.mean((rel <= 1e-4).all(1)):.4f}; largest |dp|/sigma per track: p99.9 "
                 f"{np.quantile(pull.max(1), .999):.3f}, above 0.5 for "
                 f"{int((pull.max(1) > 0.5).sum())}")
    w = int(np.argmax(pull.max(1)))
    k = c["matched"][w]
    lines.append(f"largest difference: track {k}, {len(c['strict'][k]['hits'])} clusters, "
                 f"strict {c['strict'][k]['par'].tolist()} fast {c['fast'][k]['par'].tolist()}")
    return "\n".join(lines)
