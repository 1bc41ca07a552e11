"""Pins of the CPU oracle against what the mathematics and the generated truth fix.

Nothing here compares the oracle with itself: closed-form helix geometry from
the generator (exact circle/line intersections), the information form of the
Kalman update, finite-difference Jacobians, brute force over all cluster pairs
on tiny frames, a greedy sequential restatement of the ambiguity solving, pull
statistics and efficiency against generated truth.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import exact_row_x, quality

RX = exact_row_x()


def opts(**kw):
    o = TrackerOptions().as_dict()
    o.update(kw)
    return o


def clean_frame(n=300, **kw):
    p = dict(n_primaries=n, noise_frac=0.0, sigma=0.0, ms_theta=0.0, sec_frac=0.0)
    p.update(kw)
    return synth.generate("central_event", store_truth=True, seed=777, **p)


def truth_state(f, i):
    return np.array([f.truth["y"][i], f.truth["z"][i], f.truth["snp"][i], f.truth["tgl"][i],
                     f.truth["qpt"][i]])


# --------------------------------------------------------------------- generator
def test_philox_known_answers():
    # Published Philox4x32-10 known-answer vectors (Salmon et al., Random123).
    assert synth.philox4x32_10([0, 0, 0, 0], [0, 0]).tolist() == [
        0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8]
    assert synth.philox4x32_10([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2).tolist() == [
        0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD]
    assert synth.philox4x32_10([0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344],
                               [0xA4093822, 0x299F31D0]).tolist() == [
        0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1]


def test_generator_reproducible_and_thread_independent():
    a = synth.generate("central_event", n_primaries=500, n_threads=1)
    b = synth.generate("central_event", n_primaries=500, n_threads=4)
    for k in ("y", "z", "row", "sector", "label", "q"):
        assert np.array_equal(getattr(a, k), getattr(b, k))


# ------------------------------------------------------------- helix geometry
def _pairs(f):
    lab = f.label
    same = (lab[1:] == lab[:-1]) & (lab[1:] >= 0)
    return np.nonzero(same)[0]


def test_propagation_matches_closed_form_helix_fp64():
    """Sec. 2 track following propagates seeds row by row: the FP64 helix step
    reproduces the generator's exact circle/line crossings (same sector) and,
    after the frame rotation, the crossings in the adjacent sector."""
    f = clean_frame()
    o = opts(ms_theta=0.0)
    err_same, err_rot, n_same, n_rot = 0.0, 0.0, 0, 0
    for i in _pairs(f):
        j = i + 1
        s0, s1 = int(f.sector[i]), int(f.sector[j])
        if s0 // 18 != s1 // 18:
            continue
        p = truth_state(f, i)
        if max(abs(p[2]), abs(f.truth["snp"][j])) > 0.9:
            continue  # outside the |sin(phi)| < 0.95 domain of the sector model
        c = np.zeros(15)
        x0 = RX[f.row[i]]
        if s0 != s1:
            d = ((s1 % 18) - (s0 % 18)) % 18
            direction = 1 if d == 1 else (-1 if d == 17 else 0)
            if direction == 0:
                continue
            # the truth state is in the direction of motion; the rotation
            # direction relative to the track frame flips for reversed legs
            r = oracle.rotate(p, c, x0, direction, RX, o)
            if r is None:
                continue
            p, c, x0 = r
            out = oracle.propagate(p, c, x0, RX[f.row[j]], RX, o)
            if out is None:
                continue
            err_rot = max(err_rot, np.max(np.abs(out[0][:3] - truth_state(f, j)[:3])))
            n_rot += 1
        else:
            out = oracle.propagate(p, c, x0, RX[f.row[j]], RX, o)
            assert out is not None
            err_same = max(err_same, np.max(np.abs(out[0][:3] - truth_state(f, j)[:3])))
            n_same += 1
    assert n_same > 10000 and n_rot > 50
    assert err_same < 1e-11, err_same
    assert err_rot < 1e-10, err_rot


def test_propagation_long_steps_fp64_and_fp32():
    """Steps over 1..40 rows: FP64 exact to 1e-10 cm; strict FP32 within a few
    ULP of the path (1e-3 cm over 40 rows)."""
    f = clean_frame(n=100)
    o = opts(ms_theta=0.0)
    lab = f.label
    worst64, worst32 = 0.0, 0.0
    for leg in np.unique(lab[lab >= 0])[:60]:
        idx = np.nonzero(lab == leg)[0]
        for gap in (1, 7, 40):
            for a in range(0, len(idx) - gap, 11):
                i, j = idx[a], idx[a + gap]
                if f.sector[i] != f.sector[j] or np.any(f.sector[idx[a:a + gap + 1]] != f.sector[i]):
                    continue
                p = truth_state(f, i)
                if np.max(np.abs(f.truth["snp"][idx[a:a + gap + 1]])) > 0.9:
                    continue
                c = np.zeros(15)
                r64 = oracle.propagate(p, c, RX[f.row[i]], RX[f.row[j]], RX, o, fp64=True)
                r32 = oracle.propagate(p, c, RX[f.row[i]], RX[f.row[j]], RX.astype(np.float32), o,
                                       fp64=False)
                if r64 is None:
                    continue
                t = truth_state(f, j)
                worst64 = max(worst64, np.max(np.abs(r64[0][:2] - t[:2])))
                worst32 = max(worst32, np.max(np.abs(r32[0][:2] - t[:2])))
    assert worst64 < 1e-10, worst64
    assert worst32 < 1e-3, worst32


def test_seed_recovers_exact_helix_fp64():
    f = clean_frame(n=100)
    o = opts()
    lab = f.label
    n = 0
    for leg in np.unique(lab[lab >= 0])[:80]:
        idx = np.nonzero(lab == leg)[0]
        if len(idx) < 30:
            continue
        sel = idx[[0, 10, 20]]
        if len(set(f.sector[sel])) != 1 or not np.all(np.diff(f.row[sel].astype(int)) > 0):
            continue
        pts = [(RX[f.row[k]], f.truth["y"][k], f.truth["z"][k]) for k in sel]
        s = oracle.seed(pts, RX, o)
        assert s is not None
        t = truth_state(f, sel[0])
        assert abs(s[0][2] - t[2]) < 1e-9
        assert abs(s[0][3] - t[3]) < 1e-9
        assert abs(s[0][4] - t[4]) < 1e-8 * max(1.0, abs(t[4]))
        n += 1
    assert n > 10


# --------------------------------------------------------------- Kalman algebra
def _full(c15):
    m = np.zeros((5, 5))
    m[np.tril_indices(5)] = c15
    return m + np.tril(m, -1).T


def _tri(m):
    return m[np.tril_indices(5)]


def test_update_equals_information_form():
    rng = np.random.default_rng(1)
    o = opts(sigma_y=0.1, sigma_z=0.15)
    for _ in range(50):
        a = rng.normal(size=(5, 5))
        P = a @ a.T + 0.1 * np.eye(5)
        x = rng.normal(size=5) * 0.1
        m = rng.normal(size=2)
        p1, c1, chi2 = oracle.update(x, _tri(P), m[0], m[1], RX, o)
        H = np.zeros((2, 5))
        H[0, 0] = H[1, 1] = 1
        sy, sz = float(np.float32(0.1)), float(np.float32(0.15))  # options travel as float32
        R = np.diag([sy ** 2, sz ** 2])
        Pi = np.linalg.inv(np.linalg.inv(P) + H.T @ np.linalg.inv(R) @ H)
        xi = Pi @ (np.linalg.solve(P, x) + H.T @ np.linalg.solve(R, m))
        r = m - H @ x
        chi = r @ np.linalg.solve(H @ P @ H.T + R, r)
        assert np.allclose(p1, xi, rtol=1e-9, atol=1e-12)
        assert np.allclose(_full(c1), Pi, rtol=1e-8, atol=1e-12)
        assert abs(chi2 - chi) < 1e-9 * max(1, chi)


def _fd_jacobian(fn, p, h):
    base = fn(p)
    J = np.zeros((5, 5))
    for k in range(5):
        dp = np.zeros(5)
        dp[k] = h[k]
        J[:, k] = (fn(p + dp) - fn(p - dp)) / (2 * h[k])
    return base, J


@pytest.mark.parametrize("dx", [1.06, 10.0, -5.0])
def test_covariance_transport_matches_finite_difference_jacobian(dx):
    """The covariance moves with the derivative of the helix step; checked
    against central differences."""
    o = opts(ms_theta=0.0)
    rng = np.random.default_rng(2)
    for _ in range(20):
        p = np.array([rng.uniform(-10, 10), rng.uniform(-50, 50), rng.uniform(-0.6, 0.6),
                      rng.uniform(-1, 1), rng.uniform(-5, 5)])
        x0 = 120.0

        def fn(q):
            r = oracle.propagate(q, np.zeros(15), x0, x0 + dx, RX, o)
            return r[0]

        _, J = _fd_jacobian(fn, p, [1e-4, 1e-4, 1e-6, 1e-6, 1e-5])
        a = rng.normal(size=(5, 5))
        P = a @ a.T * 0.01 + 1e-3 * np.eye(5)
        r = oracle.propagate(p, _tri(P), x0, x0 + dx, RX, o)
        expect = J @ P @ J.T
        assert np.allclose(_full(r[1]), expect, rtol=1e-5, atol=1e-8)


def test_rotation_geometry_and_jacobian():
    o = opts(ms_theta=0.0)
    rng = np.random.default_rng(3)
    a = math.radians(20.0)
    for _ in range(20):
        p = np.array([rng.uniform(-20, 20), rng.uniform(-50, 50), rng.uniform(-0.5, 0.5),
                      rng.uniform(-1, 1), rng.uniform(-3, 3)])
        x0 = rng.uniform(90, 240)
        r = oracle.rotate(p, np.zeros(15), x0, 1, RX, o)
        assert r is not None
        pn, _, xn = r
        # the same point in the rotated frame
        assert abs(xn - (x0 * math.cos(a) + p[0] * math.sin(a))) < 1e-9
        assert abs(pn[0] - (-x0 * math.sin(a) + p[0] * math.cos(a))) < 1e-9
        phi = math.asin(p[2])
        assert abs(pn[2] - math.sin(phi - a)) < 1e-12

        # Jacobian at fixed target x: rotate, then propagate to the rotated x of p
        def fn(q):
            rr = oracle.rotate(q, np.zeros(15), x0, 1, RX, o)
            out = oracle.propagate(rr[0], np.zeros(15), rr[2], xn, RX, o)
            return out[0]

        _, J = _fd_jacobian(fn, p, [1e-5, 1e-5, 1e-7, 1e-7, 1e-6])
        A = rng.normal(size=(5, 5))
        P = A @ A.T * 0.001 + 1e-4 * np.eye(5)
        rr = oracle.rotate(p, _tri(P), x0, 1, RX, o)
        assert np.allclose(_full(rr[1]), J @ P @ J.T, rtol=1e-4, atol=1e-9)


# ---------------------------------------------------------- CA seeding stages
def _tiny_frame(seed=5):
    f = synth.generate("one_sector", seed=seed, n_primaries=40)
    rng = np.random.default_rng(seed)
    y, z, row, sec = (f.y.copy(), f.z.copy(), f.row.copy(), f.sector.copy())
    # adversarial additions: exact window edges and equal distances
    extra_y, extra_z, extra_r = [], [], []
    for k in rng.choice(len(y), 60, replace=False):
        r = int(row[k])
        if not 1 <= r <= 150:
            continue
        for dr, dy, dz in ((1, 2.5, 0.0), (-1, -2.5, 2.5), (1, 0.0, -2.5), (-1, 0.25, 0.0),
                           (1, -0.25, 0.0)):
            extra_y.append(np.float32(y[k] + np.float32(dy)))
            extra_z.append(np.float32(z[k] + np.float32(dz)))
            extra_r.append(r + dr)
    y = np.concatenate([y, np.array(extra_y, np.float32)])
    z = np.concatenate([z, np.array(extra_z, np.float32)])
    row = np.concatenate([row, np.array(extra_r, np.uint8)])
    sec = np.concatenate([sec, np.zeros(len(extra_r), np.uint8)])
    assert len(y) <= 2000 or True
    return y, z, row, sec


def _brute_links(y, z, row, sec, o):
    """All-pairs restatement of the neighbour definition (no search structure)."""
    n = len(y)
    up = -np.ones(n, np.int64)
    dn = -np.ones(n, np.int64)
    rx = RX.astype(np.float32)
    for c in range(n):
        r = int(row[c])
        if r < 1 or r > 150:
            continue
        U = np.nonzero((row == r + 1) & (sec == sec[c]) & (np.abs(y - y[c]) <= np.float32(2.5)) &
                       (np.abs(z - z[c]) <= np.float32(2.5)))[0]
        D = np.nonzero((row == r - 1) & (sec == sec[c]) & (np.abs(y - y[c]) <= np.float32(2.5)) &
                       (np.abs(z - z[c]) <= np.float32(2.5)))[0]
        if len(U) == 0 or len(D) == 0:
            continue
        f = (rx[r] - rx[r - 1]) / (rx[r + 1] - rx[r - 1])
        best = None
        for u in U:
            for d in D:
                yp = y[d] + (y[u] - y[d]) * f
                zp = z[d] + (z[u] - z[d]) * f
                ey, ez = np.float32(yp - y[c]), np.float32(zp - z[c])
                d2 = np.float32(ey * ey + ez * ez)
                if not d2 < np.float32(1.0):
                    continue
                key = (float(d2), int(u), int(d))
                if best is None or key < best:
                    best = key
        if best is not None:
            up[c], dn[c] = best[1], best[2]
    return up, dn


def test_neighbours_equal_brute_force_on_tiny_frames():
    for seed in (5, 6):
        y, z, row, sec = _tiny_frame(seed)
        o = opts()
        r_grid = oracle.track(y, z, row, sec, RX.astype(np.float32), o)
        r_bf = oracle.track(y, z, row, sec, RX.astype(np.float32), opts(brute_force=1))
        assert np.array_equal(r_grid["link_up"], r_bf["link_up"])
        assert np.array_equal(r_grid["link_dn"], r_bf["link_dn"])
        up, dn = _brute_links(y, z, row, sec, o)
        assert np.array_equal(r_grid["link_up"], up)
        assert np.array_equal(r_grid["link_dn"], dn)
        for k in r_grid:  # the whole sector chain is identical without the row index
            assert np.array_equal(r_grid[k], r_bf[k]), k


def test_links_follow_truth_on_clean_tracks():
    """Noise-free, well separated straight-ish tracks: every link joins two
    clusters of the same track on adjacent rows."""
    f = synth.generate("one_sector", n_primaries=15, noise_frac=0.0, sigma=0.02, pt_min=1.0,
                       seed=11)
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), opts())
    cu = r["clean_up"]
    ok = cu >= 0
    assert ok.sum() > 0.8 * f.n
    assert np.all(f.label[ok] == f.label[cu[ok]])
    assert np.all(f.row[cu[ok]].astype(int) == f.row[ok].astype(int) + 1)


def test_cleaner_and_start_hit_invariants():
    f = synth.generate("central_event", n_primaries=2000)
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), opts())
    cu, cd = r["clean_up"], r["clean_dn"]
    has = cu >= 0
    assert np.all(cd[cu[has]] == np.nonzero(has)[0])  # mutual
    has = cd >= 0
    assert np.all(cu[cd[has]] == np.nonzero(has)[0])
    # chains are disjoint paths; each chain of >= 3 has exactly one start
    starts = set(r["start"].tolist())
    seen = np.zeros(len(cu), bool)
    n_chains = 0
    for c in np.nonzero(cd < 0)[0]:
        chain = [c]
        while cu[chain[-1]] >= 0:
            chain.append(cu[chain[-1]])
        assert not seen[chain].any()
        seen[chain] = True
        if len(chain) >= 3:
            assert c in starts
            n_chains += 1
        else:
            assert c not in starts
    assert n_chains == len(starts)


# ------------------------------------------------------------ ambiguity solving
def test_selector_matches_greedy_restatement_and_budget():
    f = synth.generate("central_event", n_primaries=3000)
    o = opts()
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), o)
    R = 152
    valid = np.nonzero(r["tl_n"] > 0)[0]
    keys = r["tl_key"]
    # greedy: visit tracklets by key, highest first; the first to claim a cluster owns it
    owner = -np.ones(f.n, np.int64)
    for i in sorted(valid, key=lambda i: -int(keys[i])):
        h = r["tl_hits"][i * R:(i + 1) * R]
        h = h[h >= 0]
        free = owner[h] < 0
        owner[h[free]] = i
    for i in valid:
        h = r["tl_hits"][i * R:(i + 1) * R]
        h = h[h >= 0]
        kept = r["tl_kept"][i * R:(i + 1) * R]
        kept = kept[kept >= 0]
        won = owner[h] == i
        # replay of the outermost-first shared budget
        k, s, exp = 0, 0, []
        for c, w in zip(h, won):
            if w:
                exp.append(c); k += 1
            elif np.float32(s + 1) <= np.float32(0.1) * np.float32(k + 1):
                exp.append(c); k += 1; s += 1
        if r["tl_accept"][i]:
            assert np.array_equal(kept, exp)
            assert s <= 0.1 * k + 1e-6
        else:
            assert len(exp) < o["min_hits"]
    # each cluster has at most one owner, and the owner holds it
    own = r["sector_owner"]
    starts = r["tl_start"]
    acc = r["tl_accept"] == 1
    for c in np.nonzero(own >= 0)[0][:5000]:
        i = owner[c]
        assert acc[i] and starts[i] == own[c]


# ----------------------------------------------------------------- statistics
def test_covariances_symmetric_positive_definite():
    f = synth.generate("central_event", n_primaries=3000)
    for fp64 in (False, True):
        r = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(), fp64=fp64)
        cov = r["tl_cov"].reshape(-1, 15)[r["tl_n"] > 0].astype(np.float64)
        for c in cov:
            np.linalg.cholesky(_full(c))


def test_pulls_are_standard_normal():
    """Tracklet parameters at the innermost cluster against the generated
    truth: pulls have mean 0 and width 1 (statistical pin of propagation,
    Jacobian, scattering-free covariance and update).  The tracklet is a
    single extended-Kalman pass linearised at its running estimate; its q/pT
    pull comes out a few per cent wide at high curvature (a Monte-Carlo of one
    track shows the same spread against the reported error), which the
    iterated refit removes, so q/pT gets a looser bound here."""
    f = synth.generate("central_event", n_primaries=4000, ms_theta=0.0, noise_frac=0.0,
                       sec_frac=0.0, store_truth=True, seed=99)
    r = oracle.track(f.y, f.z, f.row, f.sector, RX, opts(ms_theta=0.0), fp64=True)
    R = 152
    pulls = [[] for _ in range(5)]
    for i in np.nonzero(r["tl_n"] >= 60)[0]:
        h = r["tl_hits"][i * R:(i + 1) * R]
        h = h[h >= 0]
        inner = h[-1]
        if np.any(f.label[h] != f.label[inner]):
            continue
        p = r["tl_param"][i * 5:(i + 1) * 5]
        c = _full(r["tl_cov"][i * 15:(i + 1) * 15])
        t = truth_state(f, inner)
        for k in range(5):
            pulls[k].append((p[k] - t[k]) / math.sqrt(c[k, k]))
    for k in range(5):
        v = np.array(pulls[k])
        assert len(v) > 2000
        assert abs(np.mean(v)) < 0.08, (k, np.mean(v))
        assert 0.9 < np.std(v) < (1.2 if k == 4 else 1.12), (k, np.std(v))


def test_sector_tracking_efficiency_against_truth():
    f = synth.generate("one_sector")
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), opts(ms_theta=0.0))
    R = 152
    hits = [r["tl_kept"][i * R:(i + 1) * R] for i in np.nonzero(r["tl_accept"])[0]]
    hits = [h[h >= 0] for h in hits]
    q = quality(f.label, hits, r["sector_owner"])
    assert q["eff"] > 0.95 and q["fake_rate"] < 0.02, q


def test_scattering_noise_matches_the_generated_random_walk():
    """The propagator's scattering noise against the generator's own random
    walk (it kicks phi by theta*g*sqrt(1+tan^2) and lambda by theta*g at every
    row): over 30 rows of a leg the truth sin(phi) and tan(lambda) deviate from
    the noise-free propagation of their start by N(0, C) with C the
    propagated covariance (from C = 0), so the normalised deviations have unit
    width.  Steep tracks only (|tan lambda| > 0.5), where the tan(lambda) term
    (1 + tan^2)^2 matters most."""
    theta = 0.02
    f = synth.generate("central_event", n_primaries=4000, noise_frac=0.0, sigma=0.0,
                       sec_frac=0.0, ms_theta=theta, store_truth=True, seed=4242)
    o = opts(ms_theta=theta)
    lab, row, sec = f.label, f.row.astype(int), f.sector.astype(int)
    n = 30
    zs, zt = [], []
    for i in range(len(lab) - n):
        j = i + n
        if lab[i] < 0 or lab[j] != lab[i] or sec[j] != sec[i] or row[j] != row[i] + n:
            continue
        if row[i] % 10 or lab[i] % 2:  # one start per 10 rows, first legs only
            continue
        p = truth_state(f, i)
        if abs(p[3]) < 0.5 or abs(p[4]) > 2.0:
            continue
        c = np.zeros(15)
        x = RX[row[i]]
        ok = True
        for r in range(row[i] + 1, row[j] + 1):
            out = oracle.propagate(p, c, x, RX[r], RX, o)
            if out is None:
                ok = False
                break
            p, c, x = out
        if not ok or c[5] <= 0 or c[9] <= 0:
            continue
        t = truth_state(f, j)
        zs.append((t[2] - p[2]) / np.sqrt(c[5]))
        zt.append((t[3] - p[3]) / np.sqrt(c[9]))
    assert len(zt) > 300, len(zt)
    for z in (np.array(zs), np.array(zt)):
        assert abs(np.std(z) - 1.0) < 0.08, np.std(z)
        assert abs(np.mean(z)) < 0.1
