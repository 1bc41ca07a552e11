"""Pins of the oracle's refit gradient: the FP64 reverse-mode tape against
central finite differences of the frozen FP64 refit (the derivative the
hand-written adjoint must reproduce), and invariants of the refit."""
from __future__ import annotations

import numpy as np

import oracle
from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions
from tests.helpers import exact_row_x

RX = exact_row_x()


def _event():
    f = synth.generate("central_event", n_primaries=300, distort=True)
    o = TrackerOptions().as_dict()
    r = oracle.track(f.y, f.z, f.row, f.sector, RX.astype(np.float32), o, full=True,
                     dist_map=f.map)
    return f, o, oracle.tracks_for_refit(r)


def test_tape_gradient_equals_central_differences():
    f, o, T = _event()
    base = oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T, dist_map=f.map, mode="f64")
    w = np.random.default_rng(0).uniform(0.5, 1.5, len(T["par"]))
    g = oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T, dist_map=f.map, weights=w,
                     mode="tape")["grad"]
    m = f.map.ravel()
    for i in np.argsort(-np.abs(g))[:8]:
        mp, mm = m.copy(), m.copy()
        mp[i] = np.float32(m[i] + 1e-2)
        mm[i] = np.float32(m[i] - 1e-2)
        step = float(mp[i]) - float(mm[i])
        lp = (w * oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T,
                               dist_map=mp.reshape(f.map.shape), frozen=base,
                               mode="f64")["rf_chi2"]).sum()
        lm = (w * oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T,
                               dist_map=mm.reshape(f.map.shape), frozen=base,
                               mode="f64")["rf_chi2"]).sum()
        fd = (lp - lm) / step
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]), (i, fd, g[i])


def test_refit_is_quadratic_without_x_shift():
    """With only y/z map components the frozen refit chi2 is exactly quadratic
    in the map: second differences are constant (no x-projection term)."""
    f, o, T = _event()
    cmap = f.map.copy()
    cmap[0] = 0.0  # no radial (x) displacement
    base = oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T, dist_map=cmap, mode="f64")
    i = int(np.argmax(np.abs(cmap[1]).ravel())) + cmap[0].size
    vals = []
    for h in (-0.02, 0.0, 0.02, 0.04):
        m = cmap.ravel().astype(np.float64).copy()
        m[i] += h
        vals.append(oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T,
                                 dist_map=m.reshape(cmap.shape).astype(np.float32), frozen=base,
                                 mode="f64")["rf_chi2"].sum())
    d2a = vals[0] - 2 * vals[1] + vals[2]
    d2b = vals[1] - 2 * vals[2] + vals[3]
    assert abs(d2a - d2b) <= 1e-6 * max(1.0, abs(d2a))


def test_refit_reproduces_final_fit_chi2_scale():
    f, o, T = _event()
    r = oracle.refit(f.y, f.z, f.row, f.sector, RX, o, T, dist_map=f.map, mode="f64")
    ok = r["rf_ok"] == 1
    assert ok.mean() > 0.95
    ndf = 2 * r["rf_n"][ok] - 5
    assert 0.8 < np.median(r["rf_chi2"][ok] / ndf) < 1.3
