"""Shared test utilities: truth matching (no tracking arithmetic)."""
from __future__ import annotations

import numpy as np

N_ROWS = 152


def exact_row_x() -> np.ndarray:
    return 85.0 + np.arange(N_ROWS, dtype=np.float64) * (160.0 / 151.0)


def majority(labels: np.ndarray):
    vals, cnt = np.unique(labels, return_counts=True)
    j = int(cnt.argmax())
    return int(vals[j]), float(cnt[j]) / float(len(labels))


def quality(label: np.ndarray, track_hits: list[np.ndarray], attach: np.ndarray | None = None,
            min_findable: int = 70, fake_frac: float = 0.9) -> dict:
    """Efficiency / clone / fake rates against generator truth (paper Fig. 2
    definitions: findable = at least 70 clusters; fake = majority fraction < 0.9)."""
    legs, cnt = np.unique(label[label >= 0], return_counts=True)
    findable = set(legs[cnt >= min_findable].tolist())
    found = {}
    fakes = 0
    for hits in track_hits:
        lab, frac = majority(label[hits])
        if lab < 0 or frac < fake_frac:
            fakes += 1
            continue
        found[lab] = found.get(lab, 0) + 1
    n = max(1, len(track_hits))
    eff = np.mean([leg in found for leg in findable]) if findable else float("nan")
    clones = sum(v - 1 for k, v in found.items() if k in findable)
    out = dict(n_tracks=len(track_hits), findable=len(findable), eff=float(eff),
               fake_rate=fakes / n, clone_rate=clones / n)
    if attach is not None:
        att = attach >= 0
        out["attached"] = float(att.mean())
    return out
