"""CPU oracle of the TPC tracking chain -- TEST INFRASTRUCTURE ONLY.

ctypes binding of ``oracle.cpp``.  Only ``tests/``, ``__graft_entry__.smoke()``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA library; the options arrive as a plain
dict of values (the same dict the tests hand to the CUDA path).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = os.path.join(_HERE, "liboracle.so")
# A test may point the binding at a variant of the oracle built elsewhere
# (tests/test_oracle_mutations.py plants mistakes to show that pins catch them).
_VARIANT = os.environ.get("TPC_ORACLE_VARIANT_LIB")
_lib = None

_DT = {"i4": np.int32, "f4": np.float32, "f8": np.float64, "u8": np.uint64}


class _Opt(ctypes.Structure):
    _fields_ = [
        ("bz", ctypes.c_float),
        ("sigma_y", ctypes.c_float),
        ("sigma_z", ctypes.c_float),
        ("ms_theta", ctypes.c_float),
        ("link_wy", ctypes.c_float),
        ("link_wz", ctypes.c_float),
        ("link_chi2", ctypes.c_float),
        ("seed_c", ctypes.c_float * 5),
        ("follow_chi2", ctypes.c_float),
        ("max_snp", ctypes.c_float),
        ("fit_max_snp", ctypes.c_float),
        ("score_w", ctypes.c_float),
        ("shared_frac", ctypes.c_float),
        ("merge_chi2", ctypes.c_float),
        ("merge_dy", ctypes.c_float),
        ("merge_dz", ctypes.c_float),
        ("int_chi2", ctypes.c_float),
        ("final_chi2", ctypes.c_float),
        ("attach_margin", ctypes.c_float),
        ("looper_qpt", ctypes.c_float),
        ("edge_margin", ctypes.c_float),
        ("ext_chi2", ctypes.c_float),
        ("cr_qpt", ctypes.c_float),
        ("cr_protect", ctypes.c_float),
        ("cr_remove", ctypes.c_float),
        ("cr_edge", ctypes.c_float),
        ("cr_occ_w", ctypes.c_float),
        ("cr_p2_grow", ctypes.c_float),
        ("cr_p2_shrink", ctypes.c_float),
        ("cr_leg_dq", ctypes.c_float),
        ("cr_leg_dtgl", ctypes.c_float),
        ("cr_leg_dc", ctypes.c_float),
        ("max_miss", ctypes.c_int32),
        ("min_hits", ctypes.c_int32),
        ("merge_max_gap", ctypes.c_int32),
        ("inner_rows", ctypes.c_int32),
        ("cand_k", ctypes.c_int32),
        ("brute_force", ctypes.c_int32),
        ("n_rows", ctypes.c_int32),
        ("n_sectors", ctypes.c_int32),
        ("ext_rows", ctypes.c_int32),
        ("seed_iters", ctypes.c_int32),
        ("cr_mode", ctypes.c_int32),
        ("cr_occ_max", ctypes.c_int32),
        ("ac_merge", ctypes.c_int32),
        ("edge_rows", ctypes.c_int32),
        ("edge_min", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so: strict IEEE evaluation (no contraction, no fast math)."""
    if _VARIANT:
        return _VARIANT
    src = os.path.join(_HERE, "oracle.cpp")
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(src):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math",
                               "-fPIC", "-shared", src, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        lib.orc_track.restype = ctypes.c_int
        lib.orc_track.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 5 + [
            ctypes.POINTER(_Opt), ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
            ctypes.POINTER(ctypes.c_void_p)]
        lib.orc_track_f64.restype = ctypes.c_int
        lib.orc_track_f64.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 5 + [
            ctypes.POINTER(_Opt), ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        lib.orc_correct.restype = ctypes.c_int
        lib.orc_correct.argtypes = [ctypes.POINTER(_Opt), ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p]
        lib.orc_info.restype = ctypes.c_long
        lib.orc_info.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_char_p]
        lib.orc_copy.restype = ctypes.c_int
        lib.orc_copy.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_long]
        lib.orc_names.restype = ctypes.c_long
        lib.orc_names.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_long]
        lib.orc_op.restype = ctypes.c_int
        lib.orc_op.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_Opt), ctypes.c_void_p,
                               ctypes.c_void_p]
        lib.orc_second_ambiguity.restype = ctypes.c_int
        lib.orc_second_ambiguity.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int] + \
            [ctypes.c_void_p] * 5
        lib.orc_free.restype = None
        lib.orc_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def _opt(opts: dict) -> _Opt:
    o = _Opt()
    for name, typ in _Opt._fields_:
        if name == "seed_c":
            for i, v in enumerate(opts["seed_c"]):
                o.seed_c[i] = float(v)
        elif typ is ctypes.c_float:
            setattr(o, name, float(opts[name]))
        else:
            setattr(o, name, int(opts[name]))
    return o


class _Map(ctypes.Structure):
    _fields_ = [("n_phi", ctypes.c_int32), ("n_r", ctypes.c_int32), ("n_z", ctypes.c_int32),
                ("r_min", ctypes.c_float), ("r_max", ctypes.c_float), ("z_min", ctypes.c_float),
                ("z_max", ctypes.c_float), ("coeff", ctypes.c_void_p)]


def _map(coeff, r_range=(85.0, 245.0), z_range=(-250.0, 250.0)):
    if coeff is None:
        return None, None
    c = np.ascontiguousarray(coeff, dtype=np.float32)
    nz, nr, nphi = c.shape[1:]
    return _Map(nphi, nr, nz, r_range[0], r_range[1], z_range[0], z_range[1], c.ctypes.data), c


class Result(dict):
    """Named arrays produced by one oracle run."""


def _collect(lib, h) -> Result:
    n = lib.orc_names(h, None, 0)
    buf = ctypes.create_string_buffer(n)
    lib.orc_names(h, buf, n)
    res = Result()
    for name in buf.value.decode().split():
        dt = ctypes.create_string_buffer(8)
        nb = lib.orc_info(h, name.encode(), dt)
        a = np.empty(nb // np.dtype(_DT[dt.value.decode()]).itemsize, dtype=_DT[dt.value.decode()])
        if nb:
            lib.orc_copy(h, name.encode(), a.ctypes.data, nb)
        res[name] = a
    return res


def track(y, z, row, sector, row_x, opts: dict, *, fp64: bool = False, full: bool = False,
          dist_map=None) -> Result:
    """Run the oracle chain on host arrays; ``fp64`` selects the double build,
    ``full`` adds merging, the three-iteration fit and the attachment, with the
    optional correction map ``dist_map`` ([3][n_z][n_r][n_phi] control points)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    row = np.ascontiguousarray(row, dtype=np.uint8)
    sector = np.ascontiguousarray(sector, dtype=np.uint8)
    rx = np.ascontiguousarray(row_x, dtype=np.float64)
    o = _opt(opts)
    m, _keep = _map(dist_map)
    h = ctypes.c_void_p()
    rc = lib.orc_track(len(y), y.ctypes.data, z.ctypes.data, row.ctypes.data, sector.ctypes.data,
                       rx.ctypes.data, ctypes.byref(o), ctypes.byref(m) if m is not None else None,
                       int(full), int(fp64), ctypes.byref(h))
    if rc:
        raise ValueError(f"oracle rejected the input (code {rc})")
    try:
        return _collect(lib, h)
    finally:
        lib.orc_free(h)


def _op(op: int, io: np.ndarray, row_x, opts: dict, fp64: bool) -> tuple[int, np.ndarray]:
    lib = _load()
    io = np.ascontiguousarray(io, dtype=np.float64).copy()
    rx = np.ascontiguousarray(row_x, dtype=np.float64)
    o = _opt(opts)
    rc = lib.orc_op(op, int(fp64), ctypes.byref(o), rx.ctypes.data, io.ctypes.data)
    return rc, io


def propagate(p, c, x0, x1, row_x, opts, fp64=True):
    """EKF helix propagation (with scattering noise) of (p[5], c[15]) from x0 to x1."""
    io = np.zeros(32)
    io[:5], io[5:20], io[20], io[21] = p, c, x0, x1
    rc, io = _op(0, io, row_x, opts, fp64)
    return (None if rc else (io[:5], io[5:20], io[20]))


def update(p, c, my, mz, row_x, opts, fp64=True):
    """Kalman update with a (y, z) measurement; returns (p, c, chi2)."""
    io = np.zeros(32)
    io[:5], io[5:20], io[20], io[21] = p, c, my, mz
    rc, io = _op(1, io, row_x, opts, fp64)
    return io[:5], io[5:20], io[22]


def rotate(p, c, x, direction, row_x, opts, fp64=True):
    """Re-express the state in the adjacent sector frame (+1: +20 deg, -1: -20 deg)."""
    io = np.zeros(32)
    io[:5], io[5:20], io[20], io[21] = p, c, x, direction
    rc, io = _op(2, io, row_x, opts, fp64)
    return (None if rc else (io[:5], io[5:20], io[20]))


def seed(points, row_x, opts, fp64=True):
    """Three-point seed; points = [(x, y, z)] * 3.  Returns (p, c, x) or None."""
    io = np.zeros(32)
    io[:9] = np.asarray(points, dtype=np.float64).ravel()
    rc, io = _op(3, io, row_x, opts, fp64)
    return (None if rc else (io[9:14], io[14:29], io[29]))


def second_ambiguity(key, ncand, cand, chi2):
    """Phase II second ambiguity on given candidates: key [T], ncand [T, S],
    cand / chi2 [T, S, K] (best first).  Returns assigned [T, S] (-1: none)."""
    key = np.ascontiguousarray(key, dtype=np.int32)
    ncand = np.ascontiguousarray(ncand, dtype=np.int32)
    cand = np.ascontiguousarray(cand, dtype=np.int32)
    chi2 = np.ascontiguousarray(chi2, dtype=np.float32)
    T, S, K = cand.shape
    assert ncand.shape == (T, S) and chi2.shape == (T, S, K) and key.shape == (T,)
    out = np.full((T, S), -1, np.int32)
    rc = _load().orc_second_ambiguity(T, S, K, key.ctypes.data, ncand.ctypes.data,
                                      cand.ctypes.data, chi2.ctypes.data, out.ctypes.data)
    if rc:
        raise RuntimeError(f"orc_second_ambiguity failed ({rc})")
    return out


def track_f64(y, z, row, sector, row_x, opts: dict, *, full: bool = True, dist_map=None) -> Result:
    """FP64 oracle chain with FP64 cluster coordinates (exact-input pins)."""
    lib = _load()
    y = np.ascontiguousarray(y, dtype=np.float64)
    z = np.ascontiguousarray(z, dtype=np.float64)
    row = np.ascontiguousarray(row, dtype=np.uint8)
    sector = np.ascontiguousarray(sector, dtype=np.uint8)
    rx = np.ascontiguousarray(row_x, dtype=np.float64)
    o = _opt(opts)
    m, _keep = _map(dist_map)
    h = ctypes.c_void_p()
    rc = lib.orc_track_f64(len(y), y.ctypes.data, z.ctypes.data, row.ctypes.data,
                           sector.ctypes.data, rx.ctypes.data, ctypes.byref(o),
                           ctypes.byref(m) if m is not None else None, int(full), ctypes.byref(h))
    if rc:
        raise ValueError(f"oracle rejected the input (code {rc})")
    try:
        return _collect(lib, h)
    finally:
        lib.orc_free(h)


def correct(sector, x, y, z, z0, ref, row_x, opts, dist_map):
    """FP64 map displacement D and the measurement projected on the row along `ref`."""
    lib = _load()
    io = np.zeros(16)
    io[:5] = (sector, x, y, z, z0)
    io[5:10] = ref
    o = _opt(opts)
    m, _keep = _map(dist_map)
    rx = np.ascontiguousarray(row_x, dtype=np.float64)
    rc = lib.orc_correct(ctypes.byref(o), rx.ctypes.data, ctypes.byref(m) if m is not None else None,
                         io.ctypes.data)
    if rc:
        return None
    return io[10:13].copy(), io[13:15].copy()


class _TracksIn(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_long), ("offset", ctypes.c_void_p), ("ids", ctypes.c_void_p),
                ("par", ctypes.c_void_p), ("x", ctypes.c_void_p), ("sector", ctypes.c_void_p),
                ("zshift", ctypes.c_void_p)]


class _Frozen(ctypes.Structure):
    _fields_ = [("ref", ctypes.c_void_p), ("flag", ctypes.c_void_p), ("acc", ctypes.c_void_p)]


def refit(y, z, row, sector, row_x, opts: dict, tracks: dict, *, dist_map=None, frozen=None,
          weights=None, mode: str = "f64") -> Result:
    """Refit tracks with fixed cluster lists (a12).  ``tracks``: offset, ids
    (innermost first), par [n,5] and x, sector of the start parameters, and
    optionally z_shift [n] (tracks merged across the central electrode: shift
    of the measured z on the side other than the innermost cluster's).
    ``frozen``: the frz_* arrays of a previous call (references and decisions
    held fixed).  mode: "f32", "f64" or "tape" (FP64 plus the gradient of
    sum w_t chi2_t with respect to the map coefficients, key "grad")."""
    lib = _load()
    if not hasattr(lib, "_refit_typed"):
        lib.orc_refit.restype = ctypes.c_int
        lib.orc_refit.argtypes = [ctypes.c_long] + [ctypes.c_void_p] * 5 + [
            ctypes.POINTER(_Opt), ctypes.c_void_p, ctypes.POINTER(_TracksIn), ctypes.c_void_p,
            ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]
        lib._refit_typed = True
    y = np.ascontiguousarray(y, dtype=np.float32)
    z = np.ascontiguousarray(z, dtype=np.float32)
    row = np.ascontiguousarray(row, dtype=np.uint8)
    sector = np.ascontiguousarray(sector, dtype=np.uint8)
    rx = np.ascontiguousarray(row_x, dtype=np.float64)
    off = np.ascontiguousarray(tracks["offset"], dtype=np.int32)
    ids = np.ascontiguousarray(tracks["ids"], dtype=np.int32)
    par = np.ascontiguousarray(tracks["par"], dtype=np.float64)
    tx = np.ascontiguousarray(tracks["x"], dtype=np.float64)
    ts = np.ascontiguousarray(tracks["sector"], dtype=np.int32)
    nt = len(off) - 1
    zsh = None
    if tracks.get("z_shift") is not None:
        zsh = np.ascontiguousarray(tracks["z_shift"], dtype=np.float64)
    T = _TracksIn(nt, off.ctypes.data, ids.ctypes.data, par.ctypes.data, tx.ctypes.data,
                  ts.ctypes.data, zsh.ctypes.data if zsh is not None else None)
    w = np.ascontiguousarray(np.ones(nt) if weights is None else weights, dtype=np.float64)
    keep = []
    fz = None
    if frozen is not None:
        fr = [np.ascontiguousarray(frozen["frz_ref"], dtype=np.float64),
              np.ascontiguousarray(frozen["frz_flag"], dtype=np.int32),
              np.ascontiguousarray(frozen["frz_acc"], dtype=np.int32)]
        keep += fr
        fz = _Frozen(fr[0].ctypes.data, fr[1].ctypes.data, fr[2].ctypes.data)
    o = _opt(opts)
    m, _keep = _map(dist_map)
    h = ctypes.c_void_p()
    rc = lib.orc_refit(len(y), y.ctypes.data, z.ctypes.data, row.ctypes.data, sector.ctypes.data,
                       rx.ctypes.data, ctypes.byref(o), ctypes.byref(m) if m is not None else None,
                       ctypes.byref(T), ctypes.byref(fz) if fz is not None else None,
                       w.ctypes.data, {"f32": 0, "f64": 1, "tape": 2}[mode], ctypes.byref(h))
    if rc:
        raise ValueError(f"oracle refit rejected the input (code {rc})")
    try:
        return _collect(lib, h)
    finally:
        lib.orc_free(h)


def tracks_for_refit(res: Result, fp64: bool = True) -> dict:
    """Refit input built from an oracle full-chain result (start = final params)."""
    n = len(res["trk_key"])
    out = {"offset": res["trk_offset"], "ids": res["trk_ids"],
           "par": res["trk_param"].reshape(n, 5).astype(np.float64),
           "x": res["trk_x"].astype(np.float64), "sector": res["trk_sector"]}
    if "trk_zshift" in res:
        out["z_shift"] = res["trk_zshift"].astype(np.float64)
    return out
