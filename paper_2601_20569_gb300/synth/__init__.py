"""Seeded synthetic TPC time frames (ctypes binding of ``synth.cpp``).

The generator simulates helix tracks in a solenoidal field crossing the pad
rows of the 36 TPC sectors (Sec. 2 of the paper: two halves of 18 trapezoidal
sectors), with the continuous-readout structure of Sec. 1 (overlapping
collisions inside a 2.8 ms time frame).  It holds no tracking arithmetic: it
serves the CUDA tracker, the CPU oracle and the benchmark alike.

Workload presets (sizes and distributions of a 50 kHz Pb-Pb time frame):

* ``one_sector``   -- 200 primaries from the origin in one sector, no scattering.
* ``central_event``-- 12,000 primaries over all 36 sectors, 2 % secondaries,
  1 mrad multiple scattering per row, 5 % noise (about 1.8e6 clusters).
* ``timeframe``    -- Poisson(140) collisions in 2.8 ms, multiplicity
  Exp(1000) capped at 12,000, drift 2.58 cm/us, per-sector occupancy factors
  in [0.1, 1] (about 2e7 clusters per frame).
* ``timeframe_distorted`` -- ``timeframe`` plus the B-spline space-charge field.
* ``stress``       -- Poisson(280) collisions, distortions, 20 % loopers at
  pT in [0.06, 0.15] GeV.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libsynth.so")
_lib = None

N_SECTORS = 36
N_ROWS = 152
MAP_SHAPE = (18, 16, 20)  # (n_phi, n_r, n_z)
MAP_R = (85.0, 245.0)
MAP_Z = (-250.0, 250.0)


def row_x() -> np.ndarray:
    """Pad-row radii x_r = 85 + r*160/151 cm (float32, 152 rows)."""
    return (85.0 + np.arange(N_ROWS, dtype=np.float64) * (160.0 / 151.0)).astype(np.float32)


class _Config(ctypes.Structure):
    _fields_ = [
        ("seed", ctypes.c_uint64),
        ("frame", ctypes.c_int32),
        ("mode", ctypes.c_int32),
        ("n_primaries", ctypes.c_int32),
        ("mult_cap", ctypes.c_int32),
        ("mean_collisions", ctypes.c_double),
        ("mean_mult", ctypes.c_double),
        ("frame_us", ctypes.c_double),
        ("vdrift", ctypes.c_double),
        ("bz", ctypes.c_double),
        ("pt_min", ctypes.c_double),
        ("pt_max", ctypes.c_double),
        ("pt_power", ctypes.c_double),
        ("eta_min", ctypes.c_double),
        ("eta_max", ctypes.c_double),
        ("phi_min", ctypes.c_double),
        ("phi_max", ctypes.c_double),
        ("sec_frac", ctypes.c_double),
        ("sec_rmax", ctypes.c_double),
        ("ms_theta", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("noise_frac", ctypes.c_double),
        ("looper_frac", ctypes.c_double),
        ("looper_pt_min", ctypes.c_double),
        ("looper_pt_max", ctypes.c_double),
        ("only_sector", ctypes.c_int32),
        ("thin_sectors", ctypes.c_int32),
        ("max_legs", ctypes.c_int32),
        ("n_threads", ctypes.c_int32),
        ("store_truth", ctypes.c_int32),
        ("shuffle", ctypes.c_int32),
        ("aim_radius", ctypes.c_double),
        ("map", ctypes.c_void_p),
        ("map_nphi", ctypes.c_int32),
        ("map_nr", ctypes.c_int32),
        ("map_nz", ctypes.c_int32),
        ("map_pad", ctypes.c_int32),
        ("map_rmin", ctypes.c_double),
        ("map_rmax", ctypes.c_double),
        ("map_zmin", ctypes.c_double),
        ("map_zmax", ctypes.c_double),
        ("vz_sigma", ctypes.c_double),
    ]


def build(force: bool = False) -> str:
    """Compile libsynth.so in-tree with the host C++ compiler."""
    src = os.path.join(_HERE, "synth.cpp")
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(src):
        import subprocess

        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", src, "-o", tmp]
        )
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.synth_generate.argtypes = [ctypes.POINTER(_Config), ctypes.POINTER(ctypes.c_void_p)]
        lib.synth_generate.restype = ctypes.c_int
        lib.synth_count.argtypes = [ctypes.c_void_p, ctypes.c_char_p]
        lib.synth_count.restype = ctypes.c_long
        lib.synth_copy.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p, ctypes.c_long]
        lib.synth_copy.restype = ctypes.c_int
        lib.synth_free.argtypes = [ctypes.c_void_p]
        lib.synth_free.restype = None
        lib.synth_philox.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        lib.synth_philox.restype = None
        lib.synth_distortion_profile.argtypes = [ctypes.c_int] * 3 + [ctypes.c_double] * 5 + [ctypes.c_void_p]
        lib.synth_distortion_profile.restype = ctypes.c_int
        lib.synth_eval_distortion.argtypes = (
            [ctypes.c_void_p] + [ctypes.c_int] * 3 + [ctypes.c_double] * 4 + [ctypes.c_int]
            + [ctypes.c_double] * 3 + [ctypes.c_void_p]
        )
        lib.synth_eval_distortion.restype = ctypes.c_int
        _lib = lib
    return _lib


def philox4x32_10(counter, key) -> np.ndarray:
    """One Philox4x32-10 block (exposed for known-answer tests)."""
    lib = _load()
    c = np.ascontiguousarray(counter, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib.synth_philox(c.ctypes.data, k.ctypes.data, out.ctypes.data)
    return out


def distortion_map(amp: float = 5.0) -> np.ndarray:
    """Control points [3][n_z][n_r][n_phi] of the synthetic space-charge field:
    radial amp*(85/r)^2*(1-|z|/250) plus half of it azimuthally (float32)."""
    nphi, nr, nz = MAP_SHAPE
    out = np.zeros((3, nz, nr, nphi), dtype=np.float32)
    _load().synth_distortion_profile(nphi, nr, nz, MAP_R[0], MAP_R[1], MAP_Z[0], MAP_Z[1], amp,
                                     out.ctypes.data)
    return out


def eval_distortion(coeff: np.ndarray, sector: int, x: float, y: float, z: float) -> np.ndarray:
    """The generator's own FP64 evaluation of the field at a sector-local point."""
    coeff = np.ascontiguousarray(coeff, dtype=np.float32)
    nz, nr, nphi = coeff.shape[1:]
    d = np.zeros(3, dtype=np.float64)
    _load().synth_eval_distortion(coeff.ctypes.data, nphi, nr, nz, MAP_R[0], MAP_R[1], MAP_Z[0],
                                  MAP_Z[1], sector, x, y, z, d.ctypes.data)
    return d


@dataclass
class Frame:
    """One synthetic frame: SoA clusters plus generator truth."""

    y: np.ndarray
    z: np.ndarray
    q: np.ndarray
    row: np.ndarray
    sector: np.ndarray
    label: np.ndarray
    z_range: np.ndarray  # [zlo_A, zhi_A, zlo_C, zhi_C] of the measured drift coordinate
    truth: dict = field(default_factory=dict)
    particles: dict = field(default_factory=dict)
    map: np.ndarray | None = None
    workload: str = ""

    @property
    def n(self) -> int:
        return int(self.y.shape[0])


PRESETS = {
    "one_sector": dict(mode=0, n_primaries=200, eta_min=0.05, eta_max=0.9,
                       phi_min=0.0, phi_max=math.radians(20.0), only_sector=0, ms_theta=0.0,
                       sec_frac=0.0, aim_radius=165.0),
    "central_event": dict(mode=0, n_primaries=12000),
    "timeframe": dict(mode=1, thin_sectors=1),
    "timeframe_distorted": dict(mode=1, thin_sectors=1, distort=True),
    "stress": dict(mode=1, thin_sectors=1, distort=True, mean_collisions=280.0,
                   looper_frac=0.2),
}

PRESET_INDEX = {"one_sector": 1, "central_event": 2, "timeframe": 3, "timeframe_distorted": 4,
                "stress": 5}


def seed_for(workload: str, frame: int = 0) -> int:
    return 20260120 + PRESET_INDEX.get(workload, 9) * 1000 + frame


def generate(workload: str = "one_sector", frame: int = 0, *, seed: int | None = None,
             store_truth: bool = False, n_threads: int = 0, shuffle: bool = False,
             **overrides) -> Frame:
    """Generate one seeded frame of the named workload (overrides patch the preset)."""
    lib = _load()
    p = dict(
        mode=0, n_primaries=200, mult_cap=12000, mean_collisions=140.0, mean_mult=1000.0,
        frame_us=2800.0, vdrift=2.58, bz=0.5, pt_min=0.1, pt_max=10.0, pt_power=2.5,
        eta_min=-0.9, eta_max=0.9, phi_min=0.0, phi_max=2 * math.pi, sec_frac=0.02,
        sec_rmax=30.0, ms_theta=1e-3, sigma=0.1, noise_frac=0.05, looper_frac=0.0,
        looper_pt_min=0.06, looper_pt_max=0.15, only_sector=-1, thin_sectors=0, max_legs=2,
        distort=False, map_amp=5.0, aim_radius=0.0, vz_sigma=0.0,
    )
    p.update(PRESETS[workload])
    p.update(overrides)
    cfg = _Config()
    cfg.seed = seed if seed is not None else seed_for(workload, frame)
    cfg.frame = frame
    for k in ("mode", "n_primaries", "mult_cap", "only_sector", "thin_sectors", "max_legs"):
        setattr(cfg, k, int(p[k]))
    for k in ("mean_collisions", "mean_mult", "frame_us", "vdrift", "bz", "pt_min", "pt_max",
              "pt_power", "eta_min", "eta_max", "phi_min", "phi_max", "sec_frac", "sec_rmax",
              "ms_theta", "sigma", "noise_frac", "looper_frac", "looper_pt_min", "looper_pt_max",
              "aim_radius", "vz_sigma"):
        setattr(cfg, k, float(p[k]))
    cfg.n_threads = n_threads
    cfg.store_truth = int(store_truth)
    cfg.shuffle = int(shuffle)
    cmap = None
    if p["distort"]:
        cmap = distortion_map(p["map_amp"]) if not isinstance(p["distort"], np.ndarray) else \
            np.ascontiguousarray(p["distort"], dtype=np.float32)
        cfg.map = cmap.ctypes.data
        cfg.map_nz, cfg.map_nr, cfg.map_nphi = cmap.shape[1:]
        cfg.map_rmin, cfg.map_rmax = MAP_R
        cfg.map_zmin, cfg.map_zmax = MAP_Z
    h = ctypes.c_void_p()
    rc = lib.synth_generate(ctypes.byref(cfg), ctypes.byref(h))
    if rc != 0:
        raise RuntimeError(f"synth_generate failed ({rc})")
    try:
        n = lib.synth_count(h, b"clusters")
        npart = lib.synth_count(h, b"particles")

        def get(name, dtype, count):
            a = np.empty(count, dtype=dtype)
            if count:
                rc2 = lib.synth_copy(h, name.encode(), a.ctypes.data, a.nbytes)
                if rc2:
                    raise RuntimeError(f"synth_copy({name}) failed ({rc2})")
            return a

        fr = Frame(
            y=get("y", np.float32, n), z=get("z", np.float32, n), q=get("q", np.uint16, n),
            row=get("row", np.uint8, n), sector=get("sector", np.uint8, n),
            label=get("label", np.int32, n), z_range=get("z_range", np.float64, 4),
            map=cmap, workload=workload,
        )
        if store_truth:
            for k in ("ty", "tz", "tsnp", "ttgl", "tqpt", "tyu", "tzu"):
                fr.truth[k[1:]] = get(k, np.float64, n)
        for k, dt in (("p_pt", np.float64), ("p_q", np.float64), ("p_tgl", np.float64),
                      ("p_phi", np.float64), ("p_t0", np.float64), ("p_vx", np.float64),
                      ("p_vy", np.float64), ("p_secondary", np.int32), ("p_ncl_leg0", np.int32),
                      ("p_ncl_leg1", np.int32)):
            fr.particles[k[2:]] = get(k, dt, npart)
        fr.particles["sector_thin"] = get("sector_thin", np.float64, 36)
    finally:
        lib.synth_free(h)
    return fr
