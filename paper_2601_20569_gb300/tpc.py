"""Python binding of libtpc.so (ctypes): argument marshalling only.

Every step of the reconstruction runs in the CUDA library; PyTorch provides
device memory and streams.  There is no CPU fallback: if the library is not
built or cannot be loaded, constructing a Tracker raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .options import TrackerOptions

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtpc.so")
_lib = None

STATUS = {0: "TPC_OK", 1: "TPC_ERR_INVALID_ARG", 2: "TPC_ERR_INVALID_INPUT",
          3: "TPC_ERR_CAPACITY", 4: "TPC_ERR_CUDA", 5: "TPC_ERR_OOM", 6: "TPC_ERR_TIMEOUT",
          7: "TPC_ERR_STATE"}


class TpcError(RuntimeError):
    def __init__(self, status: int, msg: str, needed: int = 0):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status
        self.needed = needed


class Geometry(ctypes.Structure):
    _fields_ = [("n_sectors", ctypes.c_int32), ("n_rows", ctypes.c_int32),
                ("row_x", ctypes.c_void_p)]


class Map(ctypes.Structure):
    _fields_ = [("n_phi", ctypes.c_int32), ("n_r", ctypes.c_int32), ("n_z", ctypes.c_int32),
                ("r_min", ctypes.c_float), ("r_max", ctypes.c_float), ("z_min", ctypes.c_float),
                ("z_max", ctypes.c_float), ("coeff", ctypes.c_void_p)]


class Options(ctypes.Structure):
    _fields_ = [
        ("bz", ctypes.c_float), ("sigma_y", ctypes.c_float), ("sigma_z", ctypes.c_float),
        ("ms_theta", ctypes.c_float), ("link_wy", ctypes.c_float), ("link_wz", ctypes.c_float),
        ("link_chi2", ctypes.c_float), ("seed_c", ctypes.c_float * 5),
        ("follow_chi2", ctypes.c_float), ("max_snp", ctypes.c_float),
        ("fit_max_snp", ctypes.c_float), ("score_w", ctypes.c_float),
        ("shared_frac", ctypes.c_float), ("merge_chi2", ctypes.c_float),
        ("merge_dy", ctypes.c_float), ("merge_dz", ctypes.c_float), ("int_chi2", ctypes.c_float),
        ("final_chi2", ctypes.c_float), ("attach_margin", ctypes.c_float),
        ("edge_margin", ctypes.c_float), ("looper_qpt", ctypes.c_float),
        ("ext_chi2", ctypes.c_float),
        ("max_miss", ctypes.c_int32),
        ("min_hits", ctypes.c_int32), ("merge_max_gap", ctypes.c_int32),
        ("inner_rows", ctypes.c_int32), ("cand_k", ctypes.c_int32), ("mode", ctypes.c_int32),
        ("max_frames", ctypes.c_int32), ("use_graphs", ctypes.c_int32),
        ("ext_rows", ctypes.c_int32), ("seed_iters", ctypes.c_int32), ("ac_merge", ctypes.c_int32),
        ("edge_rows", ctypes.c_int32), ("edge_min", ctypes.c_int32),
        ("cap_clusters", ctypes.c_int64), ("cap_tracklets", ctypes.c_int64),
        ("cap_tracks", ctypes.c_int64),
    ]


class Clusters(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("y", ctypes.c_void_p), ("z", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("row", ctypes.c_void_p), ("sector", ctypes.c_void_p)]


class Tracks(ctypes.Structure):
    _fields_ = [("n_tracks", ctypes.c_int64), ("n_cluster_refs", ctypes.c_int64),
                ("params", ctypes.c_void_p), ("cov", ctypes.c_void_p), ("chi2", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("ndf", ctypes.c_void_p), ("sector", ctypes.c_void_p),
                ("n_clusters", ctypes.c_void_p), ("cl_offset", ctypes.c_void_p),
                ("cl_ids", ctypes.c_void_p), ("key", ctypes.c_void_p), ("attach", ctypes.c_void_p),
                ("z_shift", ctypes.c_void_p)]


class RemovalOptions(ctypes.Structure):
    _fields_ = [(k, ctypes.c_float) for k in ("qpt", "protect", "remove", "edge", "occ_w",
                                              "p2_grow", "p2_shrink", "leg_dq", "leg_dtgl",
                                              "leg_dc")] + \
               [("mode", ctypes.c_int32), ("occ_max", ctypes.c_int32)]


class Removal(ctypes.Structure):
    _fields_ = [("n_clusters", ctypes.c_int64), ("n_tracks", ctypes.c_int64),
                ("n_removed", ctypes.c_int64), ("flags", ctypes.c_void_p),
                ("track_class", ctypes.c_void_p), ("leg_parent", ctypes.c_void_p)]


class _DevArray:
    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr or 0), False), "version": 2}


def wrap_device(ptr, shape, typestr):
    """Zero-copy torch view of library-owned device memory (valid until the next call)."""
    import torch

    if not ptr or 0 in tuple(shape):
        dt = {"<i4": torch.int32, "<f4": torch.float32, "|u1": torch.uint8}[typestr]
        return torch.empty(shape, dtype=dt, device="cuda")
    return torch.as_tensor(_DevArray(ptr, shape, typestr), device="cuda")


def load():
    """Load libtpc.so (raises if it was not built: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libtpc.so not built ({LIB_PATH}); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    P = ctypes.POINTER
    lib.tpc_init.argtypes = [P(Geometry), ctypes.c_float, P(Map), P(Options),
                             P(ctypes.c_void_p)]
    lib.tpc_track_timeframe.argtypes = [ctypes.c_void_p, P(Clusters), P(Tracks), ctypes.c_void_p,
                                        P(ctypes.c_int64)]
    lib.tpc_set_map.argtypes = [ctypes.c_void_p, P(Map)]
    lib.tpc_debug_copy.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_void_p,
                                   ctypes.c_int64, P(ctypes.c_int64)]
    lib.tpc_last_error.argtypes = [ctypes.c_void_p]
    lib.tpc_last_error.restype = ctypes.c_char_p
    lib.tpc_profile.argtypes = [ctypes.c_void_p, ctypes.c_int]
    lib.tpc_profile.restype = ctypes.c_int
    lib.tpc_stage_stats.argtypes = [ctypes.c_void_p, ctypes.c_int32, P(ctypes.c_char_p),
                                    P(ctypes.c_double), P(ctypes.c_int64), P(ctypes.c_int64)]
    lib.tpc_stage_stats.restype = ctypes.c_int
    lib.tpc_last_launches.argtypes = [ctypes.c_void_p]
    lib.tpc_last_launches.restype = ctypes.c_int64
    lib.tpc_refit_generation.argtypes = [ctypes.c_void_p]
    lib.tpc_refit_generation.restype = ctypes.c_int64
    lib.tpc_destroy.argtypes = [ctypes.c_void_p]
    lib.tpc_destroy.restype = None
    for name in ("tpc_init", "tpc_track_timeframe", "tpc_set_map", "tpc_debug_copy"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def make_options(opts: dict | TrackerOptions | None = None, *, mode: int = 0,
                 cap_clusters: int = 1 << 20, cap_tracklets: int = 0,
                 cap_tracks: int = 0, max_frames: int = 1, use_graphs: bool = False) -> Options:
    if opts is None:
        opts = TrackerOptions()
    d = opts.as_dict() if isinstance(opts, TrackerOptions) else dict(opts)
    o = Options()
    for name, typ in Options._fields_:
        if name == "seed_c":
            for i, v in enumerate(d["seed_c"]):
                o.seed_c[i] = float(v)
        elif name == "mode":
            o.mode = int(d.get("mode", mode))
        elif name == "cap_clusters":
            o.cap_clusters = int(cap_clusters)
        elif name == "cap_tracklets":
            o.cap_tracklets = int(cap_tracklets)
        elif name == "cap_tracks":
            o.cap_tracks = int(cap_tracks)
        elif name == "max_frames":
            o.max_frames = int(max_frames)
        elif name == "use_graphs":
            o.use_graphs = int(bool(use_graphs))
        elif typ is ctypes.c_float:
            setattr(o, name, float(d[name]))
        else:
            setattr(o, name, int(d[name]))
    return o


_DBG_DTYPE = {
    "rows": None, "bin_first": np.int32, "syz": np.float32, "sid": np.int32,
    "srow": np.uint16, "lup": np.int32, "ldn": np.int32, "cup": np.int32, "cdn": np.int32,
    "starts": np.int32, "tl_n": np.int32, "tl_rlo": np.int32, "tl_rhi": np.int32,
    "tl_chi2": np.float32, "tl_x": np.float32, "tl_par": np.float32, "tl_cov": np.float32,
    "tl_hits": np.int32, "tl_kept": np.int32, "tl_acc": np.int32, "tl_nkept": np.int32,
    "owner_key": np.uint64, "sec_owner": np.int32, "counters": np.int32,
    "sused": np.uint8, "pass_start": np.int32, "cr_flags": np.uint32, "cr_centre_x": np.float32,
    "cr_centre_y": np.float32,
    "st_tl": np.int32, "st_ok": np.int32, "st_key": np.int32, "st_next": np.int32,
    "st_bestB": np.int32, "st_bestchi": np.float32, "st_bestA": np.uint64,
    "st_ie": np.float32, "st_oe": np.float32, "ft_key": np.int32, "ft_ok": np.int32,
    "ft_nst": np.int32, "ft_st_cl": np.int32, "ft_st_rs": np.uint16, "ft_flag": np.uint8,
    "ft_ncand": np.uint8, "ft_cand": np.int32, "ft_cchi": np.float32, "ft_assigned": np.int32,
    "ft_n": np.int32, "ft_next": np.int32, "ft_nout": np.int32, "ft_ext_sec": np.uint16, "out_par": np.float32, "out_cov": np.float32, "out_chi2": np.float32,
    "out_x": np.float32, "out_ndf": np.int32, "out_sector": np.int32, "out_ncl": np.int32,
    "out_offset": np.int32, "out_ids": np.int32, "out_key": np.int32, "attach": np.int32,
}
STATE_F = 22       # floats per stored state: p[5], c[15], x, sector bits
MAX_INNER = 32     # inner-row slots per fit track (extrapolated rows follow them)
MAX_CAND = 8       # candidate slots per inner row
ROWGRID_DTYPE = np.dtype([("bin0", "<i4"), ("nY", "<i4"), ("nZ", "<i4"), ("ncl", "<i4"),
                          ("y0", "<f4"), ("invDy", "<f4"), ("z0", "<f4"), ("invDz", "<f4")])


class Tracker:
    """One reconstruction context (device buffers sized for ``cap_clusters``)."""

    def __init__(self, row_x, opts: dict | TrackerOptions | None = None, *, mode: int = 0,
                 cap_clusters: int = 1 << 20, cap_tracklets: int = 0, cap_tracks: int = 0,
                 bz: float | None = None, max_frames: int = 1, use_graphs: bool = False):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("the tracker needs a CUDA device")
        self.lib = load()
        self.opts = make_options(opts, mode=mode, cap_clusters=cap_clusters,
                                 cap_tracklets=cap_tracklets, cap_tracks=cap_tracks,
                                 max_frames=max_frames, use_graphs=use_graphs)
        self._row_x = np.ascontiguousarray(row_x, dtype=np.float32)
        geo = Geometry(36, len(self._row_x), self._row_x.ctypes.data)
        self._ctx = ctypes.c_void_p()
        torch.cuda.init()
        rc = self.lib.tpc_init(ctypes.byref(geo), float(self.opts.bz if bz is None else bz), None,
                               ctypes.byref(self.opts), ctypes.byref(self._ctx))
        if rc:
            raise TpcError(rc, "tpc_init failed")
        self._keep = []

    def close(self):
        if getattr(self, "_ctx", None) and self._ctx.value:
            self.lib.tpc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    __del__ = close

    def last_error(self) -> str:
        return self.lib.tpc_last_error(self._ctx).decode()

    @staticmethod
    def to_device(y, z, q, row, sector, device="cuda"):
        import torch

        def t(a, dt):
            return torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).to(device)

        return (t(y, np.float32), t(z, np.float32), t(q, np.uint16).view(torch.int16)
                if q is not None else None, t(row, np.uint8), t(sector, np.uint8))

    def track(self, y, z, q, row, sector, stream=None) -> Tracks:
        """Track one frame given device tensors (float32 y, z; uint8 row, sector)."""
        import torch

        n = int(y.shape[0])
        cl = Clusters(n, y.data_ptr(), z.data_ptr(), q.data_ptr() if q is not None else None,
                      row.data_ptr(), sector.data_ptr())
        out = Tracks()
        needed = ctypes.c_int64(0)
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = self.lib.tpc_track_timeframe(self._ctx, ctypes.byref(cl), ctypes.byref(out),
                                          ctypes.c_void_p(s.cuda_stream), ctypes.byref(needed))
        if rc:
            raise TpcError(rc, self.last_error(), needed.value)
        self._last = (out, n)
        return out

    def track_batch(self, frames, stream=None) -> Tracks:
        """Track several frames in one pass; frames: list of (y, z, q, row, sector)
        device tensors.  Tracks carry batch sectors (frame * 36 + sector) and batch
        cluster ids (offset of the frame + id)."""
        import torch

        lib = self.lib
        if not getattr(lib, "_batch_typed", False):
            P = ctypes.POINTER
            lib.tpc_track_batch.argtypes = [ctypes.c_void_p, P(Clusters), ctypes.c_int32,
                                            P(Tracks), ctypes.c_void_p, P(ctypes.c_int64)]
            lib.tpc_track_batch.restype = ctypes.c_int
            lib.tpc_autotune.argtypes = [ctypes.c_void_p, P(Clusters), ctypes.c_int32,
                                         ctypes.c_void_p]
            lib.tpc_autotune.restype = ctypes.c_int
            lib.tpc_launch_config.argtypes = [ctypes.c_void_p, ctypes.c_int32,
                                              P(ctypes.c_char_p), P(ctypes.c_int32),
                                              P(ctypes.c_int32), P(ctypes.c_int32)]
            lib.tpc_launch_config.restype = ctypes.c_int
            lib._batch_typed = True
        arr = (Clusters * len(frames))()
        n = 0
        for i, (y, z, q, row, sector) in enumerate(frames):
            arr[i] = Clusters(int(y.shape[0]), y.data_ptr(), z.data_ptr(),
                              q.data_ptr() if q is not None else None, row.data_ptr(),
                              sector.data_ptr())
            n += int(y.shape[0])
        out = Tracks()
        needed = ctypes.c_int64(0)
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = lib.tpc_track_batch(self._ctx, arr, len(frames), ctypes.byref(out),
                                 ctypes.c_void_p(s.cuda_stream), ctypes.byref(needed))
        if rc:
            raise TpcError(rc, self.last_error(), needed.value)
        self._last = (out, n)
        return out

    def autotune(self, frames, stream=None) -> list[dict]:
        """Pick block size / blocks per SM of the heavy kernels on these frames."""
        import torch

        self.track_batch(frames[:1], stream)  # binds the argtypes
        arr = (Clusters * len(frames))()
        for i, (y, z, q, row, sector) in enumerate(frames):
            arr[i] = Clusters(int(y.shape[0]), y.data_ptr(), z.data_ptr(),
                              q.data_ptr() if q is not None else None, row.data_ptr(),
                              sector.data_ptr())
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = self.lib.tpc_autotune(self._ctx, arr, len(frames), ctypes.c_void_p(s.cuda_stream))
        if rc:
            raise TpcError(rc, self.last_error())
        return self.launch_config()

    def launch_config(self) -> list[dict]:
        P = ctypes.POINTER
        self.lib.tpc_launch_config.argtypes = [ctypes.c_void_p, ctypes.c_int32,
                                               P(ctypes.c_char_p), P(ctypes.c_int32),
                                               P(ctypes.c_int32), P(ctypes.c_int32)]
        self.lib.tpc_launch_config.restype = ctypes.c_int
        out = []
        for slot in range(16):
            name = ctypes.c_char_p()
            b = ctypes.c_int32()
            q = ctypes.c_int32()
            ln = ctypes.c_int32()
            if self.lib.tpc_launch_config(self._ctx, slot, ctypes.byref(name), ctypes.byref(b),
                                          ctypes.byref(q), ctypes.byref(ln)):
                break
            out.append({"kernel": name.value.decode(), "block": b.value, "blocks_per_sm": q.value,
                        "lanes": ln.value})
        return out

    def set_launch_config(self, shapes) -> None:
        """Apply launch shapes, e.g. the list launch_config() returned earlier
        (dicts with "block", "blocks_per_sm" and optionally "lanes", in slot
        order; lanes defaults to the slot's current value)."""
        fn = self.lib.tpc_set_launch_config
        fn.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                       ctypes.c_int32]
        fn.restype = ctypes.c_int
        cur = self.launch_config()
        for slot, sh in enumerate(shapes):
            lanes = int(sh.get("lanes", cur[slot]["lanes"] if slot < len(cur) else 1))
            rc = fn(self._ctx, slot, int(sh["block"]), int(sh["blocks_per_sm"]), lanes)
            if rc:
                raise TpcError(rc, self.last_error())

    def result_attach(self):
        """Device tensor view (int32[n_clusters]) of the last call's attachments."""
        out, n = self._last
        return wrap_device(out.attach, (n,), "<i4")

    def result(self) -> dict:
        """Zero-copy device views of the last call's tracks (valid until the next call)."""
        out, n = self._last
        nt, nr = int(out.n_tracks), int(out.n_cluster_refs)
        f, i = "<f4", "<i4"
        return {
            "params": wrap_device(out.params, (nt, 5), f), "cov": wrap_device(out.cov, (nt, 15), f),
            "chi2": wrap_device(out.chi2, (nt,), f), "x": wrap_device(out.x, (nt,), f),
            "ndf": wrap_device(out.ndf, (nt,), i), "sector": wrap_device(out.sector, (nt,), i),
            "n_clusters": wrap_device(out.n_clusters, (nt,), i),
            "cl_offset": wrap_device(out.cl_offset, (nt + 1,), i),
            "cl_ids": wrap_device(out.cl_ids, (nr,), i), "key": wrap_device(out.key, (nt,), i),
            "attach": wrap_device(out.attach, (n,), i),
            "z_shift": wrap_device(out.z_shift, (nt,), f),
        }

    def cluster_removal(self, opts: dict | TrackerOptions | None = None, mode: int | None = None,
                        stream=None) -> dict:
        """Online cluster removal (tpc_cluster_removal) on the last tracking call's
        tracks, with the cr_* fields of the options (``mode`` overrides cr_mode;
        an unset cr_mode means 1).  Returns zero-copy views of the per-cluster
        flags (uint8, 1 protective tube, 2 seeding history, 4 removal tube,
        8 removed), the track classes and leg parents, and the removed count."""
        import torch

        d = (opts or TrackerOptions())
        d = d.as_dict() if isinstance(d, TrackerOptions) else dict(d)
        o = RemovalOptions()
        for k in ("qpt", "protect", "remove", "edge", "occ_w", "p2_grow", "p2_shrink", "leg_dq",
                  "leg_dtgl", "leg_dc"):
            setattr(o, k, float(d["cr_" + k]))
        o.mode = int(mode if mode is not None else (d["cr_mode"] or 1))
        o.occ_max = int(d["cr_occ_max"])
        fn = self.lib.tpc_cluster_removal
        fn.argtypes = [ctypes.c_void_p, ctypes.POINTER(RemovalOptions), ctypes.POINTER(Removal),
                       ctypes.c_void_p]
        fn.restype = ctypes.c_int
        out = Removal()
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = fn(self._ctx, ctypes.byref(o), ctypes.byref(out), ctypes.c_void_p(s.cuda_stream))
        if rc:
            raise TpcError(rc, self.last_error())
        n, nt = int(out.n_clusters), int(out.n_tracks)
        return {"flags": wrap_device(out.flags, (n,), "|u1"),
                "track_class": wrap_device(out.track_class, (nt,), "<i4"),
                "leg_parent": wrap_device(out.leg_parent, (nt,), "<i4"),
                "n_removed": int(out.n_removed)}

    def refit(self, clusters, tracks: dict, coeff=None, *, freeze: bool = False,
              r_range=(85.0, 245.0), z_range=(-250.0, 250.0), stream=None) -> dict:
        """Refit tracks with fixed clusters (tpc_refit).  clusters: (y, z, q, row,
        sector) device tensors; tracks: dict of device tensors cl_offset, cl_ids,
        params [n,5], x, sector (e.g. ``result()`` of track()); coeff: map tensor or
        None for the context's map.  Returns zero-copy views of chi2, ndf,
        n_clusters, params, cov, x, sector (valid until the next call)."""
        import torch

        lib = self.lib
        if not getattr(lib, "_refit_typed", False):
            P = ctypes.POINTER
            lib.tpc_refit.argtypes = [ctypes.c_void_p, P(Clusters), P(Tracks), P(Map),
                                      ctypes.c_int32, P(Tracks), ctypes.c_void_p]
            lib.tpc_refit.restype = ctypes.c_int
            lib.tpc_refit_backward.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                               ctypes.c_void_p]
            lib.tpc_refit_backward.restype = ctypes.c_int
            lib._refit_typed = True
        y, z, q, row, sector = clusters
        cl = Clusters(int(y.shape[0]), y.data_ptr(), z.data_ptr(),
                      q.data_ptr() if q is not None else None, row.data_ptr(), sector.data_ptr())
        keep = {k: v.contiguous() for k, v in tracks.items() if hasattr(v, "data_ptr")}
        nt = int(keep["params"].shape[0])
        tin = Tracks()
        tin.n_tracks = nt
        tin.n_cluster_refs = int(keep["cl_ids"].shape[0])
        tin.params = keep["params"].data_ptr()
        tin.x = keep["x"].data_ptr()
        tin.sector = keep["sector"].data_ptr()
        tin.cl_offset = keep["cl_offset"].data_ptr()
        tin.cl_ids = keep["cl_ids"].data_ptr()
        if "z_shift" in keep:  # tracks merged across the central electrode
            tin.z_shift = keep["z_shift"].data_ptr()
        mp = None
        if coeff is not None:
            nz, nr, nphi = coeff.shape[1:]
            mp = Map(nphi, nr, nz, r_range[0], r_range[1], z_range[0], z_range[1],
                     coeff.data_ptr())
        out = Tracks()
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = lib.tpc_refit(self._ctx, ctypes.byref(cl), ctypes.byref(tin),
                           ctypes.byref(mp) if mp is not None else None, int(bool(freeze)),
                           ctypes.byref(out), ctypes.c_void_p(s.cuda_stream))
        if rc:
            raise TpcError(rc, self.last_error())
        self._refit_keep = (keep, coeff, clusters)
        self._refit_map_shape = tuple(coeff.shape) if coeff is not None else None
        f, i = "<f4", "<i4"
        return {"chi2": wrap_device(out.chi2, (nt,), f), "ndf": wrap_device(out.ndf, (nt,), i),
                "n_clusters": wrap_device(out.n_clusters, (nt,), i),
                "params": wrap_device(out.params, (nt, 5), f),
                "cov": wrap_device(out.cov, (nt, 15), f), "x": wrap_device(out.x, (nt,), f),
                "sector": wrap_device(out.sector, (nt,), i)}

    def refit_backward(self, dl_dchi2, map_shape=None, stream=None):
        """d(sum dl_dchi2 * chi2)/d(map) of the last refit (tpc_refit_backward)."""
        import torch

        shape = map_shape or self._refit_map_shape
        g = torch.empty(shape, dtype=torch.float32, device="cuda")
        d = dl_dchi2.contiguous().to(torch.float32)
        s = stream if stream is not None else torch.cuda.current_stream()
        rc = self.lib.tpc_refit_backward(self._ctx, ctypes.c_void_p(d.data_ptr()),
                                         ctypes.c_void_p(g.data_ptr()),
                                         ctypes.c_void_p(s.cuda_stream))
        if rc:
            raise TpcError(rc, self.last_error())
        return g

    @staticmethod
    def fma_peak(fp64: bool = False, iters: int = 4096) -> float:
        """Measured FMA throughput of the current device in TFLOP/s (tpc_fma_peak)."""
        import torch

        lib = load()
        lib.tpc_fma_peak.argtypes = [ctypes.c_int32, ctypes.c_int32,
                                     ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
        lib.tpc_fma_peak.restype = ctypes.c_int
        v = ctypes.c_double(0.0)
        rc = lib.tpc_fma_peak(int(bool(fp64)), int(iters), ctypes.byref(v),
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        if rc:
            raise TpcError(rc, "tpc_fma_peak")
        return v.value

    def refit_generation(self) -> int:
        """Successful refits on this context so far (tpc_refit_generation)."""
        return int(self.lib.tpc_refit_generation(self._ctx))

    def set_map(self, coeff, r_range=(85.0, 245.0), z_range=(-250.0, 250.0)):
        """Use a correction map: float32 CUDA tensor [3][n_z][n_r][n_phi] (kept alive here)."""
        if coeff is None:
            rc = self.lib.tpc_set_map(self._ctx, None)
            self._map = None
        else:
            nz, nr, nphi = coeff.shape[1:]
            self._map = coeff
            m = Map(nphi, nr, nz, r_range[0], r_range[1], z_range[0], z_range[1],
                    coeff.data_ptr())
            rc = self.lib.tpc_set_map(self._ctx, ctypes.byref(m))
        if rc:
            raise TpcError(rc, self.last_error())

    def profile(self, enable: bool = True) -> None:
        rc = self.lib.tpc_profile(self._ctx, int(enable))
        if rc:
            raise TpcError(rc, self.last_error())

    def stage_stats(self) -> list[dict]:
        out = []
        i = 0
        while True:
            name = ctypes.c_char_p()
            ms = ctypes.c_double()
            calls = ctypes.c_int64()
            launches = ctypes.c_int64()
            if self.lib.tpc_stage_stats(self._ctx, i, ctypes.byref(name), ctypes.byref(ms),
                                        ctypes.byref(calls), ctypes.byref(launches)):
                break
            out.append(dict(name=name.value.decode(), ms=ms.value, calls=calls.value,
                            launches=launches.value))
            i += 1
        return out

    def last_launches(self) -> int:
        return int(self.lib.tpc_last_launches(self._ctx))

    def debug(self, name: str) -> np.ndarray:
        nb = ctypes.c_int64(0)
        rc = self.lib.tpc_debug_copy(self._ctx, name.encode(), None, 0, ctypes.byref(nb))
        if rc:
            raise TpcError(rc, self.last_error())
        dt = ROWGRID_DTYPE if name == "rows" else np.dtype(_DBG_DTYPE.get(name, np.uint8))
        a = np.empty(nb.value // dt.itemsize, dtype=dt)
        if nb.value:
            rc = self.lib.tpc_debug_copy(self._ctx, name.encode(), a.ctypes.data, nb.value,
                                         ctypes.byref(nb))
            if rc:
                raise TpcError(rc, self.last_error())
        return a
