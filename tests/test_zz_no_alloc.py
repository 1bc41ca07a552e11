"""The allocation-free links entry point, called through the C ABI.

It exists for callers that may not allocate device memory while they run
(allocator callbacks, runtimes with all memory reserved up front, real-time
loops).  Its cleaned neighbour links must equal those of the regular entry
point (tpc_track_timeframe, strict mode) exactly, on two calls in a row that
share the same static scratch array.  This file is collected last on purpose.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

from paper_2601_20569_gb300 import synth
from paper_2601_20569_gb300.options import TrackerOptions

pytestmark = pytest.mark.gpu

RX = synth.row_x()


def _links_regular(f, opts):
    from paper_2601_20569_gb300 import tpc

    tr = tpc.Tracker(RX, opts, mode=0, cap_clusters=max(f.n, 1024))
    tr.track(*tr.to_device(f.y, f.z, f.q, f.row, f.sector))
    sid = tr.debug("sid")
    up = np.full(f.n, -1, np.int64)
    dn = np.full(f.n, -1, np.int64)
    cu, cd = tr.debug("cup"), tr.debug("cdn")
    up[sid] = np.where(cu >= 0, sid[np.maximum(cu, 0)], -1)
    dn[sid] = np.where(cd >= 0, sid[np.maximum(cd, 0)], -1)
    tr.close()
    return up, dn


def _links_noalloc(f, opts):
    import torch

    from paper_2601_20569_gb300 import tpc

    lib = tpc.load()
    lib.tpc_links_noalloc.argtypes = [ctypes.POINTER(tpc.Geometry), ctypes.POINTER(tpc.Options),
                                      ctypes.POINTER(tpc.Clusters), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    lib.tpc_links_noalloc.restype = ctypes.c_int
    rx = np.ascontiguousarray(RX, dtype=np.float32)
    geo = tpc.Geometry(36, len(rx), rx.ctypes.data)
    o = tpc.make_options(opts, mode=0, cap_clusters=max(f.n, 1))
    y, z, q, row, sec = tpc.Tracker.to_device(f.y, f.z, f.q, f.row, f.sector)
    cl = tpc.Clusters(f.n, y.data_ptr(), z.data_ptr(), q.data_ptr(), row.data_ptr(),
                      sec.data_ptr())
    up = torch.full((max(f.n, 1),), -7, dtype=torch.int32, device="cuda")
    dn = torch.full((max(f.n, 1),), -7, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    rc = lib.tpc_links_noalloc(ctypes.byref(geo), ctypes.byref(o), ctypes.byref(cl),
                               up.data_ptr(), dn.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    return rc, up[:f.n].cpu().numpy().astype(np.int64), dn[:f.n].cpu().numpy().astype(np.int64)


def test_noalloc_links_match_regular_entry_point_twice():
    opts = TrackerOptions().as_dict()
    big = synth.generate("central_event")
    sel = np.nonzero(big.sector == 5)[0]
    frames = [
        synth.generate("one_sector"),
        synth.Frame(y=big.y[sel], z=big.z[sel], q=big.q[sel], row=big.row[sel],
                    sector=big.sector[sel], label=big.label[sel], z_range=big.z_range),
    ]
    assert all(0 < f.n <= 65536 for f in frames)
    for f in frames:  # two calls in a row on the shared scratch array
        rc, up, dn = _links_noalloc(f, opts)
        assert rc == 0
        ref_up, ref_dn = _links_regular(f, opts)
        assert (ref_up >= 0).sum() > 0.5 * f.n
        assert np.array_equal(up, ref_up)
        assert np.array_equal(dn, ref_dn)


def test_noalloc_rejects_frames_beyond_its_maximum():
    opts = TrackerOptions().as_dict()
    f = synth.generate("central_event", n_primaries=1000)
    assert f.n > 65536
    rc, _, _ = _links_noalloc(f, opts)
    assert rc == 3  # TPC_ERR_CAPACITY, nothing launched
