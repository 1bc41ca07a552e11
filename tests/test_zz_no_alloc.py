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


def _noalloc_lib():
    from paper_2601_20569_gb300 import tpc

    lib = tpc.load()
    lib.tpc_links_noalloc.argtypes = [ctypes.POINTER(tpc.Geometry), ctypes.POINTER(tpc.Options),
                                      ctypes.POINTER(tpc.Clusters), ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]
    lib.tpc_links_noalloc.restype = ctypes.c_int
    return lib


def _links_noalloc(f, opts, out=None, free_mem=None):
    """One call; `out` = preallocated (up, dn) device tensors, `free_mem` = a
    list that receives the device's free bytes just before and after the call."""
    import torch

    from paper_2601_20569_gb300 import tpc

    lib = _noalloc_lib()
    rx = np.ascontiguousarray(RX, dtype=np.float32)
    geo = tpc.Geometry(36, len(rx), rx.ctypes.data)
    o = tpc.make_options(opts, mode=0, cap_clusters=max(f.n, 1))
    y, z, q, row, sec = tpc.Tracker.to_device(f.y, f.z, f.q, f.row, f.sector)
    cl = tpc.Clusters(f.n, y.data_ptr(), z.data_ptr(), q.data_ptr(), row.data_ptr(),
                      sec.data_ptr())
    if out is None:
        up = torch.full((max(f.n, 1),), -7, dtype=torch.int32, device="cuda")
        dn = torch.full((max(f.n, 1),), -7, dtype=torch.int32, device="cuda")
    else:
        up, dn = out
    s = torch.cuda.current_stream()
    torch.cuda.synchronize()
    if free_mem is not None:
        free_mem.append(torch.cuda.mem_get_info()[0])
    rc = lib.tpc_links_noalloc(ctypes.byref(geo), ctypes.byref(o), ctypes.byref(cl),
                               up.data_ptr(), dn.data_ptr(), ctypes.c_void_p(s.cuda_stream))
    torch.cuda.synchronize()
    if free_mem is not None:
        free_mem.append(torch.cuda.mem_get_info()[0])
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
    free = []
    for f in frames:  # two calls in a row on the shared scratch array
        rc, up, dn = _links_noalloc(f, opts, free_mem=free)
        assert rc == 0
        ref_up, ref_dn = _links_regular(f, opts)
        assert (ref_up >= 0).sum() > 0.5 * f.n
        assert np.array_equal(up, ref_up)
        assert np.array_equal(dn, ref_dn)
    # the second call (kernels already loaded by the first) takes no device memory
    assert free[3] == free[2]


def test_noalloc_failed_call_writes_nothing():
    """A call rejected on the device (a NaN coordinate) after a larger valid
    call leaves every output entry untouched: the scratch then still holds the
    earlier call's sorted ids, which lie beyond the smaller call's clusters.
    The outputs are over-allocated so that a regression stays inside them."""
    import torch

    opts = TrackerOptions().as_dict()
    big = synth.generate("central_event")
    sel = np.nonzero((big.sector == 5) | (big.sector == 6))[0][:60000]
    f1 = synth.Frame(y=big.y[sel], z=big.z[sel], q=big.q[sel], row=big.row[sel],
                     sector=big.sector[sel], label=big.label[sel], z_range=big.z_range)
    assert f1.n == 60000
    out = tuple(torch.full((65536,), -7, dtype=torch.int32, device="cuda") for _ in range(2))
    rc, up, _ = _links_noalloc(f1, opts, out=out)
    assert rc == 0 and (up >= 0).sum() > 0.5 * f1.n
    f2 = synth.generate("one_sector", n_primaries=20)
    k = np.arange(800) % f2.n
    y = f2.y[k].copy()
    y[400] = np.nan
    f2 = synth.Frame(y=y, z=f2.z[k], q=f2.q[k], row=f2.row[k], sector=f2.sector[k],
                     label=f2.label[k], z_range=f2.z_range)
    out = tuple(torch.full((65536,), -7, dtype=torch.int32, device="cuda") for _ in range(2))
    rc, _, _ = _links_noalloc(f2, opts, out=out)
    assert rc == 2  # TPC_ERR_INVALID_INPUT
    for t in out:
        assert bool((t == -7).all())


def test_noalloc_rejects_frames_beyond_its_maximum():
    opts = TrackerOptions().as_dict()
    f = synth.generate("central_event", n_primaries=1000)
    assert f.n > 65536
    rc, _, _ = _links_noalloc(f, opts)
    assert rc == 3  # TPC_ERR_CAPACITY, nothing launched
