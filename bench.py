#!/usr/bin/env python
"""Throughput of TPC time-frame tracking on GB300: clusters/s.

One step = the whole reconstruction chain over a batch of synthetic 2.8 ms
Pb-Pb time frames (50 kHz: Poisson(140) collisions per frame, ~2e7 clusters
each, per-sector occupancy varying ~10x).  Inputs are generated on the host
(seeded), uploaded once and stay resident in HBM for the device-timed value;
the end-to-end figure copies each step's clusters from pinned host memory and
reads the results back inside its timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU runs are independent replicas (one process per GPU, each with its
own frames): weak scaling, no collective on the data path.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "clusters/s tracked per GB300 (2.8 ms Pb-Pb time frame) vs oracle; % HBM roofline"
UNIT = "clusters/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--frames", type=int, default=8)
    ap.add_argument("--workload", default="timeframe")
    ap.add_argument("--mode", default="fast", choices=["fast", "strict"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--launch", default="",
                    help="fixed launch shapes instead of autotuning, e.g. "
                         "256x4,128x4,256x16x16,64x8,256x8 (block x blocks per SM [x lanes "
                         "per item], slot order)")
    ap.add_argument("--collisions", type=float, default=0.0,
                    help="mean collisions per frame instead of the workload's (small "
                         "profiling cases)")
    ap.add_argument("--no-refit", action="store_true",
                    help="skip the refit + adjoint timing on one distorted frame")
    ap.add_argument("--ext-rows", type=int, default=0,
                    help="Phase III extrapolation over this many rows below and above each track (0: off)")
    ap.add_argument("--edge-rows", type=int, default=0,
                    help="edge following: rows followed into the adjacent sector beyond track "
                         "ends at a sector edge (Sec. 2; 0 = off, the default)")
    ap.add_argument("--seed-iters", type=int, default=1,
                    help="sector-tracking iterations, the later ones on leftover clusters "
                         "(Sec. 3; 1 = off, the default)")
    ap.add_argument("--profile-only", action="store_true",
                    help="run warm-up plus one step, then one cluster removal on its tracks, "
                         "and exit (for ncu launch lists)")
    return ap.parse_args()


T_START = time.perf_counter()


def note(msg: str) -> None:
    """Progress on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - T_START:7.1f}s] {msg}", file=sys.stderr, flush=True)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        sm, smax, reasons = [], 0.0, set()
        for line in (getattr(self, "out", "") or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = max(smax, float(f[2]))
            except ValueError:
                continue
            for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                                "sw_power_cap"), f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def replica_frame_ids(rank, frames):
    """Frames of one replica: every rank tracks its own frames (weak scaling,
    no data exchange between ranks)."""
    return [rank * frames + k for k in range(frames)]


def reduce_job(ms, n_local, world):
    """Whole-job view of a timed region: the slowest rank's time and the
    clusters all ranks processed (rank 0 reports their ratio)."""
    if world <= 1:
        return ms, n_local
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([ms], dtype=torch.float64, device=dev)
    n = torch.tensor([n_local], dtype=torch.int64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def make_frames(args, rank):
    from paper_2601_20569_gb300 import synth

    frames = []
    for fid in replica_frame_ids(rank, args.frames):
        kw = {"mean_collisions": args.collisions} if args.collisions > 0 else {}
        frames.append(synth.generate(args.workload, frame=fid, **kw))
    return frames


def cpu_baseline(frames, seconds):
    """The strict CPU oracle, as it stands, on a bounded sample: whole sectors
    of the first frame until about `seconds` of CPU time are spent."""
    import numpy as np

    import oracle
    from paper_2601_20569_gb300 import synth
    from paper_2601_20569_gb300.options import TrackerOptions

    f = frames[0]
    opts = TrackerOptions().as_dict()
    n_done, t_done, groups = 0, 0.0, 0
    for g in range(12):  # groups of three adjacent sectors, the whole chain on each
        idx = np.nonzero((f.sector // 3) == g)[0]
        t0 = time.perf_counter()
        oracle.track(f.y[idx], f.z[idx], f.row[idx], f.sector[idx], synth.row_x(), opts,
                     full=True)
        t_done += time.perf_counter() - t0
        n_done += len(idx)
        groups += 1
        if t_done >= seconds:
            break
    return {"value": n_done / t_done, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{3 * groups} of 36 sectors of frame 0 in groups of 3 adjacent sectors "
                      f"({n_done} clusters, {t_done:.1f} s), full chain, strict FP32 oracle, "
                      f"single thread"}


def _oracle_group(cols):
    """One oracle call on one group of sectors (a worker of the parallel baseline)."""
    import oracle
    from paper_2601_20569_gb300 import synth
    from paper_2601_20569_gb300.options import TrackerOptions

    y, z, row, sec = cols
    t0 = time.perf_counter()
    oracle.track(y, z, row, sec, synth.row_x(), TrackerOptions().as_dict(), full=True)
    return time.perf_counter() - t0


def _nothing(_):
    return 0


def cpu_baseline_parallel(frames):
    """The same oracle on all 12 groups of three adjacent sectors of the first
    frame at once, one process per group on the host cores (spawned workers,
    started and warmed before the timed region)."""
    import multiprocessing

    import numpy as np

    f = frames[0]
    groups = [np.nonzero((f.sector // 3) == g)[0] for g in range(12)]
    cols = [(f.y[i], f.z[i], f.row[i], f.sector[i]) for i in groups]
    workers = max(1, min(os.cpu_count() or 1, len(groups)))
    with multiprocessing.get_context("spawn").Pool(workers) as pool:
        pool.map(_nothing, range(workers))
        t0 = time.perf_counter()
        per = pool.map(_oracle_group, cols, chunksize=1)
        wall = time.perf_counter() - t0
    return {"value": f.n / wall, "unit": UNIT, "cores": workers, "kind": "oracle",
            "sample": f"all 36 sectors of frame 0 ({f.n} clusters) as 12 groups of 3 adjacent "
                      f"sectors, one process per group, {wall:.1f} s wall "
                      f"({sum(per):.1f} s of oracle time), full chain, strict FP32 oracle"}


def run_reference(args):
    """The CPU oracle as the reference arm, on the host cores."""
    import numpy as np

    import oracle
    from paper_2601_20569_gb300 import synth
    from paper_2601_20569_gb300.options import TrackerOptions

    f = synth.generate(args.workload, frame=0)
    opts = TrackerOptions().as_dict()
    # one step = a bounded sample: the clusters of two sectors of frame 0
    sel = np.nonzero(f.sector < 2)[0]
    run = lambda: oracle.track(f.y[sel], f.z[sel], f.row[sel], f.sector[sel], synth.row_x(), opts,
                               full=True)
    for _ in range(args.warmup):
        run()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        run()
    dt = time.perf_counter() - t0
    v = len(sel) * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": f"{args.workload} (sample: sectors 0-1 of "
                                                     f"frame 0, {len(sel)} clusters per step)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"sectors 0-1 of frame 0 ({len(sel)} clusters) per step"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# Algorithmic bytes of each stage: the minimum it must move, from the counts
# of one call (clusters n, tracklet hits th, tracklets nt, sector-track hits
# sh, sector tracks ns, fit stations fst, fitted hits fh, fit tracks nf; the
# tracklet hits rh and tracklets rt of the later seeding iterations).
def stage_bytes(name: str, c: dict) -> float:
    n, th, nt = c["clusters"], c["tl_hits"], c["tracklets"]
    rh, rt, iters = c.get("re_hits", 0), c.get("re_tracklets", 0), c.get("seed_iters", 1)
    sh, ns, fh, nf = c["st_hits"], c["sector_tracks"], c["fit_hits"], c["fit_tracks"]
    fst = c["fit_stations"]
    table = {
        # read y, z, row, sector; write sorted y, z, id, sector-row
        "grid": n * (10 + 14),
        # read sorted y, z, id; write links; cleaner reads/writes links
        "links": n * (12 + 8 + 8 + 8),
        # read cleaned links, write the start list
        "starts": n * 8 + nt * 4,
        # per hit: y, z, id read on the way up and down, hit written; state out
        "tracklets": th * (2 * 12 + 4) + nt * 96,
        # per hit: index and owner key read twice, key written; per tracklet
        "select": th * (4 * 2 + 8 * 2) + nt * 16,
        # per kept hit and pass: index, y, z, row; per track: start, two end states
        "sector_refit": sh * 2 * (4 + 8 + 2) + ns * (24 + 2 * 88),
        # both end states of every sector track, index and link words
        "merge": ns * (2 * 88 + 16),
        # per station: list entry, y, z and the stored prediction written
        # (iteration 1), read back with the flag written (iteration 2); states
        "fit12": fst * (6 + 8 + 20 + 6 + 8 + 20 + 1) + nf * 2 * 88,
        # per inner station and round: candidate, chi2, bid word
        "ambiguity2": nf * 20 * 4 * (4 + 4 + 8),
        # per station: list entry, flag, y, z, used index; states
        "fit3": fst * (6 + 1 + 8 + 4) + nf * 2 * 88,
        # used clusters and state per output track
        "output": fh * 12 + nf * 100,
        # per later iteration: taken flags and owner keys of all clusters, the
        # neighbour finding and start hits again; the tracklets and selection
        # of those iterations as above
        "reseed": (iters - 1) * n * (1 + 8 + 36 + 8) + rh * (28 + 24) + rt * (96 + 16 + 4),
    }
    return float(table.get(name, 0.0))


# Whole-chain algorithmic bytes per cluster: input 12, sorted copy written and
# read 24, links written and read 16, cleaning 8, attachment 4, cluster reads
# of the fit and refit 28.
CHAIN_BYTES_PER_CLUSTER = 92.0


def _traffic_table():
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
            return json.load(fh)
    except (OSError, ValueError):
        return {}


def measured_traffic(stage: str, c: dict):
    """DRAM bytes (read + write) per call of `stage` ("chain" = the whole pass),
    from the ncu figures in profiles/traffic.json (bytes per input cluster on
    the frame named there), scaled to this call by its clusters; (None, None)
    without a figure, or when the figure is marked stale (its kernels changed
    after the capture)."""
    t = _traffic_table().get(stage)
    if not t or t.get("stale"):
        return None, None
    return float(t["bytes_per_cluster"]) * c["clusters"], \
        f"ncu dram__bytes_read.sum + dram__bytes_write.sum per cluster ({t['kernels']}; " \
        f"{t['workload']}; profiles/traffic.json) times this call's clusters"


def refit_timing(mode):
    """Refit with fixed clusters (tpc_refit) and its adjoint (tpc_refit_backward,
    d sum(chi2) / d map) on one space-charge distorted 2.8 ms frame: ms per
    call, CUDA events on the calling stream."""
    import torch

    from paper_2601_20569_gb300 import synth, tpc
    from paper_2601_20569_gb300.options import TrackerOptions

    f = synth.generate("timeframe_distorted", frame=0)
    tr = tpc.Tracker(synth.row_x(), TrackerOptions(), mode=mode, cap_clusters=f.n)
    coeff = torch.as_tensor(f.map).cuda()
    tr.set_map(coeff)
    dev = tr.to_device(f.y, f.z, f.q, f.row, f.sector)
    tr.track(*dev)
    res = tr.result()
    tracks = {k: res[k].clone() for k in ("cl_offset", "cl_ids", "params", "x", "sector")}
    nt = int(tracks["params"].shape[0])
    w = torch.ones(nt, device="cuda")
    tr.refit(dev, tracks, coeff)
    tr.refit_backward(w)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    reps = 3
    ev[0].record(stream)
    for _ in range(reps):
        tr.refit(dev, tracks, coeff)
    ev[1].record(stream)
    for _ in range(reps):
        tr.refit_backward(w)
    ev[2].record(stream)
    torch.cuda.synchronize()
    out = {"workload": f"one distorted 2.8 ms frame: {f.n} clusters, {nt} tracks, "
                       f"map 18x16x20x3", "refit_ms": ev[0].elapsed_time(ev[1]) / reps,
           "backward_ms": ev[1].elapsed_time(ev[2]) / reps, "tracks": nt}
    tr.close()
    return out


def strict_timing(dev, topts, steps, warmup, stream, world):
    """The batched pass in strict mode (FP32 without FMA contraction, correctly
    rounded divide and square root: the mode that is bit-exact against the
    oracle) on the same resident frames, autotuned the same way."""
    import torch

    from paper_2601_20569_gb300 import synth, tpc
    from paper_2601_20569_gb300.options import MODE_STRICT

    n = sum(int(d[0].shape[0]) for d in dev)
    tr = tpc.Tracker(synth.row_x(), topts, mode=MODE_STRICT, cap_clusters=n,
                     max_frames=len(dev), use_graphs=True)
    tr.autotune(dev[:2])
    for _ in range(warmup):
        tr.track_batch(dev, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        tr.track_batch(dev, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    tr.close()
    ms, nj = reduce_job(e0.elapsed_time(e1), n, world)
    return {"value": nj * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "frac": nj * steps / (ms / 1e3) * CHAIN_BYTES_PER_CLUSTER / 1e9 / peaks()[0],
            "form": "strict mode (bit-exact against the oracle), batched + CUDA graph"}


def per_sector_timing(dev, topts, mode, steps, stream, world):
    """The plain per-sector form on the same frames: one tracking call per
    sector of every frame (each stage's kernels launched once per sector,
    without a CUDA graph).  Sector tracking is the same as in the batched pass;
    tracks are not merged between sectors, since each call sees one sector."""
    import torch

    from paper_2601_20569_gb300 import synth, tpc

    pieces = []
    for d in dev:
        sec = d[4]
        order = torch.argsort(sec.to(torch.int32), stable=True)
        counts = torch.bincount(sec.to(torch.int64), minlength=36).tolist()
        start = 0
        for c in counts:
            idx = order[start:start + c]
            start += c
            if c:
                pieces.append(tuple(a.index_select(0, idx) for a in d))
    n = sum(int(p[0].shape[0]) for p in pieces)
    tr = tpc.Tracker(synth.row_x(), topts, mode=mode,
                     cap_clusters=max(int(p[0].shape[0]) for p in pieces))
    for p in pieces:
        tr.track(*p, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        for p in pieces:
            tr.track(*p, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    launches = tr.last_launches()
    tr.close()
    ms, nj = reduce_job(e0.elapsed_time(e1), n, world)
    return {"value": nj * steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps,
            "calls_per_step": len(pieces), "kernels_per_call": launches,
            "form": "one tpc_track_timeframe call per (frame, sector): every stage launched "
                    "once per sector, no CUDA graph, no merging between sectors"}


def end_to_end(tr, frames, steps, stream, world):
    """The metric through the public API with host buffers: every step copies
    its frames' clusters from pinned host memory and reads attach[] back, all
    inside the timed region.  The copies run on a stream of their own and
    overlap the tracking of the neighbouring step (two device input buffers;
    attach[] is staged on the device, then read back while the next step
    tracks), as a pipeline over the steps: the first step's upload and the last
    step's read-back are not hidden."""
    import numpy as np
    import torch

    n_per_step = sum(f.n for f in frames)
    host = []
    for f in frames:
        host.append(tuple(torch.from_numpy(np.ascontiguousarray(a)).pin_memory() for a in
                          (f.y, f.z, f.q.view(np.int16), f.row, f.sector)))
    dbufs = [[tuple(torch.empty_like(h, device="cuda") for h in hs) for hs in host]
             for _ in range(2)]
    staged = [torch.empty(n_per_step, dtype=torch.int32, device="cuda") for _ in range(2)]
    attach_host = [torch.empty(n_per_step, dtype=torch.int32).pin_memory() for _ in range(2)]
    h2d = sum(sum(h.numel() * h.element_size() for h in hs) for hs in host)
    d2h = 4 * n_per_step
    cs = torch.cuda.Stream()

    def upload(i):
        with torch.cuda.stream(cs):
            for hs, ds in zip(host, dbufs[i % 2]):
                for h, d in zip(hs, ds):
                    d.copy_(h, non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(cs)
        return ev

    def run(k):
        ev_in = upload(0)
        for i in range(k):
            stream.wait_event(ev_in)
            if i + 1 < k:  # the other buffer's last user (step i - 1) has finished
                ev_in = upload(i + 1)
            tr.track_batch(dbufs[i % 2], stream=stream)
            staged[i % 2].copy_(tr.result_attach(), non_blocking=True)
            ev_out = torch.cuda.Event()
            ev_out.record(stream)
            cs.wait_event(ev_out)
            with torch.cuda.stream(cs):
                attach_host[i % 2].copy_(staged[i % 2], non_blocking=True)
        cs.wait_stream(stream)

    run(2)  # warm: both input buffers once
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(cs)
    run(steps)
    e1.record(cs)
    torch.cuda.synchronize()
    ms, n = reduce_job(e0.elapsed_time(e1), n_per_step, world)
    got = attach_host[(steps - 1) % 2]
    ref = tr.result_attach().cpu()
    assert torch.equal(got, ref), "attach[] read back differs from the device result"
    return {"value": n * steps / (ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": ms / steps,
            "form": "public API (tpc_track_batch) with pinned host clusters in and attach[] out "
                    "every step; copies on a second stream overlap the neighbouring steps' "
                    "tracking (double-buffered inputs)"}


def main():
    args = parse()
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        if rank == 0:
            run_reference(args)
        return
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_2601_20569_gb300 import build as libbuild
    from paper_2601_20569_gb300 import synth, tpc
    from paper_2601_20569_gb300.options import MODE_FAST, MODE_STRICT, TrackerOptions

    libbuild.build()
    note("library built")
    frames = make_frames(args, rank)
    note(f"{len(frames)} frames generated")
    n_per_step = sum(f.n for f in frames)
    mode = MODE_FAST if args.mode == "fast" else MODE_STRICT
    topts = TrackerOptions(ext_rows=args.ext_rows, seed_iters=args.seed_iters,
                           edge_rows=args.edge_rows)
    tr = tpc.Tracker(synth.row_x(), topts, mode=mode, cap_clusters=n_per_step,
                     max_frames=len(frames), use_graphs=True)
    dev = [tr.to_device(f.y, f.z, f.q, f.row, f.sector) for f in frames]
    stream = torch.cuda.current_stream()
    note("inputs resident")
    # launch shapes tuned on two frames of the batch (the frames are alike)
    if args.launch:
        shapes = []
        for x in args.launch.split(","):
            v = [int(t) for t in x.split("x")]
            shapes.append({"block": v[0], "blocks_per_sm": v[1], "lanes": v[2] if len(v) > 2 else 1})
        tr.set_launch_config(shapes)
        tuned = tr.launch_config()
    else:
        tuned = tr.autotune(dev[:2]) if not args.no_autotune else tr.launch_config()
    note("launch shapes chosen")

    def step():
        tr.track_batch(dev, stream=stream)
        return tr.last_launches()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.profile_only:
        step()
        tr.cluster_removal(TrackerOptions(cr_mode=2))  # after the step: listed apart
        torch.cuda.synchronize()
        return

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()

    note("warm-up done")
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            launches += step()
        ev1.record(stream)
        torch.cuda.synchronize()
    barrier()
    ms, n_job = reduce_job(ev0.elapsed_time(ev1), n_per_step, world)
    value = n_job * args.steps / (ms / 1e3)

    note(f"timed region: {ms:.1f} ms")
    # the plain form on the same inputs: one call (one launch per stage) per frame
    plain = tpc.Tracker(synth.row_x(), topts, mode=mode, cap_clusters=max(f.n for f in frames))
    for d in dev:
        plain.track(*d, stream=stream)
    torch.cuda.synchronize()
    p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    p0.record(stream)
    for _ in range(args.steps):
        for d in dev:
            plain.track(*d, stream=stream)
    p1.record(stream)
    torch.cuda.synchronize()
    pm, pn = reduce_job(p0.elapsed_time(p1), n_per_step, world)
    plain_value = pn * args.steps / (pm / 1e3)
    plain.close()

    note("plain per-frame form timed")
    # per-stage device times (CUDA events on the launching stream), a separate pass
    tr.profile(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    stages = tr.stage_stats()
    tr.profile(False)
    tl_n = tr.debug("tl_n")
    first = int(tr.debug("pass_start")[1]) if args.seed_iters > 1 else tl_n.size
    counts = {
        "clusters": n_per_step, "tl_hits": int(tl_n[:first].sum()), "tracklets": first,
        "re_hits": int(tl_n[first:].sum()), "re_tracklets": int(tl_n.size - first),
        "seed_iters": args.seed_iters, "st_hits": int(tr.debug("tl_nkept").sum()),
        "sector_tracks": int(tr.debug("st_key").size), "fit_hits": int(tr.debug("ft_n").sum()),
        "fit_tracks": int(tr.debug("ft_n").size), "fit_stations": int(tr.debug("ft_nst").sum()),
    }
    hbm, peak_kind = peaks()
    # the whole chain is one CUDA-graph launch per step: its algorithmic bytes
    # (92 per input cluster) over the step's CUDA-event time
    chain_bytes = CHAIN_BYTES_PER_CLUSTER * n_per_step
    achieved = chain_bytes / (ms / args.steps / 1e3) / 1e9
    traffic, traffic_src = measured_traffic("chain", counts)
    # the dominant stage alone, with the stage's own byte model
    dom = max(stages, key=lambda s: s["ms"])
    per_call_ms = dom["ms"] / max(1, dom["calls"])
    st_bytes = stage_bytes(dom["name"], counts)
    st_traffic, st_src = measured_traffic(dom["name"], counts)
    roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "traffic": traffic, "traffic_source": traffic_src,
            "kernel": f"whole chain, one CUDA-graph launch of {launches // max(1, args.steps)} "
                      f"kernels per step", "peak_source": f"{peak_kind} hbm_gbs (of {peak_kind})",
            "alg_bytes_per_cluster": CHAIN_BYTES_PER_CLUSTER, "alg_bytes_per_launch": chain_bytes,
            "stage": {"name": dom["name"], "kernels": dom["launches"] // max(1, dom["calls"]),
                      "ms_per_call": per_call_ms, "alg_bytes_per_call": st_bytes,
                      "achieved_gbs": st_bytes / (per_call_ms / 1e3) / 1e9,
                      "stage_frac": st_bytes / (per_call_ms / 1e3) / 1e9 / hbm,
                      "traffic": st_traffic, "traffic_source": st_src}}

    note("stage profile done")
    e2e = end_to_end(tr, frames, args.steps, stream, world)

    note("end-to-end timed")
    # online cluster removal (tpc_cluster_removal, protection 2) on the batch just tracked
    ropts = TrackerOptions(cr_mode=2)
    rem = tr.cluster_removal(ropts)
    torch.cuda.synchronize()
    rem_times = []
    for _ in range(5):  # median of five calls, each between its own events
        r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        r0.record(stream)
        rem = tr.cluster_removal(ropts, stream=stream)
        r1.record(stream)
        torch.cuda.synchronize()
        rem_times.append(r0.elapsed_time(r1))
    rem_ms = statistics.median(rem_times)
    removal = {"ms_per_batch": rem_ms, "clusters_per_s": n_per_step / (rem_ms / 1e3),
               "removed_fraction": rem["n_removed"] / n_per_step,
               "form": "protective / removal tubes with protection 2 and seeding history, "
                       "on the tracks of the batch"}
    note("cluster removal timed")
    tr.close()
    strict = strict_timing(dev, topts, args.steps, args.warmup, stream, world) \
        if args.mode == "fast" else None
    note("strict mode timed")
    per_sector = per_sector_timing(dev, topts, mode, args.steps, stream, world)
    note("per-sector form timed")
    refit = None
    if not args.no_refit:
        refit = refit_timing(mode)
        note("refit and adjoint timed")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: {args.frames} x 2.8 ms frames, 50 kHz Pb-Pb, "
                               f"{n_per_step} clusters per step, one batched pass", "frames": args.frames,
                   "clusters_per_step": n_per_step, "mode": args.mode,
                   "l2": "inputs larger than L2 (each frame > 129 MB resident)",
                   "parallelism": f"replicas x{world}", "launch": "batched + CUDA graph",
                   "phase3_ext_rows": args.ext_rows, "seed_iters": args.seed_iters,
                   "edge_rows": args.edge_rows},
        "roofline": roof,
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "plain_per_frame": {"value": plain_value, "unit": UNIT,
                            "form": "one call per frame (one launch per stage per frame)"},
        "plain_per_sector": per_sector,
        "stages_ms_per_batch": {s_["name"]: s_["ms"] / max(1, s_["calls"]) for s_ in stages},
        "launch_config": tuned,
    }
    line["cluster_removal"] = removal
    # measured FMA peaks (the ncu pipe utilisation of the fit kernels is read
    # against them)
    line["arith_peaks"] = {"fp32_fma_tflops": tpc.Tracker.fma_peak(False),
                           "fp64_fma_tflops": tpc.Tracker.fma_peak(True, iters=256),
                           "how": "tpc_fma_peak: 8 independent FMA chains per thread, "
                                  "8 x 256 threads per SM, CUDA events"}
    if strict is not None:
        line["strict"] = strict
    if refit is not None:
        line["refit_adjoint"] = refit
    if rank == 0 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(frames, args.cpu_seconds)
        note("cpu baseline done")
        line["cpu_baseline_parallel"] = cpu_baseline_parallel(frames)
        note("parallel cpu baseline done")
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


if __name__ == "__main__":
    main()
