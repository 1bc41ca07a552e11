/* tpc.h -- C ABI of the GB300 TPC time-frame tracker (libtpc.so).
 *
 * Reconstructs TPC tracks from the clusters of one continuous-readout time
 * frame, following the three phases of the paper's Sec. 2 ("sector tracking,
 * track merging and track fit") with the Phase I/II fit of Sec. 3:
 *
 *   per-row cluster grids -> cellular-automaton neighbour finding and cleaning
 *   -> start hits -> Kalman tracklet construction -> ambiguity solving
 *   -> sector refit and sector-to-sector merging -> three-iteration refit with
 *   space-charge distortion correction and inner-region re-attachment.
 *
 * Conventions
 *   - Sector s in 0..35: side A (z > 0) is 0..17, side C is 18..35; sector
 *     axis at azimuth ((s % 18) + 0.5) * 20 deg; local x along the axis (pad
 *     row normal), y along the row, z the measured drift coordinate [cm].
 *   - Track state at x: (y, z, sin(phi), tan(lambda), q/pT [c/GeV]); the
 *     covariance is stored as 15 floats, lower triangle row by row
 *     (yy, zy, zz, sy, sz, ss, ty, tz, ts, tt, qy, qz, qs, qt, qq).
 *   - A cluster id is its index in the caller's input arrays.
 *
 * Ownership and errors
 *   - Input pointers marked "device" are caller-owned CUDA device memory,
 *     read-only and valid for the duration of the call.
 *   - Output buffers (tpc_tracks) are owned by the context and stay valid
 *     until the next call on the same context.
 *   - Every call returns a tpc_status; no C++ exception crosses the ABI.  A
 *     failed call leaves a message for tpc_last_error().  Work is enqueued on
 *     the caller's stream; device-detected errors (invalid cluster, capacity)
 *     are read back at the end of the call with one small copy, which makes
 *     the call synchronous with respect to that stream.
 *   - One context serves one stream at a time (calls are not thread-safe on
 *     the same context).
 */
#ifndef TPC_H
#define TPC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TPC_OK = 0,
  TPC_ERR_INVALID_ARG = 1,   /* null pointer, bad size or option */
  TPC_ERR_INVALID_INPUT = 2, /* NaN/Inf coordinate, row >= n_rows, sector >= n_sectors,
                                or more than 1024 clusters in one search-grid bin (many
                                clusters at one point of a row) */
  TPC_ERR_CAPACITY = 3,      /* an internal buffer is too small; *needed reports the size */
  TPC_ERR_CUDA = 4,          /* a CUDA runtime call failed */
  TPC_ERR_OOM = 5,           /* device allocation failed */
  TPC_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
  TPC_ERR_STATE = 7          /* call order violated (e.g. backward without refit) */
} tpc_status;

typedef struct tpc_ctx tpc_ctx;

/* Detector geometry (host memory, copied at init).  row_x: n_rows pad-row
 * radii [cm], increasing. */
typedef struct {
  int32_t n_sectors; /* 36 */
  int32_t n_rows;    /* 152 */
  const float* row_x;
} tpc_geometry;

/* Space-charge correction map: uniform cubic B-spline control points,
 * [3][n_z][n_r][n_phi] floats (components dx, dy, dz in sector-local cm, added
 * to a measured cluster).  phi is periodic over the 18 azimuthal sectors
 * (coordinate u = sector + 0.5 + 0.5*(y/x)/tan(10 deg), control point j at
 * u = (j + 0.5) * 18 / n_phi); r = sqrt(x^2 + y^2) spans [r_min, r_max] and z
 * [z_min, z_max] with clamping, control point j at t = j - 1 knot spacings.
 * coeff is a device pointer; NULL means no correction. */
typedef struct {
  int32_t n_phi, n_r, n_z;
  float r_min, r_max, z_min, z_max;
  const float* coeff;
} tpc_map;

/* Reconstruction options: physical inputs and every cut (the paper states the
 * cuts only qualitatively; defaults are given in the Python binding). */
typedef struct {
  float bz;                 /* tesla */
  float sigma_y, sigma_z;   /* cluster resolution [cm] */
  float ms_theta;           /* multiple-scattering angle per pad row [rad] */
  float link_wy, link_wz;   /* CA neighbour search window [cm] */
  float link_chi2;          /* max squared distance of the middle cluster to the d-u line [cm^2] */
  float seed_c[5];          /* seed covariance diagonal */
  float follow_chi2;        /* cluster pick-up cut of the track following (2 dof) */
  float max_snp;            /* |sin(phi)| limit of seeding and following */
  float fit_max_snp;        /* |sin(phi)| limit of refits, merging and the final fit */
  float score_w;            /* ambiguity score = n_clusters - score_w * chi2/ndf */
  float shared_frac;        /* allowed shared-cluster fraction (paper default 10 %) */
  float merge_chi2, merge_dy, merge_dz; /* merging: 5-dof chi2 cut and position gates */
  float int_chi2;           /* interpolation cut of fit iteration 2, candidate cut (2 dof) */
  float final_chi2;         /* simple chi2 cut of fit iteration 3 */
  float attach_margin;      /* widening of the Phase II search window [cm] */
  float edge_margin;        /* following stops at |y| > x*tan(10 deg) + edge_margin [cm] */
  float looper_qpt;         /* |q/pT| above which the final fit's Kalman update runs in FP64
                               (low-pT loopers); 0 disables */
  float ext_chi2;           /* Phase III: candidate cut of the extrapolation (2 dof) */
  int32_t max_miss;         /* consecutive empty rows ending the following */
  int32_t min_hits;         /* minimum clusters of a tracklet / track */
  int32_t merge_max_gap;    /* max rows between merged segments */
  int32_t inner_rows;       /* rows of the inner region (Phase II re-attachment) */
  int32_t cand_k;           /* candidates kept per (track, row), <= 8 */
  int32_t mode;             /* 0 = strict FP32 (no FMA), 1 = fast FP32 (FMA) */
  int32_t max_frames;       /* frames per tpc_track_batch call (<= 64; 0 or 1: single frames) */
  int32_t use_graphs;       /* 1: replay each call's chain from a captured CUDA graph */
  int32_t ext_rows;         /* Phase III (Sec. 3): rows below a track's innermost and above its
                               outermost cluster searched by extrapolation, 0..32 (0: off) */
  int32_t seed_iters;       /* Sec. 3: sector-tracking iterations, 1..4; every later one runs the
                               neighbour finding, tracklet construction and selection again on
                               the clusters that no accepted tracklet of the earlier ones kept
                               (0 or 1: off) */
  int32_t ac_merge;         /* 1: merging also across the central electrode (Sec. 2), the far
                               side's z shifted by the estimated 2 vd t0 (Sec. 1); 0: off */
  int32_t edge_rows;        /* edge following (Sec. 2: tracks ending at a sector edge are
                               propagated into the adjacent sector before the merging and
                               followed there): rows followed beyond each track end, 0..152
                               (0: off; on, cap_clusters <= 2^29) */
  int32_t edge_min;         /* clusters a segment found by the edge following needs (>= 1) */
  int64_t cap_clusters;     /* max clusters per call (all frames of a batch) */
  int64_t cap_tracklets;    /* max tracklets per frame (0: n/16 + 4096) */
  int64_t cap_tracks;       /* max tracks per frame (0: cap_tracklets) */
} tpc_options;

/* Clusters of one time frame (device memory, structure of arrays). */
typedef struct {
  int64_t n;
  const float* y;
  const float* z;
  const uint16_t* q;   /* carried, unused by the tracking */
  const uint8_t* row;
  const uint8_t* sector;
} tpc_clusters;

/* Tracks of one frame (device memory owned by the context). */
typedef struct {
  int64_t n_tracks;
  int64_t n_cluster_refs;
  const float* params;      /* [n_tracks][5] at the innermost cluster */
  const float* cov;         /* [n_tracks][15] */
  const float* chi2;        /* [n_tracks] */
  const float* x;           /* [n_tracks] local x of params */
  const int32_t* ndf;       /* [n_tracks] */
  const int32_t* sector;    /* [n_tracks] sector frame of params */
  const int32_t* n_clusters;/* [n_tracks] */
  const int32_t* cl_offset; /* [n_tracks + 1] CSR offsets into cl_ids */
  const int32_t* cl_ids;    /* cluster ids, innermost first */
  const int32_t* key;       /* [n_tracks] identity: input id of the start cluster of
                               the track's first segment */
  const int32_t* attach;    /* [n_clusters of the frame]: owning track index or -1 */
  const float* z_shift;     /* [n_tracks] tracks merged across the central electrode: shift
                               added to the measured z of their clusters on the side other than
                               that of their innermost cluster (= -2 * side * vd * t0); else 0 */
} tpc_tracks;

/* Create a context: copies the geometry, derives the model constants from
 * bz and the options, allocates device buffers for opt->cap_clusters
 * clusters.  map may be NULL.  Sec. 2 (sector structure), Sec. 5 (the
 * deterministic mode is mode 0). */
tpc_status tpc_init(const tpc_geometry* geo, float bz_tesla, const tpc_map* map,
                    const tpc_options* opt, tpc_ctx** out);

/* Track one time frame (Sec. 1: the time frame is the unit of reconstruction;
 * Sec. 2: sector tracking, merging, fit; Sec. 3: Phase I/II fit).  On
 * TPC_ERR_CAPACITY, *needed (if not NULL) receives the required size of the
 * buffer that overflowed. */
tpc_status tpc_track_timeframe(tpc_ctx* ctx, const tpc_clusters* clusters, tpc_tracks* out,
                               void* cuda_stream, int64_t* needed);

/* Refit of given tracks with fixed cluster lists (the fit of Sec. 2/3 without
 * the Phase II search) and the data its adjoint needs.  clusters: the frame's
 * device clusters; in: tracks with cl_offset/cl_ids (innermost first) and
 * start parameters params/x/sector (e.g. the output of tpc_track_timeframe);
 * map: correction map (NULL: the context's).  An extended-Kalman pass over
 * the uncorrected clusters gives the start; iterations 1-3 use the corrected
 * clusters, linearised about references taken from the previous iteration's
 * end (Sec. 2: the initial parameters are used for the linearisation).  With
 * freeze != 0 the references and the discrete decisions (interpolation flags,
 * the final cut) of the previous refit of the same tracks are reused, making
 * the chi2 a smooth function of the map (TPC_ERR_STATE otherwise).  out:
 * chi2, ndf, n_clusters and parameters of every input track (same order);
 * cl_offset/cl_ids/key/attach/z_shift are passed through from `in`.  in->z_shift
 * may be NULL; where given (tracks merged across the central electrode), each
 * track's clusters on the side other than its innermost cluster's enter the
 * refit and the adjoint with their z plus the shift.  `in` and its arrays must
 * stay valid until the matching tpc_refit_backward.  Synchronous.
 * Not in the paper: the differentiable form serves distortion calibration
 * (Sec. 2 names the space-charge correction maps as the limiting factor). */
tpc_status tpc_refit(tpc_ctx* ctx, const tpc_clusters* clusters, const tpc_tracks* in,
                     const tpc_map* map, int32_t freeze, tpc_tracks* out, void* cuda_stream);

/* Gradient of L = sum_t dL_dchi2[t] * chi2_t of the last tpc_refit with
 * respect to the map control points, references and decisions held fixed:
 * a hand-written adjoint sweeping iterations 3, 2, 1 in reverse with the
 * filter recomputed from checkpoints every 16 stations; per-track work in
 * FP32, the cross-track reduction in FP64.  dL_dchi2: device float[n_tracks];
 * dL_dmap: device float[3*n_z*n_r*n_phi] (overwritten).  TPC_ERR_STATE
 * without a preceding refit that used a map. */
tpc_status tpc_refit_backward(tpc_ctx* ctx, const float* dL_dchi2, float* dL_dmap,
                              void* cuda_stream);

/* Online cluster removal (Sec. 4, cluster reduction) on the tracks of the
 * last successful tpc_track_timeframe / tpc_track_batch call of this
 * context.  Clusters inside a protective tube around physics tracks are kept;
 * of the others, those inside a removal tube around secondary legs of
 * looping tracks and around very-low-pT tracks are flagged for removal; the
 * clusters of the tracklets a physics track was seeded from (its history)
 * are protected as well.  The section states the rules in words; these are
 * the readings:
 *  - a track is very low pT if |q/pT| at its innermost cluster exceeds qpt;
 *  - two looper tracks (|q/pT| above the tracker's looper_qpt) of one side are
 *    legs of one looper if their |q/pT| differ by at most leg_dq relative,
 *    their tan(lambda) are opposite within leg_dtgl and their circle centres
 *    (global x, y) lie within leg_dc cm; of linked legs the one with the
 *    smallest side*z at its innermost cluster comes first (track key on exact
 *    ties), every other one is a secondary leg whose parent is the first
 *    earlier leg;
 *  - a tube follows the track's clusters (linear interpolation from the
 *    lower-row cluster over rows between two clusters of one sector) and holds
 *    the clusters of each row within the half-width in y and z;
 *  - protection 1 is the choice protect > remove; protection 2 (mode 2)
 *    multiplies the protective tube by p2_grow and the removal tube by
 *    p2_shrink on the tracker's inner_rows innermost rows, within edge cm of a
 *    sector edge and where more than occ_max clusters lie within occ_w cm of
 *    the tube centre.
 * Strict mode gives the CPU oracle's flags bit for bit. */
typedef struct {
  float qpt;         /* |q/pT| above which a track is very low pT [1/GeV] */
  float protect;     /* protective tube half-width around physics tracks [cm] */
  float remove;      /* removal tube half-width [cm] */
  float edge;        /* protection 2: sector-edge band [cm] */
  float occ_w;       /* protection 2: occupancy window half-width [cm] */
  float p2_grow;     /* protection 2: factor on the protective tube */
  float p2_shrink;   /* protection 2: factor on the removal tube */
  float leg_dq;      /* looper legs: relative |q/pT| difference */
  float leg_dtgl;    /* looper legs: |tan(lambda_a) + tan(lambda_b)| */
  float leg_dc;      /* looper legs: circle-centre distance [cm], > 0 */
  int32_t mode;      /* 1: tubes + history, 2: also protection 2 */
  int32_t occ_max;   /* protection 2: occupancy threshold */
} tpc_removal_options;

/* Results (device memory owned by the context, valid until its next call). */
typedef struct {
  int64_t n_clusters;          /* clusters of the last tracking call (all frames of a batch) */
  int64_t n_tracks;            /* tracks of the last tracking call */
  int64_t n_removed;           /* clusters flagged 8 */
  const uint8_t* flags;        /* [n_clusters] by input (batch) id: 1 in a protective tube,
                                  2 seeding history of a physics track, 4 in a removal tube,
                                  8 removed (4 and neither 1 nor 2) */
  const int32_t* track_class;  /* [n_tracks] 0 physics, 1 very low pT, 2 secondary looper leg */
  const int32_t* leg_parent;   /* [n_tracks] index of the first earlier leg of a secondary
                                  leg, else -1 */
} tpc_removal;

/* Errors: TPC_ERR_INVALID_ARG for null pointers or options out of range,
 * TPC_ERR_STATE without a preceding successful tracking call, TPC_ERR_CUDA. */
tpc_status tpc_cluster_removal(tpc_ctx* ctx, const tpc_removal_options* opt, tpc_removal* out,
                               void* cuda_stream);

/* Track several time frames in one pass: the frames are concatenated (frame
 * f's sector s becomes batch sector f*n_sectors + s, its cluster i batch id
 * sum_{g<f} n_g + i) and every stage runs once over all of them, the heavy
 * kernels as persistent grids pulling tracks from device-side work queues so
 * that sectors and frames of very uneven occupancy balance.  Results are
 * those of tracking each frame alone; tracks report batch sectors and batch
 * cluster ids.  n_frames <= opt->max_frames of tpc_init.  (Not in the paper,
 * which processes one time frame at a time: Sec. 1.) */
tpc_status tpc_track_batch(tpc_ctx* ctx, const tpc_clusters* frames, int32_t n_frames,
                           tpc_tracks* out, void* cuda_stream, int64_t* needed);

/* Autotuner: times the heavy kernels (tracklet construction, sector refit,
 * merging, fit iterations) over block sizes {64, 128, 256} x {4, 8, 16}
 * blocks per SM on the given frames (tracked as one batch) and keeps the
 * fastest shape per kernel for later calls (the analogue of the paper's
 * automatic tuning of threads and blocks per GPU, Sec. 5). */
tpc_status tpc_autotune(tpc_ctx* ctx, const tpc_clusters* frames, int32_t n_frames,
                        void* cuda_stream);

/* Launch shape chosen for heavy kernel `slot` (0..5): kernel name, block
 * size, blocks per SM, lanes per work item (1 = one thread per item; the
 * merge search of slot 2 runs one item on a group of 1, 4, 8, 16 or 32
 * lanes, the neighbour search of slot 5 one cluster on 1, 4 or 8 lanes, or
 * 32 clusters per warp with their candidates staged in shared memory (lanes =
 * 32), in one launch of 256-thread blocks over the clusters).  Any output pointer may
 * be NULL.  TPC_ERR_INVALID_ARG past the last slot. */
tpc_status tpc_launch_config(const tpc_ctx* ctx, int32_t slot, const char** kernel,
                             int32_t* block, int32_t* blocks_per_sm, int32_t* lanes);

/* Set the launch shape of heavy kernel `slot` (0..5, as tpc_launch_config
 * numbers them), e.g. to reapply a shape the autotuner chose earlier on the
 * same GPU.  block: multiple of 32 in [32, 256] (the kernels are compiled for
 * at most 256 threads per block); blocks_per_sm in [1, 32]; lanes: 1, or for
 * slot 2 (merge search) one of 4, 8, 16, 32, for slot 5 (neighbour search)
 * 4, 8 or 32 (slot 5 uses only its lanes).
 * The shape changes only scheduling: results are identical for every shape.
 * TPC_ERR_INVALID_ARG for any other value. */
tpc_status tpc_set_launch_config(tpc_ctx* ctx, int32_t slot, int32_t block,
                                 int32_t blocks_per_sm, int32_t lanes);

/* Replace the correction map (device pointer copied by reference; the caller
 * keeps it alive while the context uses it).  Any CUDA graph the context
 * captured with the previous map is recaptured on the next call. */
tpc_status tpc_set_map(tpc_ctx* ctx, const tpc_map* map);

/* Copy an internal per-stage buffer to host memory (testing and debugging).
 * name selects the buffer; *bytes receives its size; nothing is copied when
 * cap_bytes is too small (TPC_ERR_CAPACITY).  Synchronises the last stream. */
tpc_status tpc_debug_copy(tpc_ctx* ctx, const char* name, void* host_dst, int64_t cap_bytes,
                          int64_t* bytes);

/* Per-stage timing: when enabled, every tracking call records CUDA events
 * on its stream between the hot-path stages and accumulates their durations
 * (enabling resets the totals). */
tpc_status tpc_profile(tpc_ctx* ctx, int enable);

/* Totals of stage i (0-based, in execution order): name, summed milliseconds,
 * number of profiled calls, kernels launched.  TPC_ERR_INVALID_ARG past the
 * last stage. */
tpc_status tpc_stage_stats(const tpc_ctx* ctx, int32_t i, const char** name, double* ms_total,
                           int64_t* calls, int64_t* launches);

/* Kernels launched by the last tracking call. */
int64_t tpc_last_launches(const tpc_ctx* ctx);

/* Measured arithmetic peak of the current device, for reading the pipe
 * utilisation of the kernels against it: fused multiply-add throughput in
 * TFLOP/s (2 flops per FMA) of a kernel of eight independent FMA chains per
 * thread, `iters` x 128 FMAs per thread, 8 blocks of 256 threads per SM,
 * timed with CUDA events on `cuda_stream` (synchronous).  fp64 != 0 measures
 * double precision.  Allocates and frees a small result buffer (stream-ordered).
 * Not in the paper. */
tpc_status tpc_fma_peak(int32_t fp64, int32_t iters, double* tflops, void* cuda_stream);

/* Number of successful tpc_refit calls on this context (-1 for a null
 * context).  tpc_refit_backward differentiates the most recent refit only; a
 * caller that keeps a refit for a later backward pass (an autograd graph)
 * records this number after the refit and checks it before the backward
 * call, so that a refit run in between is detected instead of silently
 * differentiated. */
int64_t tpc_refit_generation(const tpc_ctx* ctx);

/* Allocation-free cellular-automaton links (this entry point has no
 * counterpart in the paper; it serves callers that may not allocate device
 * memory while they run -- code inside an allocator or memory-pool callback,
 * runtimes that reserve all device memory up front, real-time loops where
 * allocation is not allowed).
 *
 * Computes the same cleaned neighbour links as tpc_track_timeframe in strict
 * mode (per-row grids, best straight-line pair per cluster, mutual cleaning)
 * for one frame of at most TPC_NOALLOC_MAX_CLUSTERS clusters, without any
 * cudaMalloc: its working buffers (about 7.3 MB) are one static device array
 * that every GPU loading the library holds until the process exits.
 *   geo, opt: host structs as for tpc_init (opt->bz is the field; capacities
 *             and mode are ignored).  clusters: device SoA, caller-owned.
 *   link_up, link_dn: caller-owned device int32[clusters->n], receive the
 *             input id of the cluster linked on the next / previous pad row
 *             or -1.
 * Errors: TPC_ERR_CAPACITY when n exceeds TPC_NOALLOC_MAX_CLUSTERS (nothing
 * is launched) or the per-row grid would not fit; TPC_ERR_INVALID_INPUT for
 * NaN/Inf coordinates or out-of-range row/sector; TPC_ERR_INVALID_ARG for bad
 * pointers or a geometry with more than 36*160 (sector, row) pairs.
 * The call synchronises the stream.  All calls share the one array, which
 * keeps the last call's contents; calls whose GPU work overlaps (other
 * streams or host threads) race on it and must be serialised by the caller.
 * The first call on a device looks up the array's device address with that
 * device current; make it before any stream capture. */
#define TPC_NOALLOC_MAX_CLUSTERS 65536
tpc_status tpc_links_noalloc(const tpc_geometry* geo, const tpc_options* opt,
                             const tpc_clusters* clusters, int32_t* link_up, int32_t* link_dn,
                             void* cuda_stream);

/* Message of the last failed call on this context (never NULL). */
const char* tpc_last_error(const tpc_ctx* ctx);

/* Release all device memory of the context. */
void tpc_destroy(tpc_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* TPC_H */
