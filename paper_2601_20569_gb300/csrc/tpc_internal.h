// Internal types of the CUDA tracker shared by the host orchestration and the
// kernels (never exported through the C ABI).
#pragma once

#include <cstdint>

#include <vector_types.h>

namespace tpc {

constexpr int kMaxRows = 160;      // pad rows supported by the per-tracklet row arrays
constexpr int kMaxCand = 8;        // Phase II candidates per (track, row)

// Derived model constants and cuts, passed by value to every kernel.
struct KParams {
  float kb;          // curvature per unit q/pT, -Bz * 0.00299792458
  float tan_half;    // tan(10 deg)
  float rot_c, rot_s;  // cos/sin of 20 deg
  float sy2, sz2;    // measurement variances
  float ms2;         // scattering angle variance per row
  float pitch_inv;   // rows per cm
  float link_wy, link_wz, link_chi2;
  float seed_c[5];
  float follow_chi2, max_snp, fit_max_snp, score_w, shared_frac;
  float merge_chi2, merge_dy, merge_dz, merge_zspan;
  float int_chi2, final_chi2, attach_margin, edge_margin, looper_qpt, ext_chi2;
  int max_miss, min_hits, merge_max_gap, inner_rows, cand_k, ext_rows;
  int seed_iters;  // sector-tracking iterations (the later ones on leftover clusters)
  int ac_merge;    // merging across the central electrode
  int edge_rows;   // edge following: rows followed beyond a track end (0: off)
  int edge_min;    // edge following: clusters a segment needs
  int n_rows, n_sectors;  // n_sectors: all sectors of the call (frames x sectors)
  int n_phi;         // azimuthal sectors of one TPC half (sector % n_phi, side = sector / n_phi)
  float grid_dy;     // smallest y bin size [cm]
  float grid_occ;    // target clusters per bin
};

// Options of the online cluster removal (Sec. 4), derived on the host.
struct RemovalParams {
  float qpt, protect, remove, edge, occ_w, p2_grow, p2_shrink, leg_dq, leg_dtgl, leg_dc;
  float inv_cell;          // 1 / width of a centre bin (at least the leg distance)
  int mode, occ_max, nbx;  // nbx: centre bins per axis and side block over [-256, 256) cm
  int half, nsec_frame;    // sectors per side and per frame
  float sec_cos[18], sec_sin[18];  // sector axis ((s mod 18) + 0.5) * 20 deg
};

// Launch shape of the heavy per-item kernels (block size, blocks per SM),
// chosen by the autotuner.
enum LaunchSlot : int { kLTracklets = 0, kLSectorRefit, kLMerge, kLFit12, kLFit3, kLLinks, kLNum };
struct LaunchCfg {
  int block[kLNum];
  int per_sm[kLNum];
  int lanes[kLNum];  // lanes per work item (1: one thread per item; the merge search: 1..32)
};

// Work queues: counters of the dynamic item fetching (zeroed per call).
// The fit kernels keep two queues each: loopers (kQFit12, kQFit3) and the
// other tracks (kQFit12N, kQFit3N).
enum QueueSlot : int {
  kQTracklets = 0, kQSectorRefit, kQMerge, kQFit12, kQFit3, kQFit12N, kQFit3N, kQFit2, kQFit2N,
  kQTlDown, kQTlUp, kQTlRefit, kQNum
};

// Search grid of one (sector, row): bins iz*nY + iy, clusters of a bin are
// contiguous in the sorted arrays.
// One 32-byte record per (sector, row), so that a search reads it with one
// aligned sector; the row's clusters start at the sum of ncl over the rows
// before it.
struct __align__(32) RowGrid {
  int bin0;   // first global bin
  int nY, nZ;
  int ncl;
  float y0, invDy, z0, invDz;
};

// Device error word bits.
enum : int {
  kErrInput = 1,
  kErrCapTracklets = 2,
  kErrCapBins = 4,
  kErrCapTracks = 8,
  kErrCapRefs = 16,
  kErrCapCand = 32,
  kErrDense = 64,    // a search bin holds more than kMaxBinOcc clusters
  kErrCapPos = 128,  // kept-cluster positions of the sector tracks
  kErrCapEdge = 256, // segments of the edge following beyond the tracklet capacity
};

// Largest number of clusters one search bin may hold.  Bins are sized for a
// few clusters each; a frame that piles more than this into one bin (many
// clusters at one point of a row) is rejected as invalid input, which keeps
// the per-bin ordering and the window searches bounded.
constexpr int kMaxBinOcc = 1024;

constexpr int kStateF = 22;     // p[5], c[15], x, sector (as float)
constexpr int kSeedF = 8;       // tracklet seed: p[5], x, sector*n_rows + row, valid
constexpr int kIpolF = 11;      // interpolation record of an inner station
constexpr int kMergeLanesDefault = 16;  // lanes per outer end in the merge search
constexpr int kLinksLanesDefault = 1;   // lanes per cluster in the neighbour search (32: staged per warp)
constexpr int kMergeZ = 512;     // z bins per sector of the merge candidate index
constexpr int kMaxInner = 32;    // inner-region rows supported
constexpr int kMaxSeedIters = 4;  // sector-tracking iterations
constexpr int kCrMaxBinsX = 170;   // cluster removal: circle-centre bins per axis and side block
constexpr int kCrBins = 128 * kCrMaxBinsX * kCrMaxBinsX;  // 64 frames x 2 sides
constexpr int kMaxExt = 32;      // Phase III: rows extrapolated below a track (slots after the inner ones)
// Scheduling buckets of the sector refit (most clusters first).
constexpr int kOrdBuckets = 128;

// Distortion map as seen by the kernels.
struct MapDev {
  int on;
  int nphi, nr, nz;
  float rmin, zmin, zmax;
  float phi_scale, r_scale, z_scale;
  const float* c;
};

// Small device-side counters read back at the end of a call.
struct Counters {
  int err;
  int n_starts;
  int n_bins;
  int n_tracks;      // accepted sector tracks
  int n_merged;      // final tracks after merging
  int n_refs;        // cluster references of the final tracks
  int n_cand;
  int need_tracklets;
  int need_tracks;
  int n_out;         // output tracks
  int queue[kQNum];  // work-queue heads
  int n_loopers;     // fit tracks whose updates run in FP64
  int n_pos;         // kept-cluster positions of the sector tracks
  int tl_base;       // first tracklet of the current sector-tracking iteration
  int n_new;         // start hits found by the current iteration
  int pass_start[kMaxSeedIters];  // first tracklet of each iteration
  int n_removed;     // cluster removal: clusters flagged for removal
  int n_st0;         // edge following: sector tracks before the segments were added
  int n_tl_all;      // edge following: tracklet slots in use before the segments
};

// One frame of a batch call, read in place: the clusters of batch index i
// with off <= i < off + n are this frame's clusters i - off.
struct FrameSrc {
  const float* y;
  const float* z;
  const uint8_t* row;
  const uint8_t* sector;
  long off;
};

// Working set of one frame on the device.
struct FrameDev {
  // input
  const float* y;
  const float* z;
  const uint8_t* row;
  const uint8_t* sector;
  const FrameSrc* src;     // batch calls: the frames' own arrays ([nsrc], device);
  int nsrc;                // 0: one frame, read through y, z, row, sector
  int src_nsec;            // sectors per frame (batch sector = frame * src_nsec + sector)
  long n;
  const float* row_x;  // [n_rows]
  // a1 grid
  int* row_cnt;            // [n_sectors*n_rows]
  unsigned* row_zmin;      // ordered-int encoded
  unsigned* row_zmax;
  RowGrid* rows;           // [n_sectors*n_rows]
  int* row_first;          // [n_sectors*n_rows + 1] first sorted cluster of each row
  int* bin_cnt;            // [cap_bins + 1]
  int* bin_first;          // [cap_bins + 1]
  int* cl_bin;             // [n] per input cluster
  int* cl_slot;            // [n]
  long cap_bins;
  int4* srec;              // [n] grid build: (y, z, input id, bin) scattered to the sorted
                           // positions, ordered in each bin and split into syz / sid
  float2* syz;             // [n] sorted (y, z)
  int* sid;                // sorted -> input id
  uint16_t* srow;          // sorted -> sector*n_rows + row
  // a2/a3
  int* lup;
  int* ldn;
  int* cup;
  int* cdn;
  // a4
  int* flags;              // [n] scratch for compaction
  int* scan_tmp;           // block partials
  int* starts;             // [cap_tl]
  // a5
  long cap_tl;
  float* tl_par;           // [cap_tl*5]
  float* tl_cov;           // [cap_tl*15]
  float* tl_x;
  float* tl_chi2;
  unsigned long long* tl_key;  // ambiguity key of a finished tracklet (tl_n > 0)
  int* tl_n;
  int* tl_rlo;
  int* tl_rhi;
  int* tl_hits;            // [cap_tl*kMaxRows] row-indexed sorted cluster or -1
  int* tl_len;             // [cap_tl] CA chain length from the start hit
  float* tl_seed;          // [cap_tl][kSeedF] seed state, start (sector, row), valid flag
  // a6
  unsigned long long* owner_key;  // [n] sorted index space
  int* tl_acc;
  int* tl_nkept;
  int* tl_kept;            // [cap_tl*kMaxRows] outermost first
  int* sec_owner;          // [n] sorted index space: tracklet index or -1
  uint8_t* st_kept;        // [n] edge following: sorted cluster kept by a sector track
  int* edge_flag;          // [2 * cap_tl + 1] edge following: end (2 j + inner) found a segment
  int* edge_pos;           // [2 * cap_tl + 1] its exclusive prefix sum (segment index)
  uint8_t* sused;          // [n] sorted cluster taken by an accepted tracklet of an earlier
                           // sector-tracking iteration (iterations after the first)
  // online cluster removal (after a tracking call)
  unsigned* cr_flags;      // [n] sorted index space: 1 protective tube, 2 seeding history,
                           // 4 removal tube, 8 removed
  uint8_t* cr_out;         // [n] the flags in input order
  int* cr_cls;             // [cap_ft] per output track: 0 physics, 1 very low pT, 2 secondary leg
  int* cr_parent;          // [cap_ft] first leg of a secondary leg's looper, or -1
  float* cr_cx;            // [cap_ft] circle centre, global x [cm]
  float* cr_cy;            // [cap_ft] circle centre, global y [cm]
  float* cr_zk;            // [cap_ft] side * z at the innermost cluster (leg order)
  int* cr_bin_cnt;         // [kCrBins + 1] loopers per (side block, centre bin)
  int* cr_bin_first;       // [kCrBins + 1]
  int* cr_bin_items;       // [cap_ft]
  Counters* cnt;

  // a7 sector tracks (capacity cap_tl)
  int* st_tl;              // tracklet index of each accepted tracklet
  int* st_off;             // first entry of the track's kept-cluster positions
  float4* st_pos;          // [cap_pos] (x, y, z, -) of kept clusters, outermost first per track
  long cap_pos;
  int* st_order;           // order in which the sector refit takes the tracks
  int* st_obucket;         // scheduling bucket
  int* st_oslot;           // place within the bucket
  int* st_ord_cnt;         // [kOrdBuckets]
  int* st_ok;
  int* st_key;             // input id of the start cluster
  int* st_sector;
  int* st_rmin;
  int* st_rmax;
  float* st_ie;            // [cap_tl][kStateF] state at the innermost cluster
  float* st_oe;            // [cap_tl][kStateF] state at the outermost cluster
  int* st_next;
  int* st_hasprev;
  int* st_bestB;
  float* st_bestchi;
  unsigned long long* st_bestA;
  // merging across the central electrode
  int* st_xbestB;          // best chain start on the other side of a chain end
  float* st_xchi;
  float* st_xdz;           // z shift of that candidate's side
  unsigned long long* st_xbestA;
  float* st_dz;            // z shift of the side that starts at this sector track (0: none)
  int* ie_cnt;             // [n_sectors*kMergeZ*n_rows]
  int* ie_first;           // [n_sectors*kMergeZ*n_rows + 1]
  int* ie_slot;            // [cap_tl]
  int* ie_bin;             // [cap_tl]
  int* ie_idx;             // [cap_tl] sector tracks sorted by (sector, z bin)
  float4* ie_rec;          // [cap_tl] in index order: inner end (y, z, x) and track id bits
  float* sec_zlo;          // [n_sectors]
  float* sec_zinv;         // [n_sectors]

  // a9/a10 fit tracks (capacity cap_ft)
  long cap_ft;
  int* ft_head;            // first sector track of the chain
  int* ft_side0;           // TPC side of the first segment
  float* ft_zsh;           // z shift of the clusters on the other side (0: one side only)
  int* ft_last;            // last sector track of the chain
  int* ft_order;           // [cap_ft] order in which the fit kernels take the tracks:
                           // FP64-update loopers first, then the rest, each in list order
  int* ft_looper;          // [cap_ft] 1: |q/pT| of the chain's inner end above looper_qpt
  int* ft_key;
  int* ft_ok;
  int* ft_nst;             // stations
  float* ft_z0;
  int* ft_st_cl;           // [cap_ft][kMaxRows] sorted cluster or -1
  uint16_t* ft_st_rs;      // [cap_ft][kMaxRows] sector*n_rows + row
  float* ft_store;         // [cap_ft][kMaxRows][5] iteration-1 predictions
  uint8_t* ft_flag;        // [cap_ft][kMaxRows]
  float* ft_end2;          // [cap_ft][kStateF] end of iteration 2 (+ sector)
  // candidate slots per fit track: nslot = kMaxInner inner-station slots
  // (station k) followed by ext_rows extrapolation slots (row r_first - 1 - e)
  // and ext_rows outward slots (row r_last + 1 + e)
  int nslot;
  uint8_t* ft_ncand;       // [cap_ft][nslot]
  int* ft_cand;            // [cap_ft][nslot][kMaxCand]
  float* ft_cchi;          // [cap_ft][nslot][kMaxCand]
  int* ft_assigned;        // [cap_ft][nslot]
  uint8_t* ft_newly;       // [cap_ft][nslot]
  int* ft_next;            // [cap_ft] rows extrapolated below the innermost station
  int* ft_nout;            // [cap_ft] rows extrapolated above the outermost station
  uint16_t* ft_ext_sec;    // [cap_ft][2 ext_rows] sector of each extrapolated row (inward,
                           // then outward): the extrapolation may cross a sector edge
  float* ft_ipol;          // [cap_ft][kMaxInner][kIpolF] iteration-2 interpolation at inner
                           // stations (y, z, Cyy, Cyz, Czz, x, reference p[5]) for k_inner_cand
  uint8_t* ft_fixed;       // [n] sorted cluster held by a station outside the inner region
  unsigned long long* bid; // [n] per sorted cluster
  uint8_t* taken;          // [n]
  int* ft_n;               // iteration 3 results
  float* ft_chi2;
  float* ft_out;           // [cap_ft][kStateF]
  int* ft_used;            // [cap_ft][kMaxRows] sorted clusters, outermost first
  // a11 outputs
  int* ft_outidx;          // compaction index of accepted fit tracks
  float* out_par;
  float* out_cov;
  float* out_chi2;
  float* out_x;
  float* out_zsh;          // [cap_ft] z shift of the far side (central-electrode merging)
  int* out_ndf;
  int* out_sector;
  int* out_ncl;
  int* out_offset;
  int* out_ids;            // [cap_refs] input ids
  long cap_refs;
  int* out_key;
  int* attach;             // [n] input id space
  int* attach_key;         // [n] input id space
  MapDev map;              // correction map of this call
  LaunchCfg lc;            // launch shapes of the heavy kernels
};

constexpr int kCkptStride = 16;                        // stations per checkpoint segment
constexpr int kCkptSeg = (kMaxRows + kCkptStride - 1) / kCkptStride;
constexpr int kCkptF = 27;                             // p[5], c[15], ref[5], x, sector

// Refit of given tracks (fixed clusters) and its adjoint.
struct RefitDev {
  long n_tracks;
  long cap;                // track capacity
  long cap_refs;
  // inputs (device, caller-owned)
  const float* y;
  const float* z;
  const uint8_t* row;
  const uint8_t* sector;
  const int* offset;       // [n_tracks + 1]
  const int* ids;          // innermost first
  const float* in_par;     // [n_tracks][5]
  const float* in_x;
  const int* in_sector;
  const float* in_zsh;     // [n_tracks] z shift of the far side (central electrode), or NULL
  const float* row_x;
  int freeze;
  // state kept for freezing and for the adjoint
  float* ref;              // [cap][10]
  uint8_t* flag;           // [cap_refs]
  float* zref;             // [cap_refs] cluster z in the frame of the track's innermost side
  uint8_t* acc;            // [cap_refs]
  float* z0;               // [cap]
  float* ckpt;             // [cap][3][kCkptSeg][kCkptF]
  float* store;            // [cap][kMaxRows][5] iteration-1 predictions
  int* ok;
  int* nused;
  float* chi2;
  float* out;              // [cap][kStateF]
  int* ndf;
  int* out_sector;
  float* out_par;          // [cap][5]
  float* out_cov;          // [cap][15]
  float* out_x;
  // adjoint
  const float* dl_dchi2;   // [n_tracks]
  float* dD;               // [cap_refs][3]
  double* gpart;           // [blocks][ncoef]
  float* dl_dmap;          // [ncoef]
  int ncoef;
  int gblocks;
  MapDev map;
};

}  // namespace tpc
