// C ABI of the tracker: context, device buffers, stage orchestration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "tpc.h"
#include "tpc_internal.h"
#include "tpc_kernels.h"

using namespace tpc;

namespace {
using StageFn = int (*)(FrameDev&, const KParams&, int, cudaStream_t);
struct StageDef {
  const char* name;
  StageFn strict_fn;
  StageFn fast_fn;
};
// Hot-path stages in execution order.
const StageDef kStages[] = {
    {"grid", strict::stage_grid, fast::stage_grid},
    {"links", strict::stage_links, fast::stage_links},
    {"starts", strict::stage_starts, fast::stage_starts},
    {"tracklets", strict::stage_tracklets, fast::stage_tracklets},
    {"select", strict::stage_select, fast::stage_select},
    {"reseed", strict::stage_reseed, fast::stage_reseed},
    {"sector_refit", strict::stage_sector_refit, fast::stage_sector_refit},
    {"edge", strict::stage_edge, fast::stage_edge},
    {"merge", strict::stage_merge, fast::stage_merge},
    {"fit12", strict::stage_fit12, fast::stage_fit12},
    {"ambiguity2", strict::stage_ambiguity2, fast::stage_ambiguity2},
    {"fit3", strict::stage_fit3, fast::stage_fit3},
    {"output", strict::stage_output, fast::stage_output},
};
constexpr int kNumStages = sizeof(kStages) / sizeof(kStages[0]);
}  // namespace

// Identity of a captured chain: same buffers, sizes, map and launch shapes.
struct GraphKey {
  const void* y;
  const void* z;
  const void* row;
  const void* sector;
  long n;
  long nf;
  const void* map;
  long lc_version;
  GraphKey() { std::memset(this, 0, sizeof *this); }
  GraphKey(const void* a, const void* b, const void* c, const void* d, long n_, int nf_,
           const void* m, long v) {
    std::memset(this, 0, sizeof *this);
    y = a; z = b; row = c; sector = d; n = n_; nf = nf_; map = m; lc_version = v;
  }
};

struct tpc_ctx {
  tpc_options opt{};
  int max_frames = 1;
  // batch input: the frame table (the frames are read in place)
  FrameSrc* src = nullptr;
  // graph replay
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  GraphKey graph_key;
  long graph_launches = 0;
  long lc_version = 0;
  bool prof = false;
  cudaEvent_t ev[kNumStages + 1] = {};
  double stage_ms[kNumStages] = {};
  long stage_calls[kNumStages] = {};
  long stage_launches[kNumStages] = {};
  long launches_last = 0;
  KParams P{};
  int sms = 0;
  int n_rows = 0, n_sectors = 0;
  long cap_n = 0;
  std::vector<void*> allocs;
  FrameDev F{};
  tpc_map map{};
  Counters host_cnt{};
  cudaStream_t last_stream = nullptr;
  // refit and adjoint
  RefitDev R{};
  bool refit_alloc = false;
  bool refit_done = false;
  int64_t refit_gen = 0;  // successful tpc_refit calls so far
  bool tracked = false;  // the last tracking call succeeded (its tracks are resident)
  int last_nf = 1;       // frames of that call
  long refit_tracks = -1, refit_refs = -1;
  int* steps3 = nullptr;
  long gpart_cap = 0;
  std::string err = "ok";
};

namespace {

tpc_status fail(tpc_ctx* c, tpc_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return st;
}

template <typename T>
bool dalloc(tpc_ctx* c, T** p, long count) {
  void* v = nullptr;
  const size_t bytes = (size_t)(count > 0 ? count : 1) * sizeof(T);
  if (cudaMalloc(&v, bytes) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  c->allocs.push_back(v);
  *p = (T*)v;
  return true;
}

}  // namespace

namespace tpc {
// Derived constants: computed in double from the physical inputs, rounded once.
void derive(KParams& P, const tpc_options& o, float bz, const std::vector<float>& row_x) {
  const double pi = 3.14159265358979323846;
  P.kb = (float)(-(double)bz * 0.00299792458);
  P.tan_half = (float)std::tan(10.0 * pi / 180.0);
  P.rot_c = (float)std::cos(20.0 * pi / 180.0);
  P.rot_s = (float)std::sin(20.0 * pi / 180.0);
  P.sy2 = (float)((double)o.sigma_y * (double)o.sigma_y);
  P.sz2 = (float)((double)o.sigma_z * (double)o.sigma_z);
  P.ms2 = (float)((double)o.ms_theta * (double)o.ms_theta);
  const int nr = (int)row_x.size();
  P.pitch_inv = (float)((double)(nr - 1) / ((double)row_x[nr - 1] - (double)row_x[0]));
  P.link_wy = o.link_wy;
  P.link_wz = o.link_wz;
  P.link_chi2 = o.link_chi2;
  for (int i = 0; i < 5; ++i) P.seed_c[i] = o.seed_c[i];
  P.follow_chi2 = o.follow_chi2;
  P.max_snp = o.max_snp;
  P.fit_max_snp = o.fit_max_snp;
  P.score_w = o.score_w;
  P.shared_frac = o.shared_frac;
  P.merge_chi2 = o.merge_chi2;
  P.merge_dy = o.merge_dy;
  P.merge_dz = o.merge_dz;
  P.int_chi2 = o.int_chi2;
  P.final_chi2 = o.final_chi2;
  P.attach_margin = o.attach_margin;
  P.edge_margin = o.edge_margin;
  P.looper_qpt = o.looper_qpt;
  P.ext_chi2 = o.ext_chi2;
  P.ext_rows = o.ext_rows;
  P.seed_iters = o.seed_iters > 1 ? o.seed_iters : 1;
  P.ac_merge = o.ac_merge ? 1 : 0;
  P.edge_rows = o.edge_rows;
  P.edge_min = o.edge_min;
  // z reach of a merge pair: (max gap + 2) rows at the steepest allowed angle
  P.merge_zspan = (float)((double)(o.merge_max_gap + 2) *
                          (((double)row_x[nr - 1] - (double)row_x[0]) / (double)(nr - 1)) /
                          std::sqrt(1.0 - (double)o.max_snp * (double)o.max_snp));
  P.max_miss = o.max_miss;
  P.min_hits = o.min_hits;
  P.merge_max_gap = o.merge_max_gap;
  P.inner_rows = o.inner_rows;
  P.cand_k = o.cand_k;
  P.grid_dy = 2.0f;
  P.grid_occ = 0.5f;
}
}  // namespace tpc

namespace {

// Kernel view of a correction map; scales derived in double, rounded once.
MapDev make_mapdev(const tpc_map& m) {
  MapDev M{};
  if (!m.coeff) return M;
  M.on = 1;
  M.nphi = m.n_phi;
  M.nr = m.n_r;
  M.nz = m.n_z;
  M.rmin = m.r_min;
  M.zmin = m.z_min;
  M.zmax = m.z_max;
  M.phi_scale = (float)((double)m.n_phi / 18.0);
  M.r_scale = (float)((double)(m.n_r - 3) / ((double)m.r_max - (double)m.r_min));
  M.z_scale = (float)((double)(m.n_z - 3) / ((double)m.z_max - (double)m.z_min));
  M.c = m.coeff;
  return M;
}

#define CK(call)                                                                     \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(ctx, TPC_ERR_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

}  // namespace

extern "C" {

tpc_status tpc_init(const tpc_geometry* geo, float bz_tesla, const tpc_map* map,
                    const tpc_options* opt, tpc_ctx** out) {
  if (!geo || !opt || !out || !geo->row_x) return TPC_ERR_INVALID_ARG;
  *out = nullptr;
  if (geo->n_rows < 4 || geo->n_rows > kMaxRows || geo->n_sectors < 1 || geo->n_sectors > 255 ||
      geo->n_sectors * geo->n_rows > 65535 || opt->cap_clusters < 1 || opt->cand_k < 1 ||
      opt->cand_k > kMaxCand || opt->min_hits < 3 || !(opt->shared_frac >= 0.0f) ||
      (opt->mode != 0 && opt->mode != 1) || opt->cap_clusters > (1L << 30) ||
      opt->inner_rows < 0 || opt->inner_rows > kMaxInner || opt->merge_max_gap < 1 ||
      opt->ext_rows < 0 || opt->ext_rows > kMaxExt || !(opt->ext_chi2 > 0.0f) ||
      opt->seed_iters < 0 || opt->seed_iters > kMaxSeedIters ||
      opt->edge_rows < 0 || opt->edge_rows > kMaxRows ||
      (opt->edge_rows > 0 && (opt->edge_min < 1 || opt->cap_clusters > (1L << 29))) ||
      opt->max_frames < 0 || opt->max_frames > 64 ||
      (long)geo->n_sectors * (opt->max_frames > 1 ? opt->max_frames : 1) * geo->n_rows > 65535 ||
      !(opt->fit_max_snp > 0.0f && opt->fit_max_snp < 1.0f) ||
      !(opt->max_snp > 0.0f && opt->max_snp < 1.0f))
    return TPC_ERR_INVALID_ARG;
  if (map && map->coeff &&
      (map->n_phi < 1 || map->n_r < 4 || map->n_z < 4 || !(map->r_max > map->r_min) ||
       !(map->z_max > map->z_min)))
    return TPC_ERR_INVALID_ARG;
  for (int r = 1; r < geo->n_rows; ++r)
    if (!(geo->row_x[r] > geo->row_x[r - 1])) return TPC_ERR_INVALID_ARG;
  tpc_ctx* ctx = new (std::nothrow) tpc_ctx();
  if (!ctx) return TPC_ERR_OOM;
  ctx->opt = *opt;
  ctx->n_rows = geo->n_rows;
  ctx->n_sectors = geo->n_sectors;
  std::vector<float> rx(geo->row_x, geo->row_x + geo->n_rows);
  derive(ctx->P, *opt, bz_tesla, rx);
  ctx->max_frames = opt->max_frames > 1 ? opt->max_frames : 1;
  ctx->P.n_rows = geo->n_rows;
  ctx->P.n_sectors = geo->n_sectors * ctx->max_frames;
  ctx->P.n_phi = geo->n_sectors / 2 > 0 ? geo->n_sectors / 2 : 1;
  if (map) ctx->map = *map;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
  if (ctx->sms <= 0) ctx->sms = 1;
  strict::init_attributes();
  fast::init_attributes();

  const long n = opt->cap_clusters;
  ctx->cap_n = n;
  const long nsec_all = (long)geo->n_sectors * ctx->max_frames;
  const long nrr = nsec_all * geo->n_rows;
  FrameDev& F = ctx->F;
  for (int i = 0; i < kLNum; ++i) {
    F.lc.block[i] = 128;
    F.lc.per_sm[i] = 8;
    F.lc.lanes[i] = 1;
  }
  F.lc.lanes[kLMerge] = kMergeLanesDefault;
  F.lc.lanes[kLLinks] = kLinksLanesDefault;
  F.cap_bins = (long)((double)n / ctx->P.grid_occ) + nrr * 65;
  F.cap_tl = opt->cap_tracklets > 0 ? opt->cap_tracklets : n / 10 + 4096;
  bool ok = true;
  ok &= dalloc(ctx, (float**)&F.row_x, geo->n_rows);
  ok &= dalloc(ctx, &F.row_cnt, nrr);
  ok &= dalloc(ctx, &F.row_zmin, nrr);
  ok &= dalloc(ctx, &F.row_zmax, nrr);
  ok &= dalloc(ctx, &F.rows, nrr);
  ok &= dalloc(ctx, &F.row_first, nrr + 1);
  ok &= dalloc(ctx, &F.bin_cnt, F.cap_bins + 1);
  ok &= dalloc(ctx, &F.bin_first, F.cap_bins + 1);
  ok &= dalloc(ctx, &F.cl_bin, n);
  ok &= dalloc(ctx, &F.cl_slot, n);
  ok &= dalloc(ctx, &F.srec, n);
  ok &= dalloc(ctx, &F.syz, n);
  ok &= dalloc(ctx, &F.sid, n);
  ok &= dalloc(ctx, &F.srow, n);
  ok &= dalloc(ctx, &F.lup, n);
  ok &= dalloc(ctx, &F.ldn, n);
  ok &= dalloc(ctx, &F.cup, n);
  ok &= dalloc(ctx, &F.cdn, n);
  ok &= dalloc(ctx, &F.flags, n);
  ok &= dalloc(ctx, &F.scan_tmp, (F.cap_bins + n) / 256 + 4096);
  ok &= dalloc(ctx, &F.starts, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_par, F.cap_tl * 5);
  ok &= dalloc(ctx, &F.tl_cov, F.cap_tl * 15);
  ok &= dalloc(ctx, &F.tl_x, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_chi2, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_key, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_n, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_rlo, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_len, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_seed, F.cap_tl * kSeedF);
  ok &= dalloc(ctx, &F.tl_rhi, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_hits, F.cap_tl * kMaxRows);
  ok &= dalloc(ctx, &F.owner_key, n);
  ok &= dalloc(ctx, &F.tl_acc, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_nkept, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_kept, F.cap_tl * kMaxRows);
  ok &= dalloc(ctx, &F.sec_owner, n);
  ok &= dalloc(ctx, &F.sused, n);
  ok &= dalloc(ctx, &F.cr_flags, n);
  ok &= dalloc(ctx, &F.cr_out, n);
  ok &= dalloc(ctx, &F.cr_bin_cnt, kCrBins + 1);
  ok &= dalloc(ctx, &F.cr_bin_first, kCrBins + 1);
  ok &= dalloc(ctx, &F.cnt, 1);
  // a7
  const long T = F.cap_tl;
  const long nmb = nrr * kMergeZ;
  ok &= dalloc(ctx, &F.st_tl, T);
  ok &= dalloc(ctx, &F.st_off, T);
  F.cap_pos = n + n / 4 + 4096;
  ok &= dalloc(ctx, &F.st_pos, F.cap_pos);
  ok &= dalloc(ctx, &F.st_order, T);
  ok &= dalloc(ctx, &F.st_obucket, T);
  ok &= dalloc(ctx, &F.st_oslot, T);
  ok &= dalloc(ctx, &F.st_ord_cnt, kOrdBuckets);
  ok &= dalloc(ctx, &F.st_ok, T);
  ok &= dalloc(ctx, &F.st_key, T);
  ok &= dalloc(ctx, &F.st_sector, T);
  ok &= dalloc(ctx, &F.st_rmin, T);
  ok &= dalloc(ctx, &F.st_rmax, T);
  ok &= dalloc(ctx, &F.st_ie, T * kStateF);
  ok &= dalloc(ctx, &F.st_oe, T * kStateF);
  ok &= dalloc(ctx, &F.st_next, T);
  ok &= dalloc(ctx, &F.st_hasprev, T);
  ok &= dalloc(ctx, &F.st_bestB, T);
  ok &= dalloc(ctx, &F.st_bestchi, T);
  ok &= dalloc(ctx, &F.st_bestA, T);
  ok &= dalloc(ctx, &F.st_xbestB, T);
  ok &= dalloc(ctx, &F.st_xchi, T);
  ok &= dalloc(ctx, &F.st_xdz, T);
  ok &= dalloc(ctx, &F.st_xbestA, T);
  ok &= dalloc(ctx, &F.st_dz, T);
  ok &= dalloc(ctx, &F.ie_cnt, nmb + 1);
  ok &= dalloc(ctx, &F.ie_first, nmb + 1);
  ok &= dalloc(ctx, &F.ie_slot, T);
  ok &= dalloc(ctx, &F.ie_bin, T);
  ok &= dalloc(ctx, &F.ie_idx, T);
  ok &= dalloc(ctx, &F.ie_rec, T);
  ok &= dalloc(ctx, &F.sec_zlo, nsec_all);
  ok &= dalloc(ctx, &F.sec_zinv, nsec_all);
  if (ctx->max_frames > 1) ok &= dalloc(ctx, &ctx->src, ctx->max_frames);
  if (opt->edge_rows > 0) {
    ok &= dalloc(ctx, &F.st_kept, n);
    ok &= dalloc(ctx, &F.edge_flag, 2 * F.cap_tl + 1);
    ok &= dalloc(ctx, &F.edge_pos, 2 * F.cap_tl + 1);
  }
  if (opt->use_graphs) {
    ok &= cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&ctx->ev_in, cudaEventDisableTiming) == cudaSuccess;
    ok &= cudaEventCreateWithFlags(&ctx->ev_out, cudaEventDisableTiming) == cudaSuccess;
  }
  // a9/a10/a11
  F.cap_ft = opt->cap_tracks > 0 ? opt->cap_tracks : n / 40 + 4096;
  const long FT = F.cap_ft;
  ok &= dalloc(ctx, &F.ft_head, FT);
  ok &= dalloc(ctx, &F.ft_last, FT);
  ok &= dalloc(ctx, &F.ft_order, FT);
  ok &= dalloc(ctx, &F.ft_looper, FT);
  ok &= dalloc(ctx, &F.ft_key, FT);
  ok &= dalloc(ctx, &F.ft_ok, FT);
  ok &= dalloc(ctx, &F.ft_nst, FT);
  ok &= dalloc(ctx, &F.ft_z0, FT);
  ok &= dalloc(ctx, &F.ft_st_cl, FT * kMaxRows);
  ok &= dalloc(ctx, &F.ft_st_rs, FT * kMaxRows);
  ok &= dalloc(ctx, &F.ft_store, FT * kMaxRows * 5);
  ok &= dalloc(ctx, &F.ft_flag, FT * kMaxRows);
  ok &= dalloc(ctx, &F.ft_end2, FT * kStateF);
  F.nslot = kMaxInner + 2 * opt->ext_rows;
  const long NS = F.nslot;
  ok &= dalloc(ctx, &F.ft_ncand, FT * NS);
  ok &= dalloc(ctx, &F.ft_cand, FT * NS * kMaxCand);
  ok &= dalloc(ctx, &F.ft_cchi, FT * NS * kMaxCand);
  ok &= dalloc(ctx, &F.ft_assigned, FT * NS);
  ok &= dalloc(ctx, &F.ft_newly, FT * NS);
  ok &= dalloc(ctx, &F.ft_next, FT);
  ok &= dalloc(ctx, &F.ft_nout, FT);
  ok &= dalloc(ctx, &F.ft_ext_sec, FT * (opt->ext_rows > 0 ? 2 * opt->ext_rows : 1));
  ok &= dalloc(ctx, &F.ft_ipol, FT * kMaxInner * kIpolF);
  ok &= dalloc(ctx, &F.ft_fixed, n);
  ok &= dalloc(ctx, &F.bid, n);
  ok &= dalloc(ctx, &F.taken, n);
  ok &= dalloc(ctx, &F.ft_n, FT);
  ok &= dalloc(ctx, &F.ft_chi2, FT);
  ok &= dalloc(ctx, &F.ft_out, FT * kStateF);
  ok &= dalloc(ctx, &F.ft_used, FT * kMaxRows);
  ok &= dalloc(ctx, &F.ft_outidx, FT);
  ok &= dalloc(ctx, &F.cr_cls, FT);
  ok &= dalloc(ctx, &F.ft_side0, FT);
  ok &= dalloc(ctx, &F.ft_zsh, FT);
  ok &= dalloc(ctx, &F.cr_parent, FT);
  ok &= dalloc(ctx, &F.cr_cx, FT);
  ok &= dalloc(ctx, &F.cr_cy, FT);
  ok &= dalloc(ctx, &F.cr_zk, FT);
  ok &= dalloc(ctx, &F.cr_bin_items, FT);
  ok &= dalloc(ctx, &F.out_par, FT * 5);
  ok &= dalloc(ctx, &F.out_cov, FT * 15);
  ok &= dalloc(ctx, &F.out_chi2, FT);
  ok &= dalloc(ctx, &F.out_x, FT);
  ok &= dalloc(ctx, &F.out_zsh, FT);
  ok &= dalloc(ctx, &F.out_ndf, FT);
  ok &= dalloc(ctx, &F.out_sector, FT);
  ok &= dalloc(ctx, &F.out_ncl, FT);
  ok &= dalloc(ctx, &F.out_offset, FT + 1);
  F.cap_refs = n + n / 4 + 4096;
  ok &= dalloc(ctx, &F.out_ids, F.cap_refs);
  ok &= dalloc(ctx, &F.out_key, FT);
  ok &= dalloc(ctx, &F.attach, n);
  ok &= dalloc(ctx, &F.attach_key, n);
  if (!ok) {
    tpc_destroy(ctx);
    return TPC_ERR_OOM;
  }
  if (cudaMemcpy((void*)F.row_x, geo->row_x, sizeof(float) * geo->n_rows,
                 cudaMemcpyHostToDevice) != cudaSuccess) {
    tpc_destroy(ctx);
    return TPC_ERR_CUDA;
  }
  *out = ctx;
  return TPC_OK;
}

tpc_status tpc_set_map(tpc_ctx* ctx, const tpc_map* map) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (map) {
    if (map->coeff && (map->n_phi < 1 || map->n_r < 4 || map->n_z < 4 || !(map->r_max > map->r_min) ||
                       !(map->z_max > map->z_min)))
      return fail(ctx, TPC_ERR_INVALID_ARG, "invalid map shape");
    ctx->map = *map;
  } else {
    ctx->map = tpc_map{};
  }
  ++ctx->lc_version;  // captured graphs hold the map by value: recapture
  return TPC_OK;
}

}  // extern "C"

namespace {

// Enqueue the whole chain (buffer resets and all stages) for F with the
// per-call parameters Pc; returns the number of kernels.  No host sync.
tpc_status enqueue_chain(tpc_ctx* ctx, FrameDev& F, const KParams& Pc, cudaStream_t s,
                         bool events, long* launches) {
  const long nrr = (long)Pc.n_sectors * ctx->n_rows;
  const long n = F.n;
  CK(cudaMemsetAsync(F.cnt, 0, sizeof(Counters), s));
  CK(cudaMemsetAsync(F.row_cnt, 0, sizeof(int) * nrr, s));
  CK(cudaMemsetAsync(F.row_zmin, 0xFF, sizeof(unsigned) * nrr, s));
  CK(cudaMemsetAsync(F.row_zmax, 0, sizeof(unsigned) * nrr, s));
  CK(cudaMemsetAsync(F.bin_cnt, 0, sizeof(int) * (F.cap_bins + 1), s));
  if (n > 0) {
    CK(cudaMemsetAsync(F.owner_key, 0, sizeof(unsigned long long) * n, s));
    CK(cudaMemsetAsync(F.sec_owner, 0xFF, sizeof(int) * n, s));
    CK(cudaMemsetAsync(F.bid, 0xFF, sizeof(unsigned long long) * n, s));
    CK(cudaMemsetAsync(F.taken, 0, n, s));
    CK(cudaMemsetAsync(F.attach, 0xFF, sizeof(int) * n, s));
    CK(cudaMemsetAsync(F.attach_key, 0x7F, sizeof(int) * n, s));
    if (Pc.ext_rows > 0) CK(cudaMemsetAsync(F.ft_fixed, 0, n, s));
    if (Pc.seed_iters > 1) CK(cudaMemsetAsync(F.sused, 0, n, s));
  }
  CK(cudaMemsetAsync(F.ie_cnt, 0, sizeof(int) * (nrr * kMergeZ + 1), s));
  CK(cudaMemsetAsync(F.st_ord_cnt, 0, sizeof(int) * kOrdBuckets, s));
  CK(cudaMemsetAsync(F.out_offset, 0, sizeof(int), s));
  long k = 0;
  if (events) CK(cudaEventRecord(ctx->ev[0], s));
  for (int i = 0; i < kNumStages; ++i) {
    const StageFn fn = ctx->opt.mode == 0 ? kStages[i].strict_fn : kStages[i].fast_fn;
    const int ki = fn(F, Pc, ctx->sms, s);
    k += ki;
    ctx->stage_launches[i] += ki;
    if (events) CK(cudaEventRecord(ctx->ev[i + 1], s));
  }
  CK(cudaGetLastError());
  *launches = k;
  return TPC_OK;
}

// Runs the chain on the frame view F (single frame or concatenated batch of
// nf frames), through a cached CUDA graph unless profiling, then reads the
// counters back and fills `out`.
tpc_status run_chain(tpc_ctx* ctx, FrameDev& F, int nf, cudaStream_t s, tpc_tracks* out,
                     int64_t* needed) {
  KParams Pc = ctx->P;
  Pc.n_sectors = ctx->n_sectors * nf;
  F.map = make_mapdev(ctx->map);
  ctx->tracked = false;
  ctx->last_nf = nf;
  ctx->last_stream = s;
  long launches = 0;
  const bool graph = ctx->opt.use_graphs && !ctx->prof;
  if (graph) {
    // a batch reads its frames through the frame table, copied before every
    // launch: its graph does not depend on where the frames lie
    GraphKey key{F.y, F.z, F.row, F.nsrc ? (const void*)F.src : (const void*)F.sector, F.n,
                 nf, F.map.c, ctx->lc_version};
    if (!ctx->graph_exec || std::memcmp(&key, &ctx->graph_key, sizeof key) != 0) {
      if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
      ctx->graph_exec = nullptr;
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeThreadLocal));
      const tpc_status st = enqueue_chain(ctx, F, Pc, ctx->gstream, false, &launches);
      const cudaError_t e = cudaStreamEndCapture(ctx->gstream, &g);
      if (st != TPC_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return fail(ctx, TPC_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e));
      CK(cudaGraphInstantiate(&ctx->graph_exec, g, 0));
      cudaGraphDestroy(g);
      ctx->graph_key = key;
      ctx->graph_launches = launches;
    }
    launches = ctx->graph_launches;
    // order the graph after the caller's stream, and the caller after it
    CK(cudaEventRecord(ctx->ev_in, s));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->ev_in, 0));
    CK(cudaGraphLaunch(ctx->graph_exec, ctx->gstream));
    CK(cudaMemcpyAsync(&ctx->host_cnt, F.cnt, sizeof(Counters), cudaMemcpyDeviceToHost,
                       ctx->gstream));
    CK(cudaEventRecord(ctx->ev_out, ctx->gstream));
    CK(cudaStreamWaitEvent(s, ctx->ev_out, 0));
    CK(cudaStreamSynchronize(ctx->gstream));
  } else {
    const tpc_status st = enqueue_chain(ctx, F, Pc, s, ctx->prof, &launches);
    if (st != TPC_OK) return st;
    CK(cudaMemcpyAsync(&ctx->host_cnt, F.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (ctx->prof) {
      for (int i = 0; i < kNumStages; ++i) {
        float ms = 0.0f;
        CK(cudaEventElapsedTime(&ms, ctx->ev[i], ctx->ev[i + 1]));
        ctx->stage_ms[i] += ms;
        ctx->stage_calls[i] += 1;
      }
    }
  }
  ctx->launches_last = launches;
  const Counters& c = ctx->host_cnt;
  std::memset(out, 0, sizeof(*out));
  if (c.err & kErrInput) return fail(ctx, TPC_ERR_INVALID_INPUT, "invalid cluster (NaN/Inf, row or sector out of range)");
  if (c.err & kErrDense)
    return fail(ctx, TPC_ERR_INVALID_INPUT, "more than %d clusters in one search bin", kMaxBinOcc);
  if (c.err & kErrCapBins) {
    if (needed) *needed = c.n_bins;
    return fail(ctx, TPC_ERR_CAPACITY, "grid bins %d exceed capacity %ld", c.n_bins, F.cap_bins);
  }
  if (c.err & kErrCapTracklets) {
    if (needed) *needed = c.need_tracklets;
    return fail(ctx, TPC_ERR_CAPACITY, "start hits %d exceed tracklet capacity %ld", c.n_starts,
                F.cap_tl);
  }
  if (c.err & kErrCapEdge) {
    if (needed) *needed = c.need_tracklets;
    return fail(ctx, TPC_ERR_CAPACITY, "sector tracks / tracklets with the edge-following "
                "segments (%d) exceed tracklet capacity %ld", c.need_tracklets, F.cap_tl);
  }
  if (c.err & kErrCapRefs) {
    if (needed) *needed = c.n_refs;
    return fail(ctx, TPC_ERR_CAPACITY, "cluster references %d exceed capacity %ld", c.n_refs,
                F.cap_refs);
  }
  if (c.err & kErrCapPos) {
    if (needed) *needed = c.n_pos;
    return fail(ctx, TPC_ERR_CAPACITY, "kept sector-track clusters %d exceed capacity %ld",
                c.n_pos, F.cap_pos);
  }
  if (c.err & kErrCapTracks) {
    if (needed) *needed = c.need_tracks;
    return fail(ctx, TPC_ERR_CAPACITY, "merged tracks %d exceed track capacity %ld", c.n_merged,
                F.cap_ft);
  }
  out->n_tracks = c.n_out;
  out->n_cluster_refs = c.n_refs;
  out->params = F.out_par;
  out->cov = F.out_cov;
  out->chi2 = F.out_chi2;
  out->x = F.out_x;
  out->ndf = F.out_ndf;
  out->sector = F.out_sector;
  out->n_clusters = F.out_ncl;
  out->cl_offset = F.out_offset;
  out->cl_ids = F.out_ids;
  out->key = F.out_key;
  out->attach = F.attach;
  out->z_shift = F.out_zsh;
  ctx->tracked = true;
  return TPC_OK;
}

}  // namespace

extern "C" {

tpc_status tpc_track_timeframe(tpc_ctx* ctx, const tpc_clusters* cl, tpc_tracks* out,
                               void* cuda_stream, int64_t* needed) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (!cl || !out) return fail(ctx, TPC_ERR_INVALID_ARG, "null clusters or output");
  if (cl->n < 0) return fail(ctx, TPC_ERR_INVALID_ARG, "negative cluster count");
  if (cl->n > 0 && (!cl->y || !cl->z || !cl->row || !cl->sector))
    return fail(ctx, TPC_ERR_INVALID_ARG, "null cluster array");
  if (cl->n > ctx->cap_n) {
    if (needed) *needed = cl->n;
    return fail(ctx, TPC_ERR_CAPACITY, "frame has %lld clusters, capacity %ld", (long long)cl->n,
                ctx->cap_n);
  }
  FrameDev& F = ctx->F;
  F.y = cl->y;
  F.z = cl->z;
  F.row = cl->row;
  F.sector = cl->sector;
  F.src = nullptr;
  F.nsrc = 0;
  F.n = cl->n;
  return run_chain(ctx, F, 1, (cudaStream_t)cuda_stream, out, needed);
}

tpc_status tpc_track_batch(tpc_ctx* ctx, const tpc_clusters* frames, int32_t n_frames,
                           tpc_tracks* out, void* cuda_stream, int64_t* needed) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (!frames || !out || n_frames < 1)
    return fail(ctx, TPC_ERR_INVALID_ARG, "null frames/output or no frame");
  if (n_frames > ctx->max_frames)
    return fail(ctx, TPC_ERR_INVALID_ARG, "%d frames exceed the context's max_frames %d", n_frames,
                ctx->max_frames);
  // one frame: batch sectors equal the frame's own, no concatenation needed
  if (n_frames == 1) return tpc_track_timeframe(ctx, frames, out, cuda_stream, needed);
  long total = 0;
  for (int f = 0; f < n_frames; ++f) {
    if (frames[f].n < 0 || (frames[f].n > 0 && (!frames[f].y || !frames[f].z || !frames[f].row ||
                                                 !frames[f].sector)))
      return fail(ctx, TPC_ERR_INVALID_ARG, "invalid frame %d", f);
    total += frames[f].n;
  }
  if (total > ctx->cap_n) {
    if (needed) *needed = total;
    return fail(ctx, TPC_ERR_CAPACITY, "batch has %ld clusters, capacity %ld", total, ctx->cap_n);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  FrameDev& F = ctx->F;
  // frame table: batch cluster off_f + j is frame f's cluster j, and frame
  // f's sector s becomes batch sector f * n_sectors + s
  std::vector<FrameSrc> tab((size_t)n_frames);
  long off = 0;
  for (int f = 0; f < n_frames; ++f) {
    tab[f] = FrameSrc{frames[f].y, frames[f].z, frames[f].row, frames[f].sector, off};
    off += frames[f].n;
  }
  CK(cudaMemcpyAsync(ctx->src, tab.data(), sizeof(FrameSrc) * n_frames, cudaMemcpyHostToDevice,
                     s));
  F.y = nullptr;
  F.z = nullptr;
  F.row = nullptr;
  F.sector = nullptr;
  F.src = ctx->src;
  F.nsrc = n_frames;
  F.src_nsec = ctx->n_sectors;
  F.n = total;
  return run_chain(ctx, F, n_frames, s, out, needed);
}

tpc_status tpc_autotune(tpc_ctx* ctx, const tpc_clusters* frames, int32_t n_frames,
                        void* cuda_stream) {
  if (!ctx || !frames || n_frames < 1) return TPC_ERR_INVALID_ARG;
  static const char* slot_stage[kLNum] = {"tracklets", "sector_refit", "merge", "fit12", "fit3",
                                          "links"};
  static const int blocks[] = {64, 128, 256};
  static const int per_sm[] = {4, 8, 16};
  static const int merge_lanes[] = {1, 8, 16, 32};
  static const int links_lanes[] = {1, 4, 8, 32};
  const bool prof_was = ctx->prof;
  if (!ctx->ev[0])
    for (auto& e : ctx->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail(ctx, TPC_ERR_CUDA, "event create");
  ctx->prof = true;
  tpc_tracks out;
  int64_t need = 0;
  for (int slot = 0; slot < kLNum; ++slot) {
    int st = 0;
    while (st < kNumStages && std::strcmp(kStages[st].name, slot_stage[slot]) != 0) ++st;
    double best = 1e30;
    LaunchCfg best_lc = ctx->F.lc;
    // the neighbour search is one launch over the clusters: only its lanes vary
    const int nl = slot == kLMerge ? 4 : slot == kLLinks ? 4 : 1;
    const int nb = slot == kLLinks ? 1 : 3, nq = slot == kLLinks ? 1 : 3;
    for (int li = 0; li < nl; ++li)
    for (int bi = 0; bi < nb; ++bi)
      for (int qi = 0; qi < nq; ++qi) {
        ctx->F.lc.block[slot] = slot == kLLinks ? 256 : blocks[bi];
        ctx->F.lc.per_sm[slot] = slot == kLLinks ? 8 : per_sm[qi];
        ctx->F.lc.lanes[slot] = slot == kLMerge ? merge_lanes[li]
                                : slot == kLLinks ? links_lanes[li] : 1;
        double t = 0.0;
        for (int rep = 0; rep < 2; ++rep) {
          const double before = ctx->stage_ms[st];
          const tpc_status rc = tpc_track_batch(ctx, frames, n_frames, &out, cuda_stream, &need);
          if (rc != TPC_OK) {
            ctx->prof = prof_was;
            return rc;
          }
          if (rep == 1) t = ctx->stage_ms[st] - before;  // second run: warm
        }
        if (t < best) {
          best = t;
          best_lc = ctx->F.lc;
        }
      }
    ctx->F.lc = best_lc;
  }
  ctx->prof = prof_was;
  ++ctx->lc_version;
  for (int i = 0; i < kNumStages; ++i) {
    ctx->stage_ms[i] = 0.0;
    ctx->stage_calls[i] = 0;
    ctx->stage_launches[i] = 0;
  }
  return TPC_OK;
}

tpc_status tpc_launch_config(const tpc_ctx* ctx, int32_t slot, const char** kernel,
                             int32_t* block, int32_t* blocks_per_sm, int32_t* lanes) {
  static const char* names[kLNum] = {"k_tl_chain+k_tl_up+k_tl_refit+k_tl_down",
                                     "k_sector_refit", "k_merge_best", "k_fit1+k_fit2", "k_fit3",
                                     "k_links"};
  if (!ctx || slot < 0 || slot >= kLNum) return TPC_ERR_INVALID_ARG;
  if (kernel) *kernel = names[slot];
  if (block) *block = ctx->F.lc.block[slot];
  if (blocks_per_sm) *blocks_per_sm = ctx->F.lc.per_sm[slot];
  if (lanes) *lanes = ctx->F.lc.lanes[slot];
  return TPC_OK;
}

tpc_status tpc_set_launch_config(tpc_ctx* ctx, int32_t slot, int32_t block,
                                 int32_t blocks_per_sm, int32_t lanes) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  const bool lanes_ok = lanes == 1 ||
                        (slot == kLMerge && (lanes == 4 || lanes == 8 || lanes == 16 || lanes == 32)) ||
                        (slot == kLLinks && (lanes == 4 || lanes == 8 || lanes == 32));
  if (slot < 0 || slot >= kLNum || block < 32 || block > 256 || block % 32 != 0 ||
      blocks_per_sm < 1 || blocks_per_sm > 32 || !lanes_ok)
    return fail(ctx, TPC_ERR_INVALID_ARG, "launch shape slot %d: block %d, %d per SM, %d lanes",
                slot, block, blocks_per_sm, lanes);
  ctx->F.lc.block[slot] = block;
  ctx->F.lc.per_sm[slot] = blocks_per_sm;
  ctx->F.lc.lanes[slot] = lanes;
  ++ctx->lc_version;
  return TPC_OK;
}

tpc_status tpc_refit(tpc_ctx* ctx, const tpc_clusters* cl, const tpc_tracks* in,
                     const tpc_map* map, int32_t freeze, tpc_tracks* out, void* cuda_stream) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (!cl || !in || !out || in->n_tracks < 0 || in->n_cluster_refs < 0)
    return fail(ctx, TPC_ERR_INVALID_ARG, "null or negative refit input");
  if (in->n_tracks > 0 && (!in->cl_offset || !in->cl_ids || !in->params || !in->x ||
                           !in->sector || !cl->y || !cl->z || !cl->row || !cl->sector))
    return fail(ctx, TPC_ERR_INVALID_ARG, "null refit array");
  const tpc_map& mp = map ? *map : ctx->map;
  if (mp.coeff && (mp.n_phi < 1 || mp.n_r < 4 || mp.n_z < 4 || !(mp.r_max > mp.r_min) ||
                   !(mp.z_max > mp.z_min)))
    return fail(ctx, TPC_ERR_INVALID_ARG, "invalid map shape");
  FrameDev& F = ctx->F;
  if (in->n_tracks > F.cap_ft || in->n_cluster_refs > F.cap_refs)
    return fail(ctx, TPC_ERR_CAPACITY, "refit of %lld tracks / %lld clusters exceeds capacity",
                (long long)in->n_tracks, (long long)in->n_cluster_refs);
  if (freeze && (!ctx->refit_done || ctx->refit_tracks != in->n_tracks ||
                 ctx->refit_refs != in->n_cluster_refs))
    return fail(ctx, TPC_ERR_STATE, "frozen refit needs a previous refit of the same tracks");
  RefitDev& R = ctx->R;
  if (!ctx->refit_alloc) {
    const long T = F.cap_ft, NR = F.cap_refs;
    bool ok = true;
    ok &= dalloc(ctx, &R.ref, T * 10);
    ok &= dalloc(ctx, &R.flag, NR);
    ok &= dalloc(ctx, &R.zref, NR);
    ok &= dalloc(ctx, &R.acc, NR);
    ok &= dalloc(ctx, &R.z0, T);
    ok &= dalloc(ctx, &R.ckpt, T * 3 * kCkptSeg * kCkptF);
    ok &= dalloc(ctx, &R.store, T * kMaxRows * 5);
    ok &= dalloc(ctx, &R.ok, T);
    ok &= dalloc(ctx, &R.nused, T);
    ok &= dalloc(ctx, &R.chi2, T);
    ok &= dalloc(ctx, &R.ndf, T);
    ok &= dalloc(ctx, &R.out_sector, T);
    ok &= dalloc(ctx, &R.out_par, T * 5);
    ok &= dalloc(ctx, &R.out_cov, T * 15);
    ok &= dalloc(ctx, &R.out_x, T);
    ok &= dalloc(ctx, &R.dD, NR * 3);
    ok &= dalloc(ctx, &ctx->steps3, T);
    if (!ok) return fail(ctx, TPC_ERR_OOM, "refit buffers");
    R.cap = T;
    R.cap_refs = NR;
    ctx->refit_alloc = true;
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ctx->last_stream = s;
  R.n_tracks = in->n_tracks;
  R.y = cl->y;
  R.z = cl->z;
  R.row = cl->row;
  R.sector = cl->sector;
  R.offset = in->cl_offset;
  R.ids = in->cl_ids;
  R.in_par = in->params;
  R.in_x = in->x;
  R.in_sector = in->sector;
  R.in_zsh = in->z_shift;
  R.row_x = F.row_x;
  R.freeze = freeze ? 1 : 0;
  R.map = make_mapdev(mp);
  const int k = ctx->opt.mode == 0 ? strict::refit_forward(R, ctx->P, ctx->steps3, ctx->sms, s)
                                   : fast::refit_forward(R, ctx->P, ctx->steps3, ctx->sms, s);
  ctx->launches_last = k;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  ctx->refit_done = true;
  ++ctx->refit_gen;
  ctx->refit_tracks = in->n_tracks;
  ctx->refit_refs = in->n_cluster_refs;
  std::memset(out, 0, sizeof(*out));
  out->n_tracks = in->n_tracks;
  out->n_cluster_refs = in->n_cluster_refs;
  out->params = R.out_par;
  out->cov = R.out_cov;
  out->chi2 = R.chi2;
  out->x = R.out_x;
  out->ndf = R.ndf;
  out->sector = R.out_sector;
  out->n_clusters = R.nused;
  out->cl_offset = in->cl_offset;
  out->cl_ids = in->cl_ids;
  out->key = in->key;
  out->attach = in->attach;
  out->z_shift = in->z_shift;
  return TPC_OK;
}

tpc_status tpc_refit_backward(tpc_ctx* ctx, const float* dl_dchi2, float* dl_dmap,
                              void* cuda_stream) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (!ctx->refit_done) return fail(ctx, TPC_ERR_STATE, "refit_backward needs a preceding refit");
  RefitDev& R = ctx->R;
  if (!R.map.on) return fail(ctx, TPC_ERR_STATE, "the preceding refit used no correction map");
  if (!dl_dmap || (R.n_tracks > 0 && !dl_dchi2))
    return fail(ctx, TPC_ERR_INVALID_ARG, "null gradient pointer");
  const long ncoef = 3L * R.map.nz * R.map.nr * R.map.nphi;
  int dev = 0, smem_max = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if ((long)sizeof(double) * ncoef > smem_max)
    return fail(ctx, TPC_ERR_INVALID_ARG, "map of %ld coefficients exceeds the FP64 block accumulator",
                ncoef);
  R.ncoef = (int)ncoef;
  R.gblocks = ctx->sms;
  if ((long)R.gblocks * ncoef > ctx->gpart_cap) {
    if (!dalloc(ctx, &R.gpart, (long)R.gblocks * ncoef)) return fail(ctx, TPC_ERR_OOM, "gradient partials");
    ctx->gpart_cap = (long)R.gblocks * ncoef;
  }
  R.dl_dchi2 = dl_dchi2;
  R.dl_dmap = dl_dmap;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ctx->last_stream = s;
  const int k = ctx->opt.mode == 0
                    ? strict::refit_backward(R, ctx->P, ctx->steps3, ctx->sms, s)
                    : fast::refit_backward(R, ctx->P, ctx->steps3, ctx->sms, s);
  ctx->launches_last = k;
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return TPC_OK;
}

tpc_status tpc_cluster_removal(tpc_ctx* ctx, const tpc_removal_options* o, tpc_removal* out,
                               void* cuda_stream) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (!o || !out) return fail(ctx, TPC_ERR_INVALID_ARG, "null options or output");
  if ((o->mode != 1 && o->mode != 2) || !(o->qpt > 0.0f) || !(o->protect >= 0.0f) ||
      !(o->remove >= 0.0f) || !(o->edge >= 0.0f) || !(o->occ_w >= 0.0f) ||
      !(o->p2_grow >= 0.0f) || !(o->p2_shrink >= 0.0f) || !(o->leg_dq >= 0.0f) ||
      !(o->leg_dtgl >= 0.0f) || !(o->leg_dc > 0.0f) || o->occ_max < 0)
    return fail(ctx, TPC_ERR_INVALID_ARG, "cluster removal option out of range");
  if (!ctx->tracked)
    return fail(ctx, TPC_ERR_STATE, "cluster removal needs a preceding successful tracking call");
  FrameDev& F = ctx->F;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ctx->last_stream = s;
  RemovalParams R{};
  R.qpt = o->qpt; R.protect = o->protect; R.remove = o->remove; R.edge = o->edge;
  R.occ_w = o->occ_w; R.p2_grow = o->p2_grow; R.p2_shrink = o->p2_shrink;
  R.leg_dq = o->leg_dq; R.leg_dtgl = o->leg_dtgl; R.leg_dc = o->leg_dc;
  R.mode = o->mode; R.occ_max = o->occ_max;
  R.half = ctx->n_sectors / 2;
  R.nsec_frame = ctx->n_sectors;
  // centre bins at least the leg distance wide (with a margin for rounding)
  double cell = (double)o->leg_dc * 1.01 + 0.01;
  if (512.0 / cell > kCrMaxBinsX) cell = 512.0 / kCrMaxBinsX;
  R.nbx = (int)std::ceil(512.0 / cell);
  if (R.nbx < 1) R.nbx = 1;
  if (R.nbx > kCrMaxBinsX) R.nbx = kCrMaxBinsX;
  R.inv_cell = (float)(1.0 / cell);
  const double pi = 3.14159265358979323846;
  for (int k = 0; k < 18; ++k) {
    const double a = ((double)k + 0.5) * 20.0 * pi / 180.0;
    R.sec_cos[k] = (float)std::cos(a);
    R.sec_sin[k] = (float)std::sin(a);
  }
  const int nblk = (ctx->n_sectors * ctx->last_nf + R.half - 1) / R.half;
  if ((long)nblk * R.nbx * R.nbx > kCrBins)
    return fail(ctx, TPC_ERR_INVALID_ARG, "too many side blocks for the leg search");
  KParams Pc = ctx->P;
  Pc.n_sectors = ctx->n_sectors * ctx->last_nf;
  const long n = F.n;
  if (n > 0) CK(cudaMemsetAsync(F.cr_flags, 0, sizeof(unsigned) * n, s));
  CK(cudaMemsetAsync(F.cr_bin_cnt, 0, sizeof(int) * ((long)nblk * R.nbx * R.nbx + 1), s));
  CK(cudaMemsetAsync(&F.cnt->n_removed, 0, sizeof(int), s));
  const int k = ctx->opt.mode == 0 ? strict::cluster_removal(F, Pc, R, nblk, ctx->sms, s)
                                   : fast::cluster_removal(F, Pc, R, nblk, ctx->sms, s);
  ctx->launches_last = k;
  CK(cudaGetLastError());
  int nrem = 0;
  CK(cudaMemcpyAsync(&nrem, &F.cnt->n_removed, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  out->n_clusters = n;
  out->n_tracks = ctx->host_cnt.n_out;
  out->n_removed = nrem;
  out->flags = F.cr_out;
  out->track_class = F.cr_cls;
  out->leg_parent = F.cr_parent;
  return TPC_OK;
}

tpc_status tpc_debug_copy(tpc_ctx* ctx, const char* name, void* host_dst, int64_t cap,
                          int64_t* bytes) {
  if (!ctx || !name) return TPC_ERR_INVALID_ARG;
  FrameDev& F = ctx->F;
  const Counters& c = ctx->host_cnt;
  const long n = F.n;
  const long nrr = (long)ctx->n_sectors * ctx->n_rows;
  const long nst = c.n_starts < F.cap_tl ? c.n_starts : F.cap_tl;
  const long nft = c.n_merged < F.cap_ft ? c.n_merged : F.cap_ft;
  const void* src = nullptr;
  long nb = 0;
  const std::string w(name);
  if (w == "counters") { src = F.cnt; nb = sizeof(Counters); }
  else if (w == "rows") { src = F.rows; nb = sizeof(RowGrid) * nrr; }
  else if (w == "bin_first") { src = F.bin_first; nb = sizeof(int) * ((long)c.n_bins + 1); }
  else if (w == "syz") { src = F.syz; nb = 8 * n; }
  else if (w == "sid") { src = F.sid; nb = 4 * n; }
  else if (w == "srow") { src = F.srow; nb = 2 * n; }
  else if (w == "lup") { src = F.lup; nb = 4 * n; }
  else if (w == "ldn") { src = F.ldn; nb = 4 * n; }
  else if (w == "cup") { src = F.cup; nb = 4 * n; }
  else if (w == "cdn") { src = F.cdn; nb = 4 * n; }
  else if (w == "starts") { src = F.starts; nb = 4 * nst; }
  else if (w == "tl_n") { src = F.tl_n; nb = 4 * nst; }
  else if (w == "tl_rlo") { src = F.tl_rlo; nb = 4 * nst; }
  else if (w == "tl_rhi") { src = F.tl_rhi; nb = 4 * nst; }
  else if (w == "tl_chi2") { src = F.tl_chi2; nb = 4 * nst; }
  else if (w == "tl_x") { src = F.tl_x; nb = 4 * nst; }
  else if (w == "tl_par") { src = F.tl_par; nb = 4 * 5 * nst; }
  else if (w == "tl_cov") { src = F.tl_cov; nb = 4 * 15 * nst; }
  else if (w == "tl_hits") { src = F.tl_hits; nb = 4L * kMaxRows * nst; }
  else if (w == "tl_kept") { src = F.tl_kept; nb = 4L * kMaxRows * nst; }
  else if (w == "tl_acc") { src = F.tl_acc; nb = 4 * nst; }
  else if (w == "tl_nkept") { src = F.tl_nkept; nb = 4 * nst; }
  else if (w == "owner_key") { src = F.owner_key; nb = 8 * n; }
  else if (w == "sec_owner") { src = F.sec_owner; nb = 4 * n; }
  else if (w == "sused") { src = F.sused; nb = n; }
  else if (w == "cr_flags") { src = F.cr_flags; nb = 4 * n; }
  else if (w == "cr_centre_x") { src = F.cr_cx; nb = 4L * c.n_out; }
  else if (w == "cr_centre_y") { src = F.cr_cy; nb = 4L * c.n_out; }
  else if (w == "pass_start") { src = F.cnt->pass_start; nb = sizeof(int) * kMaxSeedIters; }
  else if (w == "st_tl") { src = F.st_tl; nb = 4L * c.n_tracks; }
  else if (w == "st_ok") { src = F.st_ok; nb = 4L * c.n_tracks; }
  else if (w == "st_key") { src = F.st_key; nb = 4L * c.n_tracks; }
  else if (w == "st_next") { src = F.st_next; nb = 4L * c.n_tracks; }
  else if (w == "st_bestB") { src = F.st_bestB; nb = 4L * c.n_tracks; }
  else if (w == "st_bestchi") { src = F.st_bestchi; nb = 4L * c.n_tracks; }
  else if (w == "st_bestA") { src = F.st_bestA; nb = 8L * c.n_tracks; }
  else if (w == "st_ie") { src = F.st_ie; nb = 4L * kStateF * c.n_tracks; }
  else if (w == "st_oe") { src = F.st_oe; nb = 4L * kStateF * c.n_tracks; }
  else if (w == "ft_key") { src = F.ft_key; nb = 4L * nft; }
  else if (w == "ft_ok") { src = F.ft_ok; nb = 4L * nft; }
  else if (w == "ft_nst") { src = F.ft_nst; nb = 4L * nft; }
  else if (w == "ft_st_cl") { src = F.ft_st_cl; nb = 4L * kMaxRows * nft; }
  else if (w == "ft_st_rs") { src = F.ft_st_rs; nb = 2L * kMaxRows * nft; }
  else if (w == "ft_flag") { src = F.ft_flag; nb = 1L * kMaxRows * nft; }
  else if (w == "ft_ncand") { src = F.ft_ncand; nb = 1L * F.nslot * nft; }
  else if (w == "ft_cand") { src = F.ft_cand; nb = 4L * F.nslot * kMaxCand * nft; }
  else if (w == "ft_cchi") { src = F.ft_cchi; nb = 4L * F.nslot * kMaxCand * nft; }
  else if (w == "ft_assigned") { src = F.ft_assigned; nb = 4L * F.nslot * nft; }
  else if (w == "ft_next") { src = F.ft_next; nb = 4L * nft; }
  else if (w == "ft_nout") { src = F.ft_nout; nb = 4L * nft; }
  else if (w == "ft_ext_sec") { src = F.ft_ext_sec; nb = 2L * 2 * ctx->P.ext_rows * nft; }
  else if (w == "ft_n") { src = F.ft_n; nb = 4L * nft; }
  else if (w == "out_par") { src = F.out_par; nb = 4L * 5 * c.n_out; }
  else if (w == "out_cov") { src = F.out_cov; nb = 4L * 15 * c.n_out; }
  else if (w == "out_chi2") { src = F.out_chi2; nb = 4L * c.n_out; }
  else if (w == "out_x") { src = F.out_x; nb = 4L * c.n_out; }
  else if (w == "out_ndf") { src = F.out_ndf; nb = 4L * c.n_out; }
  else if (w == "out_sector") { src = F.out_sector; nb = 4L * c.n_out; }
  else if (w == "out_ncl") { src = F.out_ncl; nb = 4L * c.n_out; }
  else if (w == "out_offset") { src = F.out_offset; nb = 4L * (c.n_out + 1); }
  else if (w == "out_ids") { src = F.out_ids; nb = 4L * c.n_refs; }
  else if (w == "out_key") { src = F.out_key; nb = 4L * c.n_out; }
  else if (w == "attach") { src = F.attach; nb = 4 * n; }
  else return fail(ctx, TPC_ERR_INVALID_ARG, "unknown buffer %s", name);
  if (bytes) *bytes = nb;
  if (!host_dst) return TPC_OK;
  if (cap < nb) return fail(ctx, TPC_ERR_CAPACITY, "buffer %s needs %ld bytes", name, nb);
  if (ctx->last_stream) cudaStreamSynchronize(ctx->last_stream);
  if (nb > 0 && cudaMemcpy(host_dst, src, nb, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(ctx, TPC_ERR_CUDA, "debug copy of %s failed", name);
  return TPC_OK;
}

tpc_status tpc_profile(tpc_ctx* ctx, int enable) {
  if (!ctx) return TPC_ERR_INVALID_ARG;
  if (enable && !ctx->ev[0]) {
    for (auto& e : ctx->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return fail(ctx, TPC_ERR_CUDA, "event create");
  }
  ctx->prof = enable != 0;
  for (int i = 0; i < kNumStages; ++i) {
    ctx->stage_ms[i] = 0.0;
    ctx->stage_calls[i] = 0;
    ctx->stage_launches[i] = 0;
  }
  return TPC_OK;
}

tpc_status tpc_stage_stats(const tpc_ctx* ctx, int32_t i, const char** name, double* ms_total,
                           int64_t* calls, int64_t* launches) {
  if (!ctx || i < 0 || i >= kNumStages) return TPC_ERR_INVALID_ARG;
  if (name) *name = kStages[i].name;
  if (ms_total) *ms_total = ctx->stage_ms[i];
  if (calls) *calls = ctx->stage_calls[i];
  if (launches) *launches = ctx->stage_launches[i];
  return TPC_OK;
}

int64_t tpc_last_launches(const tpc_ctx* ctx) { return ctx ? ctx->launches_last : 0; }

int64_t tpc_refit_generation(const tpc_ctx* ctx) { return ctx ? ctx->refit_gen : -1; }

const char* tpc_last_error(const tpc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

void tpc_destroy(tpc_ctx* ctx) {
  if (!ctx) return;
  for (void* p : ctx->allocs) cudaFree(p);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->ev_in) cudaEventDestroy(ctx->ev_in);
  if (ctx->ev_out) cudaEventDestroy(ctx->ev_out);
  if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
  delete ctx;
}

}  // extern "C"
