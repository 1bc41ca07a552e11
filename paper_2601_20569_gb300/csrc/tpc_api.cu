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
};
constexpr int kNumStages = sizeof(kStages) / sizeof(kStages[0]);
}  // namespace

struct tpc_ctx {
  tpc_options opt{};
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
  P.grid_occ = 1.0f;
}

#define CK(call)                                                                       \
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
      (opt->mode != 0 && opt->mode != 1) || opt->cap_clusters > (1L << 30))
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
  ctx->P.n_rows = geo->n_rows;
  ctx->P.n_sectors = geo->n_sectors;
  if (map) ctx->map = *map;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, dev);
  if (ctx->sms <= 0) ctx->sms = 1;

  const long n = opt->cap_clusters;
  ctx->cap_n = n;
  const long nrr = (long)geo->n_sectors * geo->n_rows;
  FrameDev& F = ctx->F;
  F.cap_bins = (long)((double)n / ctx->P.grid_occ) + nrr * 65;
  F.cap_tl = opt->cap_tracklets > 0 ? opt->cap_tracklets : n / 10 + 4096;
  bool ok = true;
  ok &= dalloc(ctx, (float**)&F.row_x, geo->n_rows);
  ok &= dalloc(ctx, &F.row_cnt, nrr);
  ok &= dalloc(ctx, &F.row_zmin, nrr);
  ok &= dalloc(ctx, &F.row_zmax, nrr);
  ok &= dalloc(ctx, &F.rows, nrr);
  ok &= dalloc(ctx, &F.bin_cnt, F.cap_bins + 1);
  ok &= dalloc(ctx, &F.bin_first, F.cap_bins + 1);
  ok &= dalloc(ctx, &F.cl_bin, n);
  ok &= dalloc(ctx, &F.cl_slot, n);
  ok &= dalloc(ctx, &F.sy, n);
  ok &= dalloc(ctx, &F.sz, n);
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
  ok &= dalloc(ctx, &F.tl_n, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_rlo, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_rhi, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_hits, F.cap_tl * kMaxRows);
  ok &= dalloc(ctx, &F.owner_key, n);
  ok &= dalloc(ctx, &F.tl_acc, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_nkept, F.cap_tl);
  ok &= dalloc(ctx, &F.tl_kept, F.cap_tl * kMaxRows);
  ok &= dalloc(ctx, &F.sec_owner, n);
  ok &= dalloc(ctx, &F.cnt, 1);
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
  return TPC_OK;
}

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
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ctx->last_stream = s;
  FrameDev& F = ctx->F;
  F.y = cl->y;
  F.z = cl->z;
  F.row = cl->row;
  F.sector = cl->sector;
  F.n = cl->n;
  const long nrr = (long)ctx->n_sectors * ctx->n_rows;
  const long n = F.n;
  CK(cudaMemsetAsync(F.cnt, 0, sizeof(Counters), s));
  CK(cudaMemsetAsync(F.row_cnt, 0, sizeof(int) * nrr, s));
  CK(cudaMemsetAsync(F.row_zmin, 0xFF, sizeof(unsigned) * nrr, s));
  CK(cudaMemsetAsync(F.row_zmax, 0, sizeof(unsigned) * nrr, s));
  CK(cudaMemsetAsync(F.bin_cnt, 0, sizeof(int) * (F.cap_bins + 1), s));
  if (n > 0) {
    CK(cudaMemsetAsync(F.owner_key, 0, sizeof(unsigned long long) * n, s));
    CK(cudaMemsetAsync(F.sec_owner, 0xFF, sizeof(int) * n, s));
  }
  ctx->launches_last = 0;
  if (ctx->prof) CK(cudaEventRecord(ctx->ev[0], s));
  for (int i = 0; i < kNumStages; ++i) {
    const StageFn fn = ctx->opt.mode == 0 ? kStages[i].strict_fn : kStages[i].fast_fn;
    const int k = fn(F, ctx->P, ctx->sms, s);
    ctx->launches_last += k;
    ctx->stage_launches[i] += k;
    if (ctx->prof) CK(cudaEventRecord(ctx->ev[i + 1], s));
  }
  CK(cudaGetLastError());
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
  const Counters& c = ctx->host_cnt;
  std::memset(out, 0, sizeof(*out));
  if (c.err & kErrInput) return fail(ctx, TPC_ERR_INVALID_INPUT, "invalid cluster (NaN/Inf, row or sector out of range)");
  if (c.err & kErrCapBins) {
    if (needed) *needed = c.n_bins;
    return fail(ctx, TPC_ERR_CAPACITY, "grid bins %d exceed capacity %ld", c.n_bins, F.cap_bins);
  }
  if (c.err & kErrCapTracklets) {
    if (needed) *needed = c.need_tracklets;
    return fail(ctx, TPC_ERR_CAPACITY, "start hits %d exceed tracklet capacity %ld", c.n_starts,
                F.cap_tl);
  }
  out->attach = F.sec_owner;
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
  const void* src = nullptr;
  long nb = 0;
  const std::string w(name);
  if (w == "counters") { src = F.cnt; nb = sizeof(Counters); }
  else if (w == "rows") { src = F.rows; nb = sizeof(RowGrid) * nrr; }
  else if (w == "bin_first") { src = F.bin_first; nb = sizeof(int) * ((long)c.n_bins + 1); }
  else if (w == "sy") { src = F.sy; nb = 4 * n; }
  else if (w == "sz") { src = F.sz; nb = 4 * n; }
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

const char* tpc_last_error(const tpc_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

void tpc_destroy(tpc_ctx* ctx) {
  if (!ctx) return;
  for (void* p : ctx->allocs) cudaFree(p);
  for (auto& e : ctx->ev)
    if (e) cudaEventDestroy(e);
  delete ctx;
}

}  // extern "C"
