// Track merging and the final fit (Sec. 2 "track merging and track fit",
// Sec. 3 Phases I and II):
//   a7  sector refit of every accepted tracklet and mutual-best merging of
//       track ends inside a sector and between adjacent sectors of one half;
//   a8  space-charge correction of clusters with a cubic B-spline map;
//   a9  three-iteration linearised Kalman fit: iteration 1 inward stores the
//       predicted (y,z) and covariance per station, iteration 2 outward
//       interpolates and flags outliers, iteration 3 inward refits;
//   a10 Phase II re-attachment on the inner rows: candidates within the
//       interpolation cut, second ambiguity solving in cand_k rounds;
//   a11 output compaction and cluster-to-track attachment.
// Compiled twice (strict / fast) like the sector kernels.
#include <cuda_runtime.h>

#include <cstdint>

#include "tpc_kernels.h"
#include "tpc_model.cuh"
#include "tpc_util.cuh"

namespace tpc {
namespace TPC_NS {

namespace {

// --------------------------------------------------------- a8 distortion map
__device__ __forceinline__ void spline_w(float f, float* w) {
  const float g = 1.0f - f;
  const float f2 = f * f, f3 = f2 * f;
  w[0] = g * g * g / 6.0f;
  w[1] = (3.0f * f3 - 6.0f * f2 + 4.0f) / 6.0f;
  w[2] = (-3.0f * f3 + 3.0f * f2 + 3.0f * f + 1.0f) / 6.0f;
  w[3] = f3 / 6.0f;
}

__device__ __forceinline__ void spline_span(float t, int n, int& i, float& f) {
  const float tmax = (float)(n - 3);
  if (t < 0.0f) t = 0.0f;
  if (t > tmax) t = tmax;
  i = (int)floorf(t);
  if (i > n - 4) i = n - 4;
  f = t - (float)i;
}

struct SplinePt {
  int ip, ir, iz;
  float wp[4], wr[4], wz[4];
};

__device__ __forceinline__ SplinePt spline_point(const MapDev& M, const KParams& P, int sector,
                                                 float x, float y, float zdrift) {
  SplinePt sp;
  const int sphi = sector % P.n_phi;
  const float u = ((float)sphi + 0.5f) + 0.5f * (y / x) / P.tan_half;
  const float tp = u * M.phi_scale - 0.5f;
  sp.ip = (int)floorf(tp);
  const float fp = tp - (float)sp.ip;
  const float r = sqrtf(x * x + y * y);
  float fr, fz;
  spline_span((r - M.rmin) * M.r_scale, M.nr, sp.ir, fr);
  float zc = zdrift;
  if (zc < M.zmin) zc = M.zmin;
  if (zc > M.zmax) zc = M.zmax;
  spline_span((zc - M.zmin) * M.z_scale, M.nz, sp.iz, fz);
  spline_w(fp, sp.wp);
  spline_w(fr, sp.wr);
  spline_w(fz, sp.wz);
  return sp;
}

__device__ __forceinline__ int phi_index(int ip, int e, int nphi) {
  return ((ip - 1 + e) % nphi + nphi) % nphi;
}

__device__ __forceinline__ void map_eval(const MapDev& M, const KParams& P, int sector, float x,
                                         float y, float zdrift, float* D) {
  D[0] = D[1] = D[2] = 0.0f;
  if (!M.on) return;
  const SplinePt sp = spline_point(M, P, sector, x, y, zdrift);
  int pidx[4];
#pragma unroll
  for (int e = 0; e < 4; ++e) pidx[e] = phi_index(sp.ip, e, M.nphi);
  for (int comp = 0; comp < 3; ++comp) {
    float acc = 0.0f;
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) {
        const float wzr = sp.wz[a] * sp.wr[b];
        const float* row = M.c + (((long)comp * M.nz + (sp.iz + a)) * M.nr + (sp.ir + b)) * M.nphi;
#pragma unroll
        for (int e = 0; e < 4; ++e) acc = acc + wzr * sp.wp[e] * __ldg(row + pidx[e]);
      }
    D[comp] = acc;
  }
}

// Corrected measurement projected back onto the pad row along the reference.
__device__ __forceinline__ bool corrected(const MapDev& M, const KParams& P, int sector, float x,
                                          float y, float z, float z0, const float* ref, float& my,
                                          float& mz) {
  float D[3];
  map_eval(M, P, sector, x, y, z - z0, D);
  my = y + D[1];
  mz = z + D[2];
  if (D[0] != 0.0f) {
    StepJ st;
    if (!helix_step(ref, D[0], P, st, P.fit_max_snp)) return false;
    my = my - (st.p0 - ref[0]);
    mz = mz - (st.p1 - ref[1]);
  }
  return true;
}

// ------------------------------------------------------ a7 sector refit
__device__ __forceinline__ unsigned long long pack_chi_key(float chi2, int key) {
  return ((unsigned long long)f2o(chi2) << 32) | (unsigned long long)(unsigned)key;
}

// Compaction of accepted tracklets into the sector-track list (tracklet order).
__global__ void k_acc_count(FrameDev F) {
  __shared__ int sh[32];
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = (!F.cnt->err && i < nst && F.tl_acc[i]) ? 1 : 0;
  int tot;
  block_exscan(f, sh, &tot);
  if (threadIdx.x == 0) F.scan_tmp[blockIdx.x] = tot;
}

__global__ void k_acc_write(FrameDev F) {
  __shared__ int sh[32];
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = (!F.cnt->err && i < nst && F.tl_acc[i]) ? 1 : 0;
  int tot;
  const int ex = block_exscan(f, sh, &tot);
  // room for the track's kept-cluster positions: one atomic per warp (the
  // layout of the position array is arbitrary; every track reads its own range)
  const int nk = f ? F.tl_nkept[i] : 0;
  const int lane = threadIdx.x & 31;
  int incl = nk;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  int base = 0;
  if (lane == 31 && incl > 0) base = atomicAdd(&F.cnt->n_pos, incl);
  base = __shfl_sync(0xffffffffu, base, 31);
  const unsigned act = __ballot_sync(0xffffffffu, f != 0);
  if (f) {
    const int j = F.scan_tmp[blockIdx.x] + ex;
    F.st_tl[j] = i;
    F.st_off[j] = base + incl - nk;
    // scheduling bucket of the sector refit: most clusters first (the lanes
    // of one bucket take their places with one atomic; the order inside a
    // bucket only schedules the refit)
    const int b = kOrdBuckets - 1 - min(kOrdBuckets - 1, nk);
    const unsigned peers = __match_any_sync(act, b);
    const int leader = __ffs(peers) - 1;
    int slot = 0;
    if (lane == leader) slot = atomicAdd(&F.st_ord_cnt[b], __popc(peers));
    slot = __shfl_sync(peers, slot, leader);
    F.st_obucket[j] = b;
    F.st_oslot[j] = slot + __popc(peers & ((1u << lane) - 1u));
  }
}

// Positions (pad-row x, y, z) of every sector track's kept clusters, in
// kept order, gathered once so that the two passes of the sector refit read
// each track's clusters as one contiguous run.
__global__ void k_st_gather(FrameDev F, KParams P) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  if (F.cnt->n_pos > F.cap_pos) {
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&F.cnt->err, kErrCapPos);
    return;
  }
  const int NR = P.n_rows;
  __shared__ float rx[kMaxRows];
  for (int r = threadIdx.x; r < NR; r += blockDim.x) rx[r] = F.row_x[r];
  __syncthreads();
  // One warp per 32 consecutive tracks: lane j loads track j's tracklet,
  // length and output place (all lanes at once), then the warp takes the
  // tracks one by one, its lanes reading the whole kept list (up to kMaxRows
  // entries, all loads issued before the positions they address) and
  // writing the positions 32 at a time.
  constexpr int kChunks = (kMaxRows + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int j0 = 32 * (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); j0 < ns;
       j0 += 32 * nw) {
    int ti = 0, nk = 0, off = 0;
    if (j0 + lane < ns) {
      ti = F.st_tl[j0 + lane];
      nk = F.tl_nkept[ti];
      off = F.st_off[j0 + lane];
    }
    for (int j = 0; j < 32; ++j) {
      const int tj = __shfl_sync(0xffffffffu, ti, j);
      const int nj = __shfl_sync(0xffffffffu, nk, j);
      const int oj = __shfl_sync(0xffffffffu, off, j);
      const int* K = F.tl_kept + (long)tj * kMaxRows;
      float4* out = F.st_pos + oj;
      int c[kChunks];
#pragma unroll
      for (int u = 0; u < kChunks; ++u) {
        const int m = lane + 32 * u;
        c[u] = m < nj ? K[m] : -1;
      }
      float2 yz[kChunks];
      int rr[kChunks];
#pragma unroll
      for (int u = 0; u < kChunks; ++u) {
        yz[u] = c[u] >= 0 ? F.syz[c[u]] : make_float2(0.0f, 0.0f);
        rr[u] = c[u] >= 0 ? F.srow[c[u]] : 0;
      }
#pragma unroll
      for (int u = 0; u < kChunks; ++u)
        if (c[u] >= 0) out[lane + 32 * u] = make_float4(rx[rr[u] % NR], yz[u].x, yz[u].y, 0.0f);
    }
  }
}

// Sector refit of one track over its kept clusters' positions PS[j], j = j0,
// j0+dj, ... (nsteps steps).  Each position is loaded one step ahead of the
// filter, so the load overlaps the arithmetic of the current step.
__device__ __forceinline__ bool refit_pass(const KParams& P, const float4* PS, int j0, int dj,
                                           int nsteps, Trk<float>& t) {
  float4 nxt = PS[j0];
  for (int s = 0; s < nsteps; ++s) {
    const float4 cur = nxt;
    if (s + 1 < nsteps) nxt = PS[j0 + (s + 1) * dj];
    if (!propagate(t, cur.x, P, P.fit_max_snp)) return false;
    update(t, residual(t, cur.y, cur.z, P));
  }
  return true;
}

__global__ void __launch_bounds__(256) k_sector_refit(FrameDev F, KParams P) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  for (int q = queue_next(&F.cnt->queue[kQSectorRefit]); q < ns;
       q = queue_next(&F.cnt->queue[kQSectorRefit])) {
    const int i = F.st_order[q];
    const int ti = F.st_tl[i];
    const int nk = F.tl_nkept[ti];
    const int* K = F.tl_kept + (long)ti * kMaxRows;  // outermost first
    const float4* PS = F.st_pos + F.st_off[i];       // same order
    const int rs = F.srow[K[nk - 1]];
    F.st_key[i] = F.sid[F.starts[ti]];
    F.st_sector[i] = rs / NR;
    F.st_rmin[i] = rs % NR;
    F.st_rmax[i] = F.srow[K[0]] % NR;
    F.st_next[i] = -1;
    F.st_hasprev[i] = 0;
    F.st_bestB[i] = -1;
    F.st_bestA[i] = ~0ull;
    F.st_xbestB[i] = -1;
    F.st_xbestA[i] = ~0ull;
    F.st_dz[i] = 0.0f;
    Trk<float> t;
#pragma unroll
    for (int k = 0; k < 5; ++k) t.p[k] = F.tl_par[(long)ti * 5 + k];
    t.x = F.tl_x[ti];
    reset_cov(t.c, P);
    // outward over the kept clusters (innermost first), then inward
    bool ok = refit_pass(P, PS, nk - 1, -1, nk, t);
    if (ok) {
      put_state(F.st_oe + (long)i * kStateF, t, rs / NR);
      reset_cov(t.c, P);
      ok = refit_pass(P, PS, 0, 1, nk, t);
      if (ok) put_state(F.st_ie + (long)i * kStateF, t, rs / NR);
    }
    F.st_ok[i] = ok ? 1 : 0;
  }
}

// z range of each sector (from the row statistics of the grid build).
__global__ void k_sector_zrange(FrameDev F, KParams P) {
  const int s = blockIdx.x;
  __shared__ unsigned lo, hi;
  if (threadIdx.x == 0) { lo = 0xFFFFFFFFu; hi = 0u; }
  __syncthreads();
  for (int r = threadIdx.x; r < P.n_rows; r += blockDim.x) {
    const int rr = s * P.n_rows + r;
    if (F.row_cnt[rr] > 0) {
      atomicMin(&lo, F.row_zmin[rr]);
      atomicMax(&hi, F.row_zmax[rr]);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    float zl = 0.0f, zh = 1.0f;
    if (hi >= lo && hi != 0u) { zl = o2f(lo); zh = o2f(hi); }
    F.sec_zlo[s] = zl;
    F.sec_zinv[s] = zh > zl ? (float)kMergeZ / (zh - zl) : 0.0f;
  }
}

// Merge candidate index: inner ends binned by (sector, z, innermost row), so
// that the rows a pair test accepts form one contiguous range per z bin.
__device__ __forceinline__ int merge_zbin(const FrameDev& F, int s, float z) {
  return clampi((int)floorf((z - F.sec_zlo[s]) * F.sec_zinv[s]), 0, kMergeZ - 1);
}
__device__ __forceinline__ int merge_bin(const FrameDev& F, int nrows, int s, int r, float z) {
  return (s * kMergeZ + merge_zbin(F, s, z)) * nrows + r;
}

__global__ void k_ie_hist(FrameDev F, KParams P) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
    // (an inner end linked by the edge following takes no part in the merging)
    if (!F.st_ok[i] || F.st_hasprev[i]) { F.ie_bin[i] = -1; continue; }
    const int b = merge_bin(F, P.n_rows, F.st_sector[i], F.st_rmin[i],
                            F.st_ie[(long)i * kStateF + 1]);
    F.ie_bin[i] = b;
    F.ie_slot[i] = atomicAdd(&F.ie_cnt[b], 1);
  }
}

__global__ void k_ie_scatter(FrameDev F) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += gridDim.x * blockDim.x) {
    const int b = F.ie_bin[i];
    if (b < 0) continue;
    const int pos = F.ie_first[b] + F.ie_slot[i];
    F.ie_idx[pos] = i;
    const float* ie = F.st_ie + (long)i * kStateF;
    F.ie_rec[pos] = make_float4(ie[0], ie[1], ie[20], __int_as_float(i));
  }
}

// n consecutive queue items per calling lane, one atomic per warp.
__device__ __forceinline__ int queue_next_n(int* q, int n) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(q, __popc(mask) * n);
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u)) * n;
}

// chi2 of a 5-vector difference with a Cholesky factorisation (-1: not PD).
__device__ __forceinline__ float chi2_5(const float* d, const float* c) {
  float L[15];  // lower triangle, same indexing as the covariance
  for (int j = 0; j < 5; ++j) {
    float s = c[j * (j + 1) / 2 + j];
    for (int k = 0; k < j; ++k) s = s - L[j * (j + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
    if (!(s > 0.0f)) return -1.0f;
    L[j * (j + 1) / 2 + j] = sqrtf(s);
    for (int i = j + 1; i < 5; ++i) {
      float v = c[i * (i + 1) / 2 + j];
      for (int k = 0; k < j; ++k) v = v - L[i * (i + 1) / 2 + k] * L[j * (j + 1) / 2 + k];
      L[i * (i + 1) / 2 + j] = v / L[j * (j + 1) / 2 + j];
    }
  }
  float yv[5];
  float chi2 = 0.0f;
  for (int i = 0; i < 5; ++i) {
    float v = d[i];
    for (int k = 0; k < i; ++k) v = v - L[i * (i + 1) / 2 + k] * yv[k];
    yv[i] = v / L[i * (i + 1) / 2 + i];
    chi2 = chi2 + yv[i] * yv[i];
  }
  return chi2;
}

// The pair test of the outer end of A against the inner end of B.
__device__ __forceinline__ bool merge_test(const FrameDev& F, const KParams& P, int a, int b,
                                           float& chi2) {
  const int half = P.n_phi;
  const int sa = F.st_sector[a], sb = F.st_sector[b];
  if (sa / half != sb / half) return false;
  const int ds = ((sb % half) - (sa % half) + half) % half;
  if (ds != 0 && ds != 1 && ds != half - 1) return false;
  const int gap = F.st_rmin[b] - F.st_rmax[a];
  if (gap < 1 || gap > P.merge_max_gap) return false;
  const float* oe = F.st_oe + (long)a * kStateF;
  const float* ie = F.st_ie + (long)b * kStateF;
  const float zwin = P.merge_dz + fabsf(oe[3]) * P.merge_zspan;
  if (!(fabsf(ie[1] - oe[1]) <= zwin)) return false;
  Trk<float> t;
  get_state(oe, t);
  if (ds == 1 && !rotate(t, 1, P, P.fit_max_snp)) return false;
  if (ds == half - 1 && !rotate(t, -1, P, P.fit_max_snp)) return false;
  if (!propagate(t, ie[20], P, P.fit_max_snp)) return false;
  float d[5], c[15];
#pragma unroll
  for (int i = 0; i < 5; ++i) d[i] = ie[i] - t.p[i];
  if (!(fabsf(d[0]) <= P.merge_dy) || !(fabsf(d[1]) <= P.merge_dz)) return false;
#pragma unroll
  for (int i = 0; i < 15; ++i) c[i] = t.c[i] + ie[5 + i];
  chi2 = chi2_5(d, c);
  return chi2 >= 0.0f && chi2 < P.merge_chi2;
}

// Position prefilter of the pair test.  A's outer end turned into the frame
// of one of the three sectors searched (q = 0: its own, 1: the next, 2: the
// previous), with the terms of the helix step that depend on A alone; then
// A's position at B's x by the helix step's own expressions for y and z.  The
// prefilter rejects a candidate only where that position lies outside the
// window by more than a rounding margin, and leaves a failed rotation or step
// to the full test, so every decision is the full test's (merge_test), in
// either arithmetic mode.  Nearly all candidates of the index end here,
// before the covariance transport and the 5x5 chi2.
struct MergeA {
  float y, z, s0, c0, kap, tgl, x;
  int ok;
};

__device__ __forceinline__ MergeA merge_a(const float* oe, int q, const KParams& P) {
  Trk<float> t;  // the covariance is not read: its transport is dropped
#pragma unroll
  for (int i = 0; i < 5; ++i) t.p[i] = oe[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) t.c[i] = 0.0f;
  t.x = oe[20];
  bool ok = true;
  if (q == 1) ok = rotate(t, 1, P, P.fit_max_snp);
  else if (q == 2) ok = rotate(t, -1, P, P.fit_max_snp);
  MergeA m;
  m.y = t.p[0];
  m.z = t.p[1];
  m.s0 = t.p[2];
  m.tgl = t.p[3];
  m.kap = t.p[4] * P.kb;
  m.x = t.x;
#ifdef TPC_FAST_ARITH
  const float a0 = 1.0f - m.s0 * m.s0;
  m.c0 = a0 * rsqrtf(a0);
#else
  m.c0 = sqrtf(1.0f - m.s0 * m.s0);
#endif
  m.ok = ok ? 1 : 0;
  return m;
}

// The position (y, z) of A at x = xb (false: no rotation or no step).
__device__ __forceinline__ bool merge_pos(const MergeA& m, float xb, const KParams& P, float& yb,
                                          float& zb) {
  if (!m.ok) return false;
  const float dx = xb - m.x;
  const float s1 = m.s0 + m.kap * dx;
  if (!(fabsf(s1) < P.fit_max_snp)) return false;
#ifdef TPC_FAST_ARITH
  const float a1 = 1.0f - s1 * s1;
  const float c1 = a1 * rsqrtf(a1);
  const float t = (m.s0 + s1) * frcp(m.c0 + c1);
  const float tt = 1.0f + t * t;
  const float L1 = tt * rsqrtf(tt);
#else
  const float c1 = sqrtf(1.0f - s1 * s1);
  const float t = (m.s0 + s1) / (m.c0 + c1);
  const float L1 = sqrtf(1.0f + t * t);
#endif
  const float chord = dx * L1;
  const float u = m.kap * chord * 0.5f;
  yb = m.y + dx * t;
  zb = m.z + m.tgl * (chord * asinc_f(u));
  return true;
}

// Best merge partner of every outer end A, searched by a group of G lanes
// (G = 1: one thread per end).  The (sector, z bin) ranges of A's candidates
// in the index are dealt out to the lanes, their sizes summed by a group scan,
// and the candidates of all ranges dealt out G at a time; each lane runs the
// pair test of its candidate and the group's smallest (chi2, key of B) is
// found by shuffles.  The minimum does not depend on the visiting order, so
// every G gives the scalar search's result bit for bit.
template <int G>
__global__ void __launch_bounds__(256, 4) k_merge_best(FrameDev F, KParams P) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const unsigned gmask = G == 32 ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
  const int half = P.n_phi;
  for (;;) {
    // kFetch ends per queue fetch: lane gl < kFetch of the group looks at
    // end base + gl; the ends with no row to search (those that reach the
    // last rows) are answered at once, the others searched one after the
    // other by the whole group.  (A few ends per fetch: the atomics stay
    // few, and the last fetches of the grid stay short.)
    constexpr int kFetch = G < 8 ? G : 8;
    int base = 0;
    if (gl == 0) base = queue_next_n(&F.cnt->queue[kQMerge], kFetch);
    base = __shfl_sync(gmask, base, 0, G);
    if (base >= ns) break;
    const int am = base + gl;
    bool live = false;
    // (an outer end linked by the edge following is not searched)
    if (gl < kFetch && am < ns && F.st_ok[am] && F.st_next[am] < 0) {
      const int rmx = F.st_rmax[am];
      live = rmx + 1 <= min(rmx + P.merge_max_gap, P.n_rows - 1);
      if (!live) {
        F.st_bestB[am] = -1;
        F.st_bestchi[am] = 0.0f;
      }
    }
    for (unsigned todo = __ballot_sync(gmask, live) & gmask; todo; todo &= todo - 1) {
      const int a = __shfl_sync(gmask, am, (__ffs(todo) - 1) & (G - 1), G);
      const int keyA = F.st_key[a];
      unsigned long long best = ~0ull;
      int bb = -1;
      const int r0 = F.st_rmax[a] + 1;
      const int r1 = min(F.st_rmax[a] + P.merge_max_gap, P.n_rows - 1);
      {
        // the pair test needs 1 <= rmin(B) - rmax(A) <= merge_max_gap: only
        // those rows of the index are visited
        const int sa = F.st_sector[a];
        const int side = sa / half, ph = sa % half;
        const float* oe = F.st_oe + (long)a * kStateF;
        const float zwin = P.merge_dz + fabsf(oe[3]) * P.merge_zspan;
        const float m = 0.01f;
        int sq[3], zq[3], nq[3];
        int nr = 0;
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          sq[q] = side * half + (ph + (q == 0 ? 0 : q == 1 ? 1 : half - 1)) % half;
          zq[q] = merge_zbin(F, sq[q], oe[1] - zwin - m);
          nq[q] = merge_zbin(F, sq[q], oe[1] + zwin + m) - zq[q] + 1;
          nr += nq[q];
        }
        // A's state in the three sectors: lanes 0-2 of the group hold one
        // each and hand it to the lanes by shuffles (one lane computes it
        // where it needs it)
        MergeA ma{};
        if (G >= 4 && gl < 3) ma = merge_a(oe, gl, P);
        const float oz = oe[1];
        for (int j0 = 0; j0 < nr; j0 += G) {
          int lo = 0, cnt = 0, qj = 0;
          int j = j0 + gl;
          if (j < nr) {
            const int q = j < nq[0] ? 0 : j < nq[0] + nq[1] ? 1 : 2;
            j -= q == 0 ? 0 : q == 1 ? nq[0] : nq[0] + nq[1];
            const int base = (sq[q] * kMergeZ + zq[q] + j) * P.n_rows;
            lo = F.ie_first[base + r0];
            cnt = F.ie_first[base + r1 + 1] - lo;
            qj = q;
          }
          int inc = cnt;  // inclusive scan of the range sizes over the group
#pragma unroll
          for (int o = 1; o < G; o <<= 1) {
            const int v = __shfl_up_sync(gmask, inc, o, G);
            if (gl >= o) inc += v;
          }
          const int total = __shfl_sync(gmask, inc, G - 1, G);
          for (int c0 = 0; c0 < total; c0 += G) {
            const int c = c0 + gl;
            int L = 0;  // the range holding candidate c: first lane with inc > c
#pragma unroll
            for (int st = G / 2; st >= 1; st >>= 1) {
              const int v = __shfl_sync(gmask, inc, L + st - 1, G);
              if (v <= c) L += st;
            }
            const int excl = __shfl_sync(gmask, inc - cnt, L, G);
            const int lo_l = __shfl_sync(gmask, lo, L, G);
            const int q_l = __shfl_sync(gmask, qj, L, G);
            MergeA mq;
            if (G >= 4) {
              mq.y = __shfl_sync(gmask, ma.y, q_l, G);
              mq.z = __shfl_sync(gmask, ma.z, q_l, G);
              mq.s0 = __shfl_sync(gmask, ma.s0, q_l, G);
              mq.c0 = __shfl_sync(gmask, ma.c0, q_l, G);
              mq.kap = __shfl_sync(gmask, ma.kap, q_l, G);
              mq.tgl = __shfl_sync(gmask, ma.tgl, q_l, G);
              mq.x = __shfl_sync(gmask, ma.x, q_l, G);
              mq.ok = __shfl_sync(gmask, ma.ok, q_l, G);
            }
            if (c >= total) continue;
            // the indexed inner end: (y, z, x, track)
            const float4 rec = F.ie_rec[lo_l + (c - excl)];
            if (!(fabsf(rec.y - oz) <= zwin)) continue;  // the full test's z window
            if (G < 4) mq = merge_a(oe, q_l, P);
            float yb, zb;
            if (merge_pos(mq, rec.z, P, yb, zb) &&
                (fabsf(rec.x - yb) > P.merge_dy + 0.01f + 1e-5f * fabsf(rec.x) ||
                 fabsf(rec.y - zb) > P.merge_dz + 0.01f + 1e-5f * fabsf(rec.y)))
              continue;
            const int b = __float_as_int(rec.w);
            if (b == a || !F.st_ok[b]) continue;
            float chi2;
            if (!merge_test(F, P, a, b, chi2)) continue;
            const unsigned long long kb = pack_chi_key(chi2, F.st_key[b]);
            if (kb < best) {
              best = kb;
              bb = b;
            }
            atomicMin(&F.st_bestA[b], pack_chi_key(chi2, keyA));
          }
        }
      }
#pragma unroll
      for (int o = G / 2; o >= 1; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(gmask, best, o, G);
        const int obb = __shfl_xor_sync(gmask, bb, o, G);
        if (ob < best) {
          best = ob;
          bb = obb;
        }
      }
      if (gl == 0) {
        F.st_bestB[a] = bb;
        F.st_bestchi[a] = bb >= 0 ? o2f((unsigned)(best >> 32)) : 0.0f;
      }
    }
  }
}

__global__ void k_merge_link(FrameDev F) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < ns; a += gridDim.x * blockDim.x) {
    const int b = F.st_bestB[a];
    if (b < 0) continue;
    if (F.st_bestA[b] == pack_chi_key(F.st_bestchi[a], F.st_key[a])) {
      F.st_next[a] = b;
      F.st_hasprev[b] = 1;
    }
  }
}

// ------------------------------------------ across the central electrode
// chi2 of the 4-vector (y, sin phi, tan lambda, q/pT) of a 5-vector difference
// with the marginal covariance (z left out).
__device__ __forceinline__ float chi2_4z(const float* d, const float* c) {
  const int ix[4] = {0, 2, 3, 4};
  float L[4][4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float sj = c[ix[j] * (ix[j] + 1) / 2 + ix[j]];
    for (int k = 0; k < j; ++k) sj = sj - L[j][k] * L[j][k];
    if (!(sj > 0.0f)) return -1.0f;
    L[j][j] = sqrtf(sj);
    for (int i = j + 1; i < 4; ++i) {
      float v = c[ix[i] * (ix[i] + 1) / 2 + ix[j]];
      for (int k = 0; k < j; ++k) v = v - L[i][k] * L[j][k];
      L[i][j] = v / L[j][j];
    }
  }
  float yv[4];
  float chi2 = 0.0f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float v = d[ix[i]];
    for (int k = 0; k < i; ++k) v = v - L[i][k] * yv[k];
    yv[i] = v / L[i][i];
    chi2 = chi2 + yv[i] * yv[i];
  }
  return chi2;
}

// Pair test across the central electrode (Sec. 2 merges "then across the
// central electrode"): the outer end of A and the inner end of B in the same
// azimuthal sector of one frame on the two sides, B's innermost row 1 to
// merge_max_gap rows above A's outermost.  The measured z of the two sides
// differ by 2 vd t0 with t0 unknown in continuous readout (Sec. 1): z stays out
// of the chi2 (4 dof, summed covariances, below merge_chi2), and the sum of
// the two ends' z, in which t0 cancels, must lie within twice merge_dz +
// |tan lambda| * merge_zspan.  dz = z_A - z_B at B's x is the shift that
// brings B's side into A's measured z.
__device__ __forceinline__ bool cross_test(const FrameDev& F, const KParams& P, int a, int b,
                                           float& chi2, float& dz) {
  const int half = P.n_phi;
  const int sa = F.st_sector[a], sb = F.st_sector[b];
  if (sa / (2 * half) != sb / (2 * half) || sa / half == sb / half || sa % half != sb % half)
    return false;
  const int gap = F.st_rmin[b] - F.st_rmax[a];
  if (gap < 1 || gap > P.merge_max_gap) return false;
  const float* oe = F.st_oe + (long)a * kStateF;
  const float* ie = F.st_ie + (long)b * kStateF;
  const float zwin = P.merge_dz + fabsf(oe[3]) * P.merge_zspan;
  if (!(fabsf(oe[1] + ie[1]) <= zwin + zwin)) return false;
  Trk<float> t;
  get_state(oe, t);
  if (!propagate(t, ie[20], P, P.fit_max_snp)) return false;
  float d[5], c[15];
#pragma unroll
  for (int i = 0; i < 5; ++i) d[i] = ie[i] - t.p[i];
  if (!(fabsf(d[0]) <= P.merge_dy)) return false;
#pragma unroll
  for (int i = 0; i < 15; ++i) c[i] = t.c[i] + ie[5 + i];
  chi2 = chi2_4z(d, c);
  dz = t.p[1] - ie[1];
  return chi2 >= 0.0f && chi2 < P.merge_chi2;
}

// Chain ends against chain starts of the other side (after the merging within
// each side): the best start of every end; each start keeps its best end.
__global__ void k_cross_best(FrameDev F, KParams P) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  const int half = P.n_phi;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < ns; a += gridDim.x * blockDim.x) {
    if (!F.st_ok[a] || F.st_next[a] >= 0) continue;
    const int keyA = F.st_key[a];
    const int sa = F.st_sector[a];
    const int base = sa - sa % (2 * half);
    const int sb = base + (sa % (2 * half) + half) % (2 * half);
    const float* oe = F.st_oe + (long)a * kStateF;
    const float zwin = P.merge_dz + fabsf(oe[3]) * P.merge_zspan;
    const int r0 = F.st_rmax[a] + 1;
    const int r1 = min(F.st_rmax[a] + P.merge_max_gap, P.n_rows - 1);
    if (r0 > r1) continue;
    // the test needs |z_A + z_B| <= 2 zwin: B's inner-end z around -z_A
    const float m = 0.01f;
    const int z0 = merge_zbin(F, sb, -oe[1] - 2.0f * zwin - m);
    const int z1 = merge_zbin(F, sb, -oe[1] + 2.0f * zwin + m);
    int bb = -1, bkey = 0;
    float bchi = 0.0f, bdz = 0.0f;
    for (int zb = z0; zb <= z1; ++zb) {
      const int bin0 = (sb * kMergeZ + zb) * P.n_rows;
      const int lo = F.ie_first[bin0 + r0], hi = F.ie_first[bin0 + r1 + 1];
      for (int k = lo; k < hi; ++k) {
        const int b = F.ie_idx[k];
        if (!F.st_ok[b] || F.st_hasprev[b]) continue;
        float chi2, dz;
        if (!cross_test(F, P, a, b, chi2, dz)) continue;
        const int kb = F.st_key[b];
        if (bb < 0 || chi2 < bchi || (chi2 == bchi && kb < bkey)) {
          bb = b;
          bchi = chi2;
          bkey = kb;
          bdz = dz;
        }
        atomicMin(&F.st_xbestA[b], pack_chi_key(chi2, keyA));
      }
    }
    F.st_xbestB[a] = bb;
    F.st_xchi[a] = bchi;
    F.st_xdz[a] = bdz;
  }
}

__global__ void k_cross_link(FrameDev F) {
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < ns; a += gridDim.x * blockDim.x) {
    const int b = F.st_xbestB[a];
    if (b < 0) continue;
    if (F.st_xbestA[b] == pack_chi_key(F.st_xchi[a], F.st_key[a])) {
      F.st_next[a] = b;
      F.st_hasprev[b] = 1;
      F.st_dz[b] = F.st_xdz[a];
    }
  }
}

// Heads of chains -> fit tracks (compaction in sector-track order).
__device__ __forceinline__ int is_head(const FrameDev& F, int i, int ns) {
  return (i < ns && F.st_ok[i] && !F.st_hasprev[i]) ? 1 : 0;
}

__global__ void k_head_count(FrameDev F) {
  __shared__ int sh[32];
  const int ns = F.cnt->n_tracks;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = F.cnt->err ? 0 : is_head(F, i, ns);
  int tot;
  block_exscan(f, sh, &tot);
  if (threadIdx.x == 0) F.scan_tmp[blockIdx.x] = tot;
}

// Head list, plus whether the chain's fit updates run in FP64 (|q/pT| at
// its inner end above looper_qpt).
__global__ void k_head_write(FrameDev F, KParams P) {
  __shared__ int sh[32];
  const int ns = F.cnt->n_tracks;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int f = F.cnt->err ? 0 : is_head(F, i, ns);
  int tot;
  const int ex = block_exscan(f, sh, &tot);
  const int pos = F.scan_tmp[blockIdx.x] + ex;
  if (f && pos < F.cap_ft) {
    F.ft_head[pos] = i;
    const float q = fabsf(F.st_ie[(long)i * kStateF + 4]);
    F.ft_looper[pos] = (P.looper_qpt > 0.0f && q > P.looper_qpt) ? 1 : 0;
  }
}

// Processing order of the fit kernels: a stable partition of the fit tracks,
// loopers first.  On this GPU an FP64 update costs the whole warp the FP64
// pipe's time even when only one lane needs it, so loopers share warps; each
// part keeps list order (sector-major), which keeps the cluster accesses of a
// warp close together.  The two parts are served by two work queues (see
// fit_next).  No result depends on the order.
__device__ __forceinline__ int looper_flag(const FrameDev& F, int f) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  return (!F.cnt->err && f < nf) ? F.ft_looper[f] : 0;
}

__global__ void k_looper_count(FrameDev F) {
  __shared__ int sh[32];
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  int tot;
  block_exscan(looper_flag(F, f), sh, &tot);
  if (threadIdx.x == 0) F.scan_tmp[blockIdx.x] = tot;
}

__global__ void k_looper_write(FrameDev F) {
  __shared__ int sh[32];
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int fl = looper_flag(F, f);
  int tot;
  const int lr = F.scan_tmp[blockIdx.x] + block_exscan(fl, sh, &tot);  // loopers before f
  if (F.cnt->err || f >= nf) return;
  F.ft_order[fl ? lr : F.cnt->n_loopers + (f - lr)] = f;
}

__global__ void k_head_check(FrameDev F) {
  if (F.cnt->n_merged > F.cap_ft) {
    atomicOr(&F.cnt->err, kErrCapTracks);
    atomicMax(&F.cnt->need_tracks, F.cnt->n_merged);
  }
}

// Next fit track for the calling lane from the two queues of a fit kernel:
// loopers hold ft_order[0, nL), the other tracks ft_order[nL, nf).  Half of
// the warps (chosen pseudo-randomly over the grid) serve the looper queue
// first, the rest the other queue first; each turns to the other queue when
// its own is empty, so that the (narrow) FP64 pipe is in use while the other
// tracks are fitted rather than only at one end of the kernel.  Returns nf
// when both queues are empty.
__device__ __forceinline__ int fit_next(Counters* cnt, int qL, int qN, int nL, int nf) {
  const unsigned gw = (unsigned)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const bool looper_home = nL > 0 && ((gw * 2654435761u) >> 31) == 0u;
  if (looper_home) {
    const int q = queue_next(&cnt->queue[qL]);
    if (q < nL) return q;
    const int r = nL + queue_next(&cnt->queue[qN]);
    return r < nf ? r : nf;
  }
  const int r = nL + queue_next(&cnt->queue[qN]);
  if (r < nf) return r;
  const int q = nL > 0 ? queue_next(&cnt->queue[qL]) : nL;
  return q < nL ? q : nf;
}

// The fit kernels come in three parts: kPart 0 takes both queues (fit_next),
// 1 the other tracks only, 2 the loopers only.  Without a correction map
// iteration 3 runs as part 1 then part 2: part 1 carries neither the looper
// update nor the map evaluation, so it fits in 80 registers and keeps half
// as many warps again in flight as the full kernel (iteration 3: 6.7 -> 5.3
// ms per batch).  The order of the tracks changes no result.
template <int kPart>
__device__ __forceinline__ int fit_next_part(Counters* cnt, int qL, int qN, int nL, int nf) {
  if (kPart == 1) {
    const int r = nL + queue_next(&cnt->queue[qN]);
    return r < nf ? r : nf;
  }
  if (kPart == 2) {
    const int q = queue_next(&cnt->queue[qL]);
    return q < nL ? q : nf;
  }
  return fit_next(cnt, qL, qN, nL, nf);
}

// Looper flag of fit track f in part kPart (compile-time in parts 1 and 2).
template <int kPart>
__device__ __forceinline__ bool fit_looper(const FrameDev& F, int f) {
  return kPart == 2 ? true : kPart == 1 ? false : F.ft_looper[f] != 0;
}

// ------------------------------------------ a9/a10 linearised three-iteration fit
struct Lin {
  Trk<float> t;
  float r[5];
  int sector;
};

__device__ __forceinline__ void lin_start(Lin& L, const Trk<float>& s, int sector,
                                          const KParams& P) {
  L.t = s;
  reset_cov(L.t.c, P);
#pragma unroll
  for (int i = 0; i < 5; ++i) L.r[i] = s.p[i];
  L.sector = sector;
}

__device__ __forceinline__ bool lin_rotate(Lin& L, int dir, const KParams& P,
                                           float* jrec = nullptr) {
  const float ca = P.rot_c;
  const float sa = dir > 0 ? P.rot_s : -P.rot_s;
  const float snp = L.r[2];
  const float csp = sqrtf(1.0f - snp * snp);
  const float xn = L.t.x * ca + L.r[0] * sa;
  const float yn = L.r[0] * ca - L.t.x * sa;
  const float sn = snp * ca - csp * sa;
  const float cn = csp * ca + snp * sa;
  if (!(cn > 0.0f) || !(fabsf(sn) < P.fit_max_snp)) return false;
  const float j00 = csp / cn;
  const float j10 = -sa * L.r[3] / cn;
  const float j20 = -sa * (L.r[4] * P.kb);
  const float j22 = cn / csp;
  const float d0 = L.t.p[0] - L.r[0], d1 = L.t.p[1] - L.r[1], d2 = L.t.p[2] - L.r[2];
  float* c = L.t.c;
  const float m00 = c[0], m10 = c[1], m11 = c[2], m20 = c[3], m21 = c[4], m22 = c[5];
  const float m30 = c[6], m31 = c[7], m32 = c[8], m33 = c[9];
  const float m40 = c[10], m41 = c[11], m42 = c[12], m43 = c[13], m44 = c[14];
  const float a00 = j00 * m00;
  const float a10 = j10 * m00 + m10, a11 = j10 * m10 + m11;
  const float a20 = j20 * m00 + j22 * m20, a21 = j20 * m10 + j22 * m21,
              a22 = j20 * m20 + j22 * m22;
  c[0] = a00 * j00;
  c[1] = a10 * j00;
  c[2] = a10 * j10 + a11;
  c[3] = a20 * j00;
  c[4] = a20 * j10 + a21;
  c[5] = a20 * j20 + a22 * j22;
  c[6] = m30 * j00;
  c[7] = m30 * j10 + m31;
  c[8] = m30 * j20 + m32 * j22;
  c[9] = m33;
  c[10] = m40 * j00;
  c[11] = m40 * j10 + m41;
  c[12] = m40 * j20 + m42 * j22;
  c[13] = m43;
  c[14] = m44;
  L.r[0] = yn;
  L.r[2] = sn;
  L.t.x = xn;
  L.t.p[0] = L.r[0] + j00 * d0;
  L.t.p[1] = L.r[1] + (j10 * d0 + d1);
  L.t.p[2] = L.r[2] + (j20 * d0 + j22 * d2);
  if (jrec) {
    jrec[0] = j00;
    jrec[1] = j10;
    jrec[2] = j20;
    jrec[3] = j22;
  }
  return true;
}

__device__ __forceinline__ bool lin_propagate(Lin& L, float xnew, const KParams& P,
                                              StepJ* frec = nullptr) {
  const float dx = xnew - L.t.x;
  StepJ st;
  if (!helix_step(L.r, dx, P, st, P.fit_max_snp)) return false;
  if (frec) *frec = st;
  const float d0 = L.t.p[0] - L.r[0], d1 = L.t.p[1] - L.r[1], d2 = L.t.p[2] - L.r[2];
  const float d3 = L.t.p[3] - L.r[3], d4 = L.t.p[4] - L.r[4];
  L.r[0] = st.p0;
  L.r[1] = st.p1;
  L.r[2] = st.p2;
  L.t.p[0] = L.r[0] + (d0 + st.f02 * d2 + st.f04 * d4);
  L.t.p[1] = L.r[1] + (d1 + st.f12 * d2 + st.f13 * d3 + st.f14 * d4);
  L.t.p[2] = L.r[2] + (d2 + st.f24 * d4);
  cov_transport(L.t.c, st);
  add_ms(L.t.c, L.r, dx, P);
  L.t.x = xnew;
  return true;
}

// Station change: rotation (when the sector changes) and propagation.  The
// optional records receive the rotation Jacobian (jrec, *rotated set) and the
// propagation Jacobian (frec) for the adjoint.
__device__ __forceinline__ bool lin_goto(Lin& L, int sector, float x, const KParams& P,
                                         float* jrec = nullptr, bool* rotated = nullptr,
                                         StepJ* frec = nullptr) {
  if (rotated) *rotated = false;
  if (sector != L.sector) {
    const int half = P.n_phi;
    const int ds = ((sector % half) - (L.sector % half) + half) % half;
    if (ds == 1) {
      if (!lin_rotate(L, 1, P, jrec)) return false;
      if (rotated) *rotated = true;
    } else if (ds == half - 1) {
      if (!lin_rotate(L, -1, P, jrec)) return false;
      if (rotated) *rotated = true;
    } else if (ds != 0) {
      return false;
    }
    // ds == 0: the same azimuthal sector on the other side of the central
    // electrode, whose local frame is the same
    L.sector = sector;
  }
  return lin_propagate(L, x, P, frec);
}

__device__ __forceinline__ void inv2(float a00, float a01, float a11, float& i00, float& i01,
                                     float& i11) {
  const float idet = frcp(a00 * a11 - a01 * a01);
  i00 = a11 * idet;
  i01 = -a01 * idet;
  i11 = a00 * idet;
}

struct Interp {
  float y, z, c00, c01, c11;
};

__device__ __forceinline__ Interp interpolate(const float* a, const float* b) {
  float wa00, wa01, wa11, wb00, wb01, wb11;
  inv2(a[2], a[3], a[4], wa00, wa01, wa11);
  inv2(b[2], b[3], b[4], wb00, wb01, wb11);
  Interp I;
  inv2(wa00 + wb00, wa01 + wb01, wa11 + wb11, I.c00, I.c01, I.c11);
  const float v0 = (wa00 * a[0] + wa01 * a[1]) + (wb00 * b[0] + wb01 * b[1]);
  const float v1 = (wa01 * a[0] + wa11 * a[1]) + (wb01 * b[0] + wb11 * b[1]);
  I.y = I.c00 * v0 + I.c01 * v1;
  I.z = I.c01 * v0 + I.c11 * v1;
  return I;
}

__device__ __forceinline__ float chi2_interp(const Interp& I, float my, float mz,
                                             const KParams& P) {
  float w00, w01, w11;
  inv2(I.c00 + P.sy2, I.c01, I.c11 + P.sz2, w00, w01, w11);
  const float r0 = my - I.y, r1 = mz - I.z;
  return r0 * (w00 * r0 + w01 * r1) + r1 * (w01 * r0 + w11 * r1);
}

// Station list of fit track f: clusters of the chain (rows increasing) plus
// empty inner rows between two clusters of one sector.
__device__ __forceinline__ float zoff(const float* ie) {
  return ie[1] - ie[3] * sqrtf(ie[20] * ie[20] + ie[0] * ie[0]);
}

// Per fit track, ahead of the fit: the station list, the chain's last
// segment (whose outer end starts iteration 1), the identity key and the
// drift-time z offset.  One warp per track: the segments of the chain are
// taken in order, and the lanes take 32 kept clusters of a segment at a time
// (innermost first), their loads issued together.  A station is a kept
// cluster, preceded, on the inner rows of one sector, by an empty station on
// every row skipped since the previous cluster; a warp scan of the stations
// each cluster adds gives the places.  Stations beyond kMaxRows are dropped
// (none are reached: a chain's rows increase along it).
__global__ void k_fit_stations(FrameDev F, KParams P) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int f = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); f < nf; f += nw) {
    const int head = F.ft_head[f];
    int* SC = F.ft_st_cl + (long)f * kMaxRows;
    uint16_t* SR = F.ft_st_rs + (long)f * kMaxRows;
    // across the central electrode: the side of the first segment, and the
    // z shift of the clusters on the other side (set at the first segment
    // there, 0 for a chain on one side)
    const int side0 = (F.st_sector[head] / P.n_phi) & 1;
    float zsh = 0.0f;
    bool crossed = false;
    int last = head, ns = 0, prev = -1;
    for (int sg = head; sg >= 0; sg = F.st_next[sg]) {
      last = sg;
      if (!crossed && ((F.st_sector[sg] / P.n_phi) & 1) != side0) {
        crossed = true;
        zsh = F.st_dz[sg];
      }
      const int ti = F.st_tl[sg];
      const int nk = F.tl_nkept[ti];
      const int* K = F.tl_kept + (long)ti * kMaxRows;  // outermost first
      for (int j0 = 0; j0 < nk; j0 += 32) {
        const bool valid = j0 + lane < nk;
        const int c = valid ? K[nk - 1 - (j0 + lane)] : -1;
        const int rs = valid ? (int)F.srow[c] : 0;
        int prs = __shfl_up_sync(0xffffffffu, rs, 1);
        if (lane == 0) prs = prev;
        int gap = 0;
        if (valid && prs >= 0 && prs / NR == rs / NR)
          gap = max(0, min(rs % NR, P.inner_rows) - (prs % NR + 1));
        const int add = valid ? gap + 1 : 0;
        int incl = add;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int v = __shfl_up_sync(0xffffffffu, incl, o);
          if (lane >= o) incl += v;
        }
        const int pos = ns + incl - add;
        if (valid) {
          for (int q = 0; q < gap && pos + q < kMaxRows; ++q) {
            SC[pos + q] = -1;
            SR[pos + q] = (uint16_t)(rs - rs % NR + prs % NR + 1 + q);
          }
          if (pos + gap < kMaxRows) {
            SC[pos + gap] = c;
            SR[pos + gap] = (uint16_t)rs;
            // Phase III: clusters held by a station outside the inner region
            // are not extrapolation candidates of any track
            if (P.ext_rows > 0 && rs % NR >= P.inner_rows) F.ft_fixed[c] = 1;
          }
        }
        const int nvalid = min(32, nk - j0);
        ns += __shfl_sync(0xffffffffu, incl, 31);
        prev = __shfl_sync(0xffffffffu, rs, nvalid - 1);
      }
    }
    if (lane == 0) {
      F.ft_side0[f] = side0;
      F.ft_zsh[f] = zsh;
      F.ft_nst[f] = min(ns, kMaxRows);
      F.ft_key[f] = F.st_key[head];
      F.ft_last[f] = last;
      F.ft_z0[f] = zoff(F.st_ie + (long)head * kStateF);
      F.ft_next[f] = 0;
      F.ft_nout[f] = 0;
    }
  }
}

// Iterations 1 and 2 of the final fit (k_fit1, k_fit2) run as per-lane state
// machines: every loop iteration is one station (station change, then the
// iteration's own work, then the update) of the lane's current track, and a
// lane whose track ends takes the next one from the work queue, so the lanes
// of a warp issue the update (FP64 for loopers) together however unequal
// their tracks are.  Iteration 1 runs inward storing the predictions;
// iteration 2 runs outward, interpolates with them, flags outliers and
// collects the inner-row candidates (Sec. 3).  Two kernels rather than one:
// each carries only its own iteration's code and registers.
enum : int { kFitIdle = 0, kFitIn, kFitExt };

// One row step of the Phase III extrapolation, also over sector boundaries
// (Sec. 3): to row r in sector sec; beyond the sector's edge there (|y| >
// x tan 10 deg) the track continues in the neighbouring sector of the same
// side on that edge (rotation, then the row's x in the new frame), and stops
// if it still lies beyond that sector's edge plus edge_margin.
__device__ __forceinline__ bool ext_step(Lin& L, int& sec, int r, const float* rx,
                                         const KParams& P) {
  if (!lin_goto(L, sec, rx[r], P)) return false;
  if (fabsf(L.t.p[0]) > L.t.x * P.tan_half) {
    const int half = P.n_phi;
    const int base = sec - sec % half;
    const int nsec = base + (sec % half + (L.t.p[0] > 0.0f ? 1 : half - 1)) % half;
    if (!lin_goto(L, nsec, rx[r], P)) return false;
    sec = nsec;
  }
  return !(fabsf(L.t.p[0]) > L.t.x * P.tan_half + P.edge_margin);
}

// Tracks merged across the central electrode: the measured z of a cluster of
// sector sec in the frame of the track's first side (zside: the side whose
// clusters take the shift zsh, -1 for a track on one side), and the window
// centre cz of that frame in the measured z of sector sec.
__device__ __forceinline__ int shift_side(const FrameDev& F, int f) {
  return F.ft_zsh[f] != 0.0f ? 1 - F.ft_side0[f] : -1;
}
__device__ __forceinline__ float track_z(float z, int sec, int zside, float zsh, const KParams& P) {
  return zside >= 0 && ((sec / P.n_phi) & 1) == zside ? z + zsh : z;
}
// The shift that applies to the clusters of sector sec (0: none).
__device__ __forceinline__ float row_shift(int sec, int zside, float zsh, const KParams& P) {
  return zside >= 0 && ((sec / P.n_phi) & 1) == zside ? zsh : 0.0f;
}

__device__ __forceinline__ void inner_candidates(FrameDev& F, const KParams& P, const MapDev& M,
                                                 int f, int k, int rs, float x, const float* ref,
                                                 const Interp& I, float z0, float zadd) {
  const int sec = rs / P.n_rows;
  float cy = I.y, cz = I.z;
  {
    float D[3];
    map_eval(M, P, sec, x, I.y, I.z - z0, D);
    float sy = D[1], sz = D[2];
    if (D[0] != 0.0f) {
      StepJ stp;
      if (helix_step(ref, D[0], P, stp, P.fit_max_snp)) {
        sy = sy - (stp.p0 - ref[0]);
        sz = sz - (stp.p1 - ref[1]);
      }
    }
    cy = I.y - sy;
    cz = I.z - sz;
  }
  const float wy = sqrtf(P.int_chi2 * (I.c00 + P.sy2)) * 1.001f + P.attach_margin;
  const float wz = sqrtf(P.int_chi2 * (I.c11 + P.sz2)) * 1.001f + P.attach_margin;
  if (zadd != 0.0f) cz = cz - zadd;  // the row's measured z
  int* cand = F.ft_cand + ((long)f * F.nslot + k) * kMaxCand;
  float* cchi = F.ft_cchi + ((long)f * F.nslot + k) * kMaxCand;
  int nc = 0;
  int cid[kMaxCand];
  const RowGrid g = F.rows[rs];
  for_window(F.bin_first, g, cy - wy - 0.01f, cy + wy + 0.01f, cz - wz - 0.01f, cz + wz + 0.01f,
             [&](int kk) {
    const float2 pk = F.syz[kk];
    const float yk = pk.x, zk = pk.y;
    if (!(fabsf(yk - cy) <= wy && fabsf(zk - cz) <= wz)) return;
    float my, mz;
    if (!corrected(M, P, sec, x, yk, zadd != 0.0f ? zk + zadd : zk, z0, ref, my, mz)) return;
    const float c2 = chi2_interp(I, my, mz, P);
    if (!(c2 < P.int_chi2)) return;
    const int id = F.sid[kk];
    // insertion into the sorted top-cand_k list by (chi2, id)
    int pos = nc;
    while (pos > 0 && (c2 < cchi[pos - 1] || (c2 == cchi[pos - 1] && id < cid[pos - 1]))) --pos;
    if (pos >= P.cand_k) return;
    const int lim = nc < P.cand_k ? nc : P.cand_k - 1;
    for (int j = lim; j > pos; --j) {
      cand[j] = cand[j - 1];
      cchi[j] = cchi[j - 1];
      cid[j] = cid[j - 1];
    }
    cand[pos] = kk;
    cchi[pos] = c2;
    cid[pos] = id;
    if (nc < P.cand_k) ++nc;
  });
  F.ft_ncand[(long)f * F.nslot + k] = (uint8_t)nc;
  F.ft_assigned[(long)f * F.nslot + k] = -1;
}

// Phase III (Sec. 3): candidates of an extrapolated row (sorted (sector, row)
// rr) into candidate slot `js` of track f -- every cluster not held by a
// station outside the inner region whose chi2 to the prediction is below
// ext_chi2, the best cand_k by (chi2, id), for the second ambiguity solving.
__device__ __forceinline__ void ext_candidates(FrameDev& F, const KParams& P, const MapDev& M, int f,
                                            int js, int rr, const Lin& L, float z0,
                                            float zadd) {
  const int sec = rr / P.n_rows;
  float cy, cz;
  {
    float D[3];
    map_eval(M, P, sec, L.t.x, L.t.p[0], L.t.p[1] - z0, D);
    float sy = D[1], sz = D[2];
    if (D[0] != 0.0f) {
      StepJ stp;
      if (helix_step(L.r, D[0], P, stp, P.fit_max_snp)) {
        sy = sy - (stp.p0 - L.r[0]);
        sz = sz - (stp.p1 - L.r[1]);
      }
    }
    cy = L.t.p[0] - sy;
    cz = L.t.p[1] - sz;
  }
  const float wy = sqrtf(P.ext_chi2 * (L.t.c[0] + P.sy2)) * 1.001f + P.attach_margin;
  const float wz = sqrtf(P.ext_chi2 * (L.t.c[2] + P.sz2)) * 1.001f + P.attach_margin;
  if (zadd != 0.0f) cz = cz - zadd;  // the row's measured z
  const long slot = (long)f * F.nslot + js;
  int* cand = F.ft_cand + slot * kMaxCand;
  float* cchi = F.ft_cchi + slot * kMaxCand;
  int nc = 0;
  int cid[kMaxCand];
  const RowGrid g = F.rows[rr];
  for_window(F.bin_first, g, cy - wy - 0.01f, cy + wy + 0.01f, cz - wz - 0.01f, cz + wz + 0.01f,
             [&](int kk) {
    if (F.ft_fixed[kk]) return;
    const float2 pk = F.syz[kk];
    const float yk = pk.x, zk = pk.y;
    if (!(fabsf(yk - cy) <= wy && fabsf(zk - cz) <= wz)) return;
    float my, mz;
    if (!corrected(M, P, sec, L.t.x, yk, zadd != 0.0f ? zk + zadd : zk, z0, L.r, my, mz)) return;
    const float c2 = chi2_of(L.t, my, mz, P);
    if (!(c2 < P.ext_chi2)) return;
    const int id = F.sid[kk];
    int pos = nc;
    while (pos > 0 && (c2 < cchi[pos - 1] || (c2 == cchi[pos - 1] && id < cid[pos - 1]))) --pos;
    if (pos >= P.cand_k) return;
    const int lim = nc < P.cand_k ? nc : P.cand_k - 1;
    for (int j = lim; j > pos; --j) {
      cand[j] = cand[j - 1];
      cchi[j] = cchi[j - 1];
      cid[j] = cid[j - 1];
    }
    cand[pos] = kk;
    cchi[pos] = c2;
    cid[pos] = id;
    if (nc < P.cand_k) ++nc;
  });
  F.ft_ncand[slot] = (uint8_t)nc;
  F.ft_assigned[slot] = -1;
}

// Iteration 1 (inward, storing the predictions) and the Phase III
// extrapolation below the track, as a per-lane state machine: every loop
// iteration is one station (or extrapolated row) of the lane's current track,
// and a lane whose track ends takes the next one from the work queue.  The
// end state of iteration 1 goes to ft_end2 for k_fit2.
template <bool kMap, int kPart>
__global__ void __launch_bounds__(256, kPart == 1 ? 3 : 2)
    k_fit1(FrameDev F, KParams P, MapDev M) {
  if (!kMap) M.on = 0;  // (the map evaluation is compiled out)
  __shared__ float rx[kMaxRows];
  for (int r = threadIdx.x; r < P.n_rows; r += blockDim.x) rx[r] = F.row_x[r];
  __syncthreads();
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const int nL = min(F.cnt->n_loopers, nf);
  const int NR = P.n_rows;
  int phase = kFitIdle;
  int f = 0, ns = 0, k = 0;
  bool lp = false;  // FP64 updates (low-pT looper)
  float z0 = 0.0f;
  int zside = -1;   // central-electrode merging: side whose z takes zsh
  float zsh = 0.0f;
  int xsec = 0;     // sector of the extrapolation
  const int* SC = nullptr;
  const uint16_t* SR = nullptr;
  float* store = nullptr;
  Lin L;
  for (;;) {
    if (phase == kFitIdle) {
      const int q = fit_next_part<kPart>(F.cnt, kQFit12, kQFit12N, nL, nf);
      if (q >= nf) break;
      f = F.ft_order[q];
      lp = fit_looper<kPart>(F, f);
      ns = F.ft_nst[f];
      F.ft_ok[f] = 0;
      if (ns == 0) continue;  // not reached: every chain holds clusters
      z0 = F.ft_z0[f];
      zsh = F.ft_zsh[f];
      zside = shift_side(F, f);
      SC = F.ft_st_cl + (long)f * kMaxRows;
      SR = F.ft_st_rs + (long)f * kMaxRows;
      store = F.ft_store + (long)f * kMaxRows * 5;
      Trk<float> s0;
      get_state(F.st_oe + (long)F.ft_last[f] * kStateF, s0);
      lin_start(L, s0, SR[ns - 1] / NR, P);
      k = ns - 1;
      phase = kFitIn;
      continue;
    }
    if (phase == kFitExt) {
      // Phase III: one row of the inward extrapolation below the innermost
      // station (k counts the rows done)
      const int r = SR[0] % NR - 1 - k;
      bool go = k < P.ext_rows && r >= 0;
      if (go) go = ext_step(L, xsec, r, rx, P);
      if (go) {
        ext_candidates(F, P, M, f, kMaxInner + k, xsec * NR + r, L, z0,
                       row_shift(xsec, zside, zsh, P));
        F.ft_ext_sec[(long)f * 2 * P.ext_rows + k] = (uint16_t)xsec;
        ++k;
      } else {
        F.ft_next[f] = k;
        F.ft_ok[f] = 1;
        phase = kFitIdle;
      }
      continue;
    }
    // ---- one station.  The cluster does not depend on the state: it is
    // requested before the station change so that its latency overlaps the
    // arithmetic.
    const int rs = SR[k];
    const int c = SC[k];
    const int sec = rs / NR, row = rs % NR;
    float cy = 0.0f, cz = 0.0f;
    if (c >= 0) {
      const float2 pc = F.syz[c];
      cy = pc.x;
      cz = track_z(pc.y, sec, zside, zsh, P);
    }
    bool ok = true;
    if (k != ns - 1) ok = lin_goto(L, sec, rx[row], P);
    bool have = false;
    float my = 0.0f, mz = 0.0f;
    if (ok) {
      float* st = store + k * 5;
      st[0] = L.t.p[0]; st[1] = L.t.p[1]; st[2] = L.t.c[0]; st[3] = L.t.c[1]; st[4] = L.t.c[2];
      if (c >= 0) {
        ok = corrected(M, P, sec, L.t.x, cy, cz, z0, L.r, my, mz);
        have = ok;
      }
    }
    if (have) update_as(L.t, residual(L.t, my, mz, P), lp);
    if (!ok) {
      phase = kFitIdle;
      continue;
    }
    if (--k < 0) {
      // the end of iteration 1 starts iteration 2
      put_state(F.ft_end2 + (long)f * kStateF, L.t, L.sector);
      if (P.ext_rows > 0) {
        k = 0;
        xsec = SR[0] / NR;
        phase = kFitExt;
      } else {
        F.ft_ok[f] = 1;
        phase = kFitIdle;
      }
    }
  }
}

// Iteration 2 (outward) as the same kind of state machine: interpolation with
// the stored predictions, flags of outliers, inner-row candidates (Sec. 3,
// Phases I and II), then the Phase III extrapolation above the outermost
// station.  Starts from the end of iteration 1, ends in ft_end2.
enum : int { kFit2Idle = 0, kFit2St, kFit2Out };

template <bool kMap, int kPart>
__global__ void __launch_bounds__(256, kPart == 1 ? 3 : 2)
    k_fit2(FrameDev F, KParams P, MapDev M) {
  if (!kMap) M.on = 0;  // (the map evaluation is compiled out)
  __shared__ float rx[kMaxRows];
  for (int r = threadIdx.x; r < P.n_rows; r += blockDim.x) rx[r] = F.row_x[r];
  __syncthreads();
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const int nL = min(F.cnt->n_loopers, nf);
  const int NR = P.n_rows;
  int phase = kFit2Idle;
  int f = 0, ns = 0, k = 0;
  bool lp = false;  // FP64 updates (low-pT looper)
  float z0 = 0.0f;
  int zside = -1;   // central-electrode merging: side whose z takes zsh
  float zsh = 0.0f;
  int xsec = 0;     // sector of the extrapolation
  const int* SC = nullptr;
  const uint16_t* SR = nullptr;
  const float* store = nullptr;
  uint8_t* flag = nullptr;
  Lin L;
  for (;;) {
    if (phase == kFit2Idle) {
      const int q = fit_next_part<kPart>(F.cnt, kQFit2, kQFit2N, nL, nf);
      if (q >= nf) break;
      f = F.ft_order[q];
      if (!F.ft_ok[f]) continue;
      lp = fit_looper<kPart>(F, f);
      ns = F.ft_nst[f];
      z0 = F.ft_z0[f];
      zsh = F.ft_zsh[f];
      zside = shift_side(F, f);
      SC = F.ft_st_cl + (long)f * kMaxRows;
      SR = F.ft_st_rs + (long)f * kMaxRows;
      store = F.ft_store + (long)f * kMaxRows * 5;
      flag = F.ft_flag + (long)f * kMaxRows;
      Trk<float> s1;
      get_state(F.ft_end2 + (long)f * kStateF, s1);
      lin_start(L, s1, SR[0] / NR, P);
      k = 0;
      phase = kFit2St;
      continue;
    }
    if (phase == kFit2Out) {
      // Phase III: one row of the outward extrapolation above the outermost
      // station (k counts the rows done)
      const int r = SR[ns - 1] % NR + 1 + k;
      bool go = k < P.ext_rows && r < NR;
      if (go) go = ext_step(L, xsec, r, rx, P);
      if (go) {
        ext_candidates(F, P, M, f, kMaxInner + P.ext_rows + k, xsec * NR + r, L, z0,
                       row_shift(xsec, zside, zsh, P));
        F.ft_ext_sec[(long)f * 2 * P.ext_rows + P.ext_rows + k] = (uint16_t)xsec;
        ++k;
      } else {
        F.ft_nout[f] = k;
        phase = kFit2Idle;
      }
      continue;
    }
    // ---- one station.  The cluster and the stored prediction do not depend
    // on the state: they are requested before the station change.
    const int rs = SR[k];
    const int c = SC[k];
    const int sec = rs / NR, row = rs % NR;
    float cy = 0.0f, cz = 0.0f;
    if (c >= 0) {
      const float2 pc = F.syz[c];
      cy = pc.x;
      cz = track_z(pc.y, sec, zside, zsh, P);
    }
    float sv[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) sv[i] = store[k * 5 + i];
    bool ok = true;
    if (k != 0) ok = lin_goto(L, sec, rx[row], P);
    const bool inner = row < P.inner_rows;
    bool have = false;
    float my = 0.0f, mz = 0.0f;
    if (ok) {
      const float a[5] = {L.t.p[0], L.t.p[1], L.t.c[0], L.t.c[1], L.t.c[2]};
      const Interp I = interpolate(a, sv);
      flag[k] = 0;
      if (c >= 0 && !inner) {
        ok = corrected(M, P, sec, L.t.x, cy, cz, z0, L.r, my, mz);
        have = ok;
        if (ok) flag[k] = chi2_interp(I, my, mz, P) > P.int_chi2 ? 1 : 0;
      }
      if (ok && inner) {
        // Phase II candidates of this inner station: the search runs later in
        // k_inner_cand, over all (track, inner station) pairs at once
        float* ip = F.ft_ipol + ((long)f * kMaxInner + k) * kIpolF;
        ip[0] = I.y; ip[1] = I.z; ip[2] = I.c00; ip[3] = I.c01; ip[4] = I.c11;
        ip[5] = L.t.x;
#pragma unroll
        for (int i = 0; i < 5; ++i) ip[6 + i] = L.r[i];
        if (c >= 0) {
          ok = corrected(M, P, sec, L.t.x, cy, cz, z0, L.r, my, mz);
          have = ok;
        }
      }
    }
    if (have) update_as(L.t, residual(L.t, my, mz, P), lp);
    if (!ok) {
      F.ft_ok[f] = 0;
      phase = kFit2Idle;
      continue;
    }
    if (++k == ns) {
      put_state(F.ft_end2 + (long)f * kStateF, L.t, L.sector);
      k = 0;
      xsec = SR[ns - 1] / NR;
      phase = P.ext_rows > 0 ? kFit2Out : kFit2Idle;
    }
  }
}

// Second ambiguity solving, round k: bids (chi2, track key) per free cluster.
__device__ __forceinline__ bool inner_station(const FrameDev& F, const KParams& P, int f, int k) {
  return k < F.ft_nst[f] && (F.ft_st_rs[(long)f * kMaxRows + k] % P.n_rows) < P.inner_rows;
}

// Phase II candidate search of every inner station of every fit track, from
// the interpolation k_fit2 left for it (one thread per (track, station)).
template <bool kMap>
__global__ void k_inner_cand(FrameDev F, KParams P, MapDev M) {
  if (!kMap) M.on = 0;  // (the map evaluation is compiled out: 48 registers instead of 110)
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const long tot = (long)nf * P.inner_rows;
  for (long w = (long)blockIdx.x * blockDim.x + threadIdx.x; w < tot;
       w += (long)gridDim.x * blockDim.x) {
    const int f = (int)(w / P.inner_rows), k = (int)(w % P.inner_rows);
    if (!F.ft_ok[f] || !inner_station(F, P, f, k)) continue;
    const float* ip = F.ft_ipol + ((long)f * kMaxInner + k) * kIpolF;
    Interp I;
    I.y = ip[0];
    I.z = ip[1];
    I.c00 = ip[2];
    I.c01 = ip[3];
    I.c11 = ip[4];
    float ref[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) ref[i] = ip[6 + i];
    const int rs = F.ft_st_rs[(long)f * kMaxRows + k];
    inner_candidates(F, P, M, f, k, rs, ip[5], ref, I, F.ft_z0[f],
                     row_shift(rs / P.n_rows, shift_side(F, f), F.ft_zsh[f], P));
  }
}

// Work item w of the second ambiguity: (fit track, candidate slot).  Slots
// 0..inner_rows-1 are the inner stations, the next ext_rows slots the rows
// extrapolated below the track, the ext_rows after them the rows extrapolated
// above it (Phase III); returns -1 for an unused slot.
__device__ __forceinline__ int amb_per(const KParams& P) { return P.inner_rows + 2 * P.ext_rows; }

__device__ __forceinline__ long amb_slot(const FrameDev& F, const KParams& P, long w, int& f) {
  const int per = amb_per(P);
  f = (int)(w / per);
  const int k = (int)(w % per);
  if (!F.ft_ok[f]) return -1;
  if (k < P.inner_rows) return inner_station(F, P, f, k) ? (long)f * F.nslot + k : -1;
  const int e = k - P.inner_rows;
  if (e < P.ext_rows) return e < F.ft_next[f] ? (long)f * F.nslot + kMaxInner + e : -1;
  const int eo = e - P.ext_rows;
  return eo < F.ft_nout[f] ? (long)f * F.nslot + kMaxInner + P.ext_rows + eo : -1;
}

__global__ void k_amb_bid(FrameDev F, KParams P, int round) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const long tot = (long)nf * amb_per(P);
  for (long w = (long)blockIdx.x * blockDim.x + threadIdx.x; w < tot;
       w += (long)gridDim.x * blockDim.x) {
    int f;
    const long sk = amb_slot(F, P, w, f);
    if (sk < 0) continue;
    if (F.ft_assigned[sk] >= 0 || F.ft_ncand[sk] <= round) continue;
    const int c = F.ft_cand[sk * kMaxCand + round];
    if (F.taken[c]) continue;
    atomicMin(&F.bid[c], pack_chi_key(F.ft_cchi[sk * kMaxCand + round], F.ft_key[f]));
  }
}

__global__ void k_amb_resolve(FrameDev F, KParams P, int round) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const long tot = (long)nf * amb_per(P);
  for (long w = (long)blockIdx.x * blockDim.x + threadIdx.x; w < tot;
       w += (long)gridDim.x * blockDim.x) {
    int f;
    const long sk = amb_slot(F, P, w, f);
    if (sk < 0) continue;
    F.ft_newly[sk] = 0;
    if (F.ft_assigned[sk] >= 0 || F.ft_ncand[sk] <= round) continue;
    const int c = F.ft_cand[sk * kMaxCand + round];
    if (F.taken[c]) continue;
    if (F.bid[c] == pack_chi_key(F.ft_cchi[sk * kMaxCand + round], F.ft_key[f])) {
      F.ft_assigned[sk] = c;
      F.ft_newly[sk] = 1;
    }
  }
}

__global__ void k_amb_mark(FrameDev F, KParams P, int round) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const long tot = (long)nf * amb_per(P);
  for (long w = (long)blockIdx.x * blockDim.x + threadIdx.x; w < tot;
       w += (long)gridDim.x * blockDim.x) {
    int f;
    const long sk = amb_slot(F, P, w, f);
    if (sk < 0) continue;
    if (F.ft_ncand[sk] <= round) continue;
    const int c = F.ft_cand[sk * kMaxCand + round];
    if (F.ft_newly[sk]) F.taken[c] = 1;
    F.bid[c] = ~0ull;
  }
}

// Iteration 3: inward with the surviving and re-attached clusters, simple cut.
template <bool kMap, int kPart>
__global__ void __launch_bounds__(256, kPart == 1 ? 3 : 2)
    k_fit3(FrameDev F, KParams P, MapDev M) {
  if (!kMap) M.on = 0;  // (the map evaluation is compiled out)
  __shared__ float rx[kMaxRows];
  for (int r = threadIdx.x; r < P.n_rows; r += blockDim.x) rx[r] = F.row_x[r];
  __syncthreads();
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  const int nL = min(F.cnt->n_loopers, nf);
  for (int q = fit_next_part<kPart>(F.cnt, kQFit3, kQFit3N, nL, nf); q < nf;
       q = fit_next_part<kPart>(F.cnt, kQFit3, kQFit3N, nL, nf)) {
    const int f = F.ft_order[q];
    const bool lp = fit_looper<kPart>(F, f);  // FP64 updates (low-pT looper)
    F.ft_n[f] = 0;
    if (!F.ft_ok[f]) continue;
    const int ns = F.ft_nst[f];
    const int* SC = F.ft_st_cl + (long)f * kMaxRows;
    const uint16_t* SR = F.ft_st_rs + (long)f * kMaxRows;
    const uint8_t* flag = F.ft_flag + (long)f * kMaxRows;
    int* used = F.ft_used + (long)f * kMaxRows;
    const float z0 = F.ft_z0[f];
    const float zsh = F.ft_zsh[f];
    const int zside = shift_side(F, f);
    Trk<float> s2;
    const float* e2 = F.ft_end2 + (long)f * kStateF;
    get_state(e2, s2);
    Lin L;
    lin_start(L, s2, SR[ns - 1] / NR, P);
    float chi2 = 0.0f;
    int n = 0;
    Trk<float> out = L.t;
    int out_sec = L.sector;
    bool have = false;
    // Phase III outward rows: each assigned cluster is tested and filtered
    // against a forward extrapolation of the iteration-2 end state (its own
    // covariance), so that it joins the track without moving the fit of the
    // stations; in the list the outward clusters precede the stations
    const int nout = P.ext_rows > 0 ? F.ft_nout[f] : 0;
    if (nout > 0) {
      const int rsl = SR[ns - 1];
      const int secl = rsl / NR, rl = rsl % NR;
      Lin E;
      E.t = s2;
#pragma unroll
      for (int i = 0; i < 5; ++i) E.r[i] = s2.p[i];
      E.sector = secl;
      const long o0 = (long)f * F.nslot + kMaxInner + P.ext_rows;
      const uint16_t* xs = F.ft_ext_sec + (long)f * 2 * P.ext_rows + P.ext_rows;
      for (int e = 0; e < nout; ++e) {
        const int sx = xs[e];
        if (!lin_goto(E, sx, rx[rl + 1 + e], P)) break;
        const int c = F.ft_assigned[o0 + e];
        if (c < 0) continue;
        const float2 pc = F.syz[c];
        float my, mz;
        if (!corrected(M, P, sx, E.t.x, pc.x, track_z(pc.y, sx, zside, zsh, P), z0, E.r, my,
                       mz))
          continue;
        const Resid R = residual(E.t, my, mz, P);
        if (R.chi2 > P.final_chi2) continue;
        chi2 = chi2 + R.chi2;
        update_as(E.t, R, lp);
        used[n] = c;
        ++n;
      }
      for (int i = 0, j = n - 1; i < j; ++i, --j) {  // outermost first
        const int u = used[i];
        used[i] = used[j];
        used[j] = u;
      }
    }
    // the stations inward, then the rows extrapolated below the innermost one
    const int next = P.ext_rows > 0 ? F.ft_next[f] : 0;
    const int rs0 = SR[0];
    for (int k = ns - 1; k >= -next; --k) {
      // the station's cluster is requested before the station change (it
      // does not depend on the state); inner stations hold at most
      // inner_rows <= kMaxInner entries, as rows increase along a track
      int sec, row, c;
      if (k >= 0) {
        const int rs = SR[k];
        sec = rs / NR;
        row = rs % NR;
        const bool inner = row < P.inner_rows;
        c = inner ? F.ft_assigned[(long)f * F.nslot + k] : (flag[k] ? -1 : SC[k]);
      } else {
        sec = F.ft_ext_sec[(long)f * 2 * P.ext_rows - 1 - k];
        row = rs0 % NR + k;
        c = F.ft_assigned[(long)f * F.nslot + kMaxInner - 1 - k];
      }
      float cy = 0.0f, cz = 0.0f;
      if (c >= 0) {
        const float2 pc = F.syz[c];
        cy = pc.x;
        cz = track_z(pc.y, sec, zside, zsh, P);
      }
      if (k != ns - 1 && !lin_goto(L, sec, rx[row], P)) break;
      if (c < 0) continue;
      float my, mz;
      if (!corrected(M, P, sec, L.t.x, cy, cz, z0, L.r, my, mz)) continue;
      const Resid R = residual(L.t, my, mz, P);
      if (R.chi2 > P.final_chi2) continue;
      chi2 = chi2 + R.chi2;
      update_as(L.t, R, lp);
      used[n] = c;
      ++n;
      out = L.t;
      out_sec = L.sector;
      have = true;
    }
    F.ft_n[f] = have ? n : 0;
    F.ft_chi2[f] = chi2;
    put_state(F.ft_out + (long)f * kStateF, out, out_sec);
  }
}

// ------------------------------------------------------------ a11 outputs
__device__ __forceinline__ int out_flag(const FrameDev& F, const KParams& P, int f, int nf) {
  return (f < nf && F.ft_ok[f] && F.ft_n[f] >= P.min_hits) ? 1 : 0;
}

__global__ void k_out_count(FrameDev F, KParams P) {
  __shared__ int sh[32];
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int fl = F.cnt->err ? 0 : out_flag(F, P, f, nf);
  const int v = fl ? F.ft_n[f] : 0;
  int tot_t, tot_r;
  block_exscan(fl, sh, &tot_t);
  block_exscan(v, sh, &tot_r);
  if (threadIdx.x == 0) {
    F.scan_tmp[2 * blockIdx.x] = tot_t;
    F.scan_tmp[2 * blockIdx.x + 1] = tot_r;
  }
}

// Exclusive scan of the interleaved (tracks, refs) block partials.
__global__ void k_out_scan(FrameDev F, int nparts) {
  __shared__ int sh[32];
  __shared__ int ct, cr;
  if (threadIdx.x == 0) { ct = 0; cr = 0; }
  __syncthreads();
  for (int base = 0; base < nparts; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int vt = i < nparts ? F.scan_tmp[2 * i] : 0;
    const int vr = i < nparts ? F.scan_tmp[2 * i + 1] : 0;
    int tt, tr;
    const int et = block_exscan(vt, sh, &tt);
    const int er = block_exscan(vr, sh, &tr);
    if (i < nparts) {
      F.scan_tmp[2 * i] = ct + et;
      F.scan_tmp[2 * i + 1] = cr + er;
    }
    __syncthreads();
    if (threadIdx.x == 0) { ct += tt; cr += tr; }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F.cnt->n_refs = cr;
    F.cnt->n_out = ct;
  }
}

__global__ void k_out_write(FrameDev F, KParams P) {
  __shared__ int sh[32];
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  const int fl = F.cnt->err ? 0 : out_flag(F, P, f, nf);
  const int v = fl ? F.ft_n[f] : 0;
  int tt, tr;
  const int et = block_exscan(fl, sh, &tt);
  const int er = block_exscan(v, sh, &tr);
  int off = 0, key = 0, fits = 0;
  if (!fl) {
    if (f < nf) F.ft_outidx[f] = -1;
  } else {
    const int t = F.scan_tmp[2 * blockIdx.x] + et;
    off = F.scan_tmp[2 * blockIdx.x + 1] + er;
    F.ft_outidx[f] = t;
    const float* o = F.ft_out + (long)f * kStateF;
    for (int i = 0; i < 5; ++i) F.out_par[(long)t * 5 + i] = o[i];
    for (int i = 0; i < 15; ++i) F.out_cov[(long)t * 15 + i] = o[5 + i];
    F.out_x[t] = o[20];
    F.out_zsh[t] = F.ft_zsh[f];
    F.out_sector[t] = __float_as_int(o[21]);
    F.out_chi2[t] = F.ft_chi2[f];
    F.out_ndf[t] = 2 * v - 5;
    F.out_ncl[t] = v;
    key = F.ft_key[f];
    F.out_key[t] = key;
    F.out_offset[t] = off;
    fits = (long)off + v <= F.cap_refs;
    if (!fits) atomicOr(&F.cnt->err, kErrCapRefs);
  }
  // Cluster lists: the warp takes its lanes' tracks one by one, its lanes
  // over the track's clusters (the used list read innermost first, all loads
  // issued before the ids they address), writing the input ids 32 at a time
  // and lowering their attachment keys.
  constexpr int kChunks = (kMaxRows + 31) / 32;
  const int lane = threadIdx.x & 31;
  for (unsigned todo = __ballot_sync(0xffffffffu, fl != 0); todo; todo &= todo - 1) {
    const int j = __ffs(todo) - 1;
    const int fj = f - lane + j;
    const int nj = __shfl_sync(0xffffffffu, v, j);
    const int oj = __shfl_sync(0xffffffffu, off, j);
    const int kj = __shfl_sync(0xffffffffu, key, j);
    const int fitj = __shfl_sync(0xffffffffu, fits, j);
    const int* used = F.ft_used + (long)fj * kMaxRows;
    int u[kChunks], id[kChunks];
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      const int q = lane + 32 * c;
      u[c] = q < nj ? used[nj - 1 - q] : -1;
    }
#pragma unroll
    for (int c = 0; c < kChunks; ++c) id[c] = u[c] >= 0 ? F.sid[u[c]] : -1;
#pragma unroll
    for (int c = 0; c < kChunks; ++c) {
      if (id[c] < 0) continue;
      if (fitj) F.out_ids[oj + lane + 32 * c] = id[c];
      atomicMin(&F.attach_key[id[c]], kj);
    }
  }
}

// Attachment: every cluster goes to the track with the smallest key among
// those that use it.  One warp per 32 consecutive fit tracks, taken one by
// one with the lanes over the track's clusters.
__global__ void k_out_attach(FrameDev F, KParams P) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  if (F.cnt->err) return;
  constexpr int kChunks = (kMaxRows + 31) / 32;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int f0 = 32 * (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)); f0 < nf;
       f0 += 32 * nw) {
    const int f = f0 + lane;
    int t = -1, n = 0, key = 0, off = 0;
    if (f < nf) {
      t = F.ft_outidx[f];
      if (t >= 0) {
        n = F.ft_n[f];
        key = F.ft_key[f];
        off = F.out_offset[t];
        if (t == F.cnt->n_out - 1) F.out_offset[t + 1] = F.cnt->n_refs;
      }
    }
    for (unsigned todo = __ballot_sync(0xffffffffu, t >= 0); todo; todo &= todo - 1) {
      const int j = __ffs(todo) - 1;
      const int tj = __shfl_sync(0xffffffffu, t, j);
      const int nj = __shfl_sync(0xffffffffu, n, j);
      const int kj = __shfl_sync(0xffffffffu, key, j);
      const int oj = __shfl_sync(0xffffffffu, off, j);
      const int* ids = F.out_ids + oj;
      int id[kChunks], ak[kChunks];
#pragma unroll
      for (int c = 0; c < kChunks; ++c) {
        const int q = lane + 32 * c;
        id[c] = q < nj ? ids[q] : -1;
      }
#pragma unroll
      for (int c = 0; c < kChunks; ++c) ak[c] = id[c] >= 0 ? F.attach_key[id[c]] : 0;
#pragma unroll
      for (int c = 0; c < kChunks; ++c)
        if (id[c] >= 0 && ak[c] == kj) F.attach[id[c]] = tj;
    }
  }
}

// ------------------------------------------- a12 refit with fixed clusters
// Tracks merged across the central electrode carry the shift of their far
// side (in_zsh): zsh and the side whose clusters take it (zside, -1: none;
// the other side than the innermost cluster's), for track_z.
__device__ __forceinline__ void refit_shift(const RefitDev& R, const KParams& P, int t,
                                            float& zsh, int& zside) {
  zsh = R.in_zsh ? R.in_zsh[t] : 0.0f;
  zside = zsh != 0.0f ? 1 - ((R.sector[R.ids[R.offset[t]]] / P.n_phi) & 1) : -1;
}
__device__ __forceinline__ void save_ckpt(float* d, const Lin& L) {
#pragma unroll
  for (int i = 0; i < 5; ++i) d[i] = L.t.p[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) d[5 + i] = L.t.c[i];
#pragma unroll
  for (int i = 0; i < 5; ++i) d[20 + i] = L.r[i];
  d[25] = L.t.x;
  d[26] = __int_as_float(L.sector);
}

__device__ __forceinline__ void load_ckpt(const float* d, Lin& L) {
#pragma unroll
  for (int i = 0; i < 5; ++i) L.t.p[i] = d[i];
#pragma unroll
  for (int i = 0; i < 15; ++i) L.t.c[i] = d[5 + i];
#pragma unroll
  for (int i = 0; i < 5; ++i) L.r[i] = d[20 + i];
  L.t.x = d[25];
  L.sector = __float_as_int(d[26]);
}

__device__ __forceinline__ void lin_start2(Lin& L, const Trk<float>& s, const float* ref,
                                           int sector, const KParams& P) {
  L.t = s;
  reset_cov(L.t.c, P);
#pragma unroll
  for (int i = 0; i < 5; ++i) L.r[i] = ref[i];
  L.sector = sector;
}

// Forward refit (see the oracle's definition): extended-Kalman start pass on
// uncorrected clusters, then iterations 1-3 with checkpoints of the filter
// (state, covariance, reference) every kCkptStride stations.
__global__ void __launch_bounds__(128) k_refit(RefitDev R, KParams P, int* steps3) {
  const MapDev M = R.map;
  const int half = P.n_phi;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < R.n_tracks;
       t += gridDim.x * blockDim.x) {
    R.ok[t] = 0;
    R.nused[t] = 0;
    R.chi2[t] = 0.0f;
    steps3[t] = 0;
    const int o0 = R.offset[t], ns = R.offset[t + 1] - o0;
    if (ns < 1 || ns > kMaxRows) continue;
    const int* ids = R.ids + o0;
    float ip[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) ip[i] = R.in_par[(long)t * 5 + i];
    const float inx = R.in_x[t];
    const float z0 = ip[1] - ip[3] * sqrtf(inx * inx + ip[0] * ip[0]);
    R.z0[t] = z0;
    float* zr = R.zref + o0;  // each cluster's z in the innermost side's frame
    {
      float zsh;
      int zside;
      refit_shift(R, P, t, zsh, zside);
      for (int k = 0; k < ns; ++k) zr[k] = track_z(R.z[ids[k]], R.sector[ids[k]], zside, zsh, P);
    }
    Trk<float> t0;
#pragma unroll
    for (int i = 0; i < 5; ++i) t0.p[i] = ip[i];
    t0.x = inx;
    reset_cov(t0.c, P);
    int sec = R.in_sector[t];
    bool ok = true;
    for (int k = 0; k < ns && ok; ++k) {
      const int c = ids[k];
      const int s = R.sector[c];
      if (s != sec) {
        const int ds = ((s % half) - (sec % half) + half) % half;
        // ds == 0: the same azimuthal sector across the central electrode
        if ((ds != 0 && ds != 1 && ds != half - 1) ||
            (ds != 0 && !rotate(t0, ds == 1 ? 1 : -1, P, P.fit_max_snp))) {
          ok = false;
          break;
        }
        sec = s;
      }
      if (!propagate(t0, R.row_x[R.row[c]], P, P.fit_max_snp)) { ok = false; break; }
      update(t0, residual(t0, R.y[c], zr[k], P));
    }
    if (!ok) continue;
    float* store = R.store + (long)t * kMaxRows * 5;
    float* ck = R.ckpt + (long)t * 3 * kCkptSeg * kCkptF;
    float* ref = R.ref + (long)t * 10;
    uint8_t* flag = R.flag + o0;
    uint8_t* acc = R.acc + o0;
    Lin L;
    lin_start(L, t0, R.sector[ids[ns - 1]], P);
    for (int j = 0; j < ns && ok; ++j) {  // iteration 1: inward
      const int k = ns - 1 - j, c = ids[k];
      if (j % kCkptStride == 0) save_ckpt(ck + (0 * kCkptSeg + j / kCkptStride) * kCkptF, L);
      if (j != 0 && !lin_goto(L, R.sector[c], R.row_x[R.row[c]], P)) { ok = false; break; }
      float* sv = store + k * 5;
      sv[0] = L.t.p[0]; sv[1] = L.t.p[1]; sv[2] = L.t.c[0]; sv[3] = L.t.c[1]; sv[4] = L.t.c[2];
      float my, mz;
      if (!corrected(M, P, R.sector[c], L.t.x, R.y[c], zr[k], z0, L.r, my, mz)) {
        ok = false;
        break;
      }
      fit_update(L.t, residual(L.t, my, mz, P), P);
    }
    if (!ok) continue;
    {
      const Trk<float> s1 = L.t;
      if (!R.freeze)
        for (int i = 0; i < 5; ++i) ref[i] = s1.p[i];
      lin_start2(L, s1, ref, R.sector[ids[0]], P);
    }
    for (int j = 0; j < ns && ok; ++j) {  // iteration 2: outward
      const int k = j, c = ids[k];
      if (j % kCkptStride == 0) save_ckpt(ck + (1 * kCkptSeg + j / kCkptStride) * kCkptF, L);
      if (j != 0 && !lin_goto(L, R.sector[c], R.row_x[R.row[c]], P)) { ok = false; break; }
      const float a[5] = {L.t.p[0], L.t.p[1], L.t.c[0], L.t.c[1], L.t.c[2]};
      const Interp I = interpolate(a, store + k * 5);
      float my, mz;
      if (!corrected(M, P, R.sector[c], L.t.x, R.y[c], zr[k], z0, L.r, my, mz)) {
        ok = false;
        break;
      }
      if (!R.freeze) flag[k] = chi2_interp(I, my, mz, P) > P.int_chi2 ? 1 : 0;
      fit_update(L.t, residual(L.t, my, mz, P), P);
    }
    if (!ok) continue;
    {
      const Trk<float> s2 = L.t;
      if (!R.freeze)
        for (int i = 0; i < 5; ++i) ref[5 + i] = s2.p[i];
      lin_start2(L, s2, ref + 5, R.sector[ids[ns - 1]], P);
    }
    float chi2 = 0.0f;
    int n = 0;
    Trk<float> out = L.t;
    int out_sec = L.sector;
    int j = 0;
    for (; j < ns; ++j) {  // iteration 3: inward
      const int k = ns - 1 - j, c = ids[k];
      if (j % kCkptStride == 0) save_ckpt(ck + (2 * kCkptSeg + j / kCkptStride) * kCkptF, L);
      if (j != 0 && !lin_goto(L, R.sector[c], R.row_x[R.row[c]], P)) break;
      if (flag[k]) continue;
      float my, mz;
      if (!corrected(M, P, R.sector[c], L.t.x, R.y[c], zr[k], z0, L.r, my, mz))
        continue;
      const Resid Rs = residual(L.t, my, mz, P);
      const bool accept = R.freeze ? acc[k] != 0 : !(Rs.chi2 > P.final_chi2);
      if (!R.freeze) acc[k] = accept ? 1 : 0;
      if (!accept) continue;
      chi2 = chi2 + Rs.chi2;
      fit_update(L.t, Rs, P);
      ++n;
      out = L.t;
      out_sec = L.sector;
    }
    steps3[t] = j;
    R.ok[t] = n > 0 ? 1 : 0;
    R.nused[t] = n;
    R.chi2[t] = chi2;
    R.ndf[t] = 2 * n - 5;
    R.out_sector[t] = out_sec;
    R.out_x[t] = out.x;
    for (int i = 0; i < 5; ++i) R.out_par[(long)t * 5 + i] = out.p[i];
    for (int i = 0; i < 15; ++i) R.out_cov[(long)t * 15 + i] = out.c[i];
  }
}

// One recomputed forward step of the refit, kept for the reverse sweep.
struct StepRec {
  float j00, j10, j20, j22;
  StepJ F;
  float k0[5], k1[5];
  float w00, w01, w11, r0, r1;
  float gy, gz;  // d(measurement)/d(Dx)
  int bits;      // 1 rotated, 2 propagated, 4 updated, 8 counted in chi2
};

// Replays forward step j of iteration `it` (0: first inward, 1: outward,
// 2: last inward) from the current filter state, with identical arithmetic,
// recording the Jacobians, gain and residual.  Returns false when the
// forward pass stopped at this step.
__device__ __forceinline__ bool replay_step(const RefitDev& R, const KParams& P, int t, int it,
                                            int j, int ns, const int* ids, const float* zr,
                                            float z0, Lin& L, StepRec& S) {
  const int k = it == 1 ? j : ns - 1 - j;
  const int c = ids[k];
  S.bits = 0;
  if (j != 0) {
    bool rot = false;
    float jr[4];
    if (!lin_goto(L, R.sector[c], R.row_x[R.row[c]], P, jr, &rot, &S.F)) return false;
    S.bits |= 2;
    if (rot) {
      S.bits |= 1;
      S.j00 = jr[0]; S.j10 = jr[1]; S.j20 = jr[2]; S.j22 = jr[3];
    }
  }
  if (it == 2 && R.flag[R.offset[t] + k]) return true;
  // measurement with its derivative by the x displacement
  float D[3];
  const float zc = zr[k];
  map_eval(R.map, P, R.sector[c], L.t.x, R.y[c], zc - z0, D);
  float my = R.y[c] + D[1], mz = zc + D[2];
  float snp1 = L.r[2];
  if (D[0] != 0.0f) {
    StepJ st;
    if (!helix_step(L.r, D[0], P, st, P.fit_max_snp)) return it == 2;  // it 2: skipped cluster
    my = my - (st.p0 - L.r[0]);
    mz = mz - (st.p1 - L.r[1]);
    snp1 = st.p2;
  }
  const float csp1 = sqrtf(1.0f - snp1 * snp1);
  S.gy = -snp1 / csp1;
  S.gz = -L.r[3] / csp1;
  const Resid Rs = residual(L.t, my, mz, P);
  if (it == 2) {
    if (!R.acc[R.offset[t] + k]) return true;
    S.bits |= 8;
  }
  const float h0[5] = {L.t.c[0], L.t.c[1], L.t.c[3], L.t.c[6], L.t.c[10]};
  const float h1[5] = {L.t.c[1], L.t.c[2], L.t.c[4], L.t.c[7], L.t.c[11]};
#pragma unroll
  for (int i = 0; i < 5; ++i) {
    S.k0[i] = h0[i] * Rs.w00 + h1[i] * Rs.w01;
    S.k1[i] = h0[i] * Rs.w01 + h1[i] * Rs.w11;
  }
  S.w00 = Rs.w00; S.w01 = Rs.w01; S.w11 = Rs.w11; S.r0 = Rs.r0; S.r1 = Rs.r1;
  S.bits |= 4;
  fit_update(L.t, Rs, P);
  return true;
}

// Adjoint of the refit: d(sum_t w_t chi2_t)/d(map) with references and
// decisions held fixed.  One thread per track: reverse sweep over iterations
// 3, 2, 1, each segment of kCkptStride stations recomputed forward from its
// checkpoint; per-cluster gradients of the (dx, dy, dz) correction are then
// scattered through the 64 spline weights into an FP64 accumulator of the
// block (cross-track reduction in FP64), written per block and summed in a
// fixed order by k_grad_reduce.
__global__ void __launch_bounds__(256) k_refit_adjoint(RefitDev R, KParams P,
                                                       const int* steps3) {
  extern __shared__ double gacc[];
  for (int i = threadIdx.x; i < R.ncoef; i += blockDim.x) gacc[i] = 0.0;
  __syncthreads();
  const MapDev M = R.map;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < R.n_tracks;
       t += gridDim.x * blockDim.x) {
    if (!R.ok[t]) continue;
    const float w = R.dl_dchi2[t];
    const int o0 = R.offset[t], ns = R.offset[t + 1] - o0;
    const int* ids = R.ids + o0;
    const float z0 = R.z0[t];
    const float* zr = R.zref + o0;  // cluster z in the innermost side's frame (k_refit)
    float* dD = R.dD + (long)o0 * 3;
    for (int i = 0; i < 3 * ns; ++i) dD[i] = 0.0f;
    const float* ck = R.ckpt + (long)t * 3 * kCkptSeg * kCkptF;
    float lam[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int it = 2; it >= 0; --it) {
      const int nsteps = it == 2 ? steps3[t] : ns;
      const int nseg = (nsteps + kCkptStride - 1) / kCkptStride;
      for (int sg = nseg - 1; sg >= 0; --sg) {
        const int j0 = sg * kCkptStride, j1 = min(nsteps, j0 + kCkptStride);
        StepRec rec[kCkptStride];
        Lin L;
        load_ckpt(ck + (it * kCkptSeg + sg) * kCkptF, L);
        for (int j = j0; j < j1; ++j)
          replay_step(R, P, t, it, j, ns, ids, zr, z0, L, rec[j - j0]);
        for (int j = j1 - 1; j >= j0; --j) {
          const StepRec& S = rec[j - j0];
          const int k = it == 1 ? j : ns - 1 - j;
          if (S.bits & 4) {
            float g0 = 0.0f, g1 = 0.0f;
            if (S.bits & 8) {
              g0 = 2.0f * w * (S.w00 * S.r0 + S.w01 * S.r1);
              g1 = 2.0f * w * (S.w01 * S.r0 + S.w11 * S.r1);
            }
            float a0 = g0, a1 = g1;
#pragma unroll
            for (int i = 0; i < 5; ++i) {
              a0 += S.k0[i] * lam[i];
              a1 += S.k1[i] * lam[i];
            }
            dD[k * 3 + 0] += S.gy * a0 + S.gz * a1;
            dD[k * 3 + 1] += a0;
            dD[k * 3 + 2] += a1;
            lam[0] -= a0;
            lam[1] -= a1;
          }
          if (S.bits & 2) {
            const float l0 = lam[0], l1 = lam[1], l2 = lam[2];
            lam[2] = l2 + S.F.f02 * l0 + S.F.f12 * l1;
            lam[3] = lam[3] + S.F.f13 * l1;
            lam[4] = lam[4] + S.F.f04 * l0 + S.F.f14 * l1 + S.F.f24 * l2;
          }
          if (S.bits & 1) {
            const float l0 = lam[0], l1 = lam[1], l2 = lam[2];
            lam[0] = S.j00 * l0 + S.j10 * l1 + S.j20 * l2;
            lam[2] = S.j22 * l2;
          }
        }
      }
    }
    // scatter d(loss)/d(correction) through the spline weights
    if (M.on) {
      for (int k = 0; k < ns; ++k) {
        const int c = ids[k];
        const SplinePt sp =
            spline_point(M, P, R.sector[c], R.row_x[R.row[c]], R.y[c], zr[k] - z0);
        int pidx[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) pidx[e] = phi_index(sp.ip, e, M.nphi);
        for (int comp = 0; comp < 3; ++comp) {
          const double g = (double)dD[k * 3 + comp];
          if (g == 0.0) continue;
          for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) {
              const float wzr = sp.wz[a] * sp.wr[b];
              const long base = (((long)comp * M.nz + (sp.iz + a)) * M.nr + (sp.ir + b)) * M.nphi;
#pragma unroll
              for (int e = 0; e < 4; ++e)
                atomicAdd(&gacc[base + pidx[e]], (double)(wzr * sp.wp[e]) * g);
            }
        }
      }
    }
  }
  __syncthreads();
  double* part = R.gpart + (long)blockIdx.x * R.ncoef;
  for (int i = threadIdx.x; i < R.ncoef; i += blockDim.x) part[i] = gacc[i];
}

__global__ void k_grad_reduce(RefitDev R) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < R.ncoef; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < R.gblocks; ++b) s += R.gpart[(long)b * R.ncoef + i];
    R.dl_dmap[i] = (float)s;
  }
}

}  // namespace

int refit_forward(RefitDev& R, const KParams& P, int* steps3, int sms, cudaStream_t s) {
  if (R.n_tracks > 0) k_refit<<<sms * 16, 128, 0, s>>>(R, P, steps3);
  return R.n_tracks > 0 ? 1 : 0;
}

int refit_backward(RefitDev& R, const KParams& P, const int* steps3, int sms, cudaStream_t s) {
  (void)sms;
  const size_t smem = sizeof(double) * (size_t)R.ncoef;
  cudaFuncSetAttribute(k_refit_adjoint, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_refit_adjoint<<<R.gblocks, 256, smem, s>>>(R, P, steps3);
  k_grad_reduce<<<(R.ncoef + 255) / 256, 256, 0, s>>>(R);
  return 2;
}

int stage_sector_refit(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  const int nb_tl = (int)blocks_for(F.cap_tl, kBlock);
  k_acc_count<<<nb_tl, kBlock, 0, s>>>(F);
  k_scan_partials<<<1, 1024, 0, s>>>(F.scan_tmp, nb_tl, &F.cnt->n_tracks);
  k_acc_write<<<nb_tl, kBlock, 0, s>>>(F);
  k_order_scatter<<<sms * 4, kBlock, 0, s>>>(F.st_obucket, F.st_oslot, F.st_ord_cnt,
                                             &F.cnt->n_tracks, F.cap_tl, &F.cnt->err, F.st_order);
  k_st_gather<<<sms * 8, kBlock, 0, s>>>(F, P);
  k_sector_refit<<<persistent_grid(F.lc, kLSectorRefit, sms), F.lc.block[kLSectorRefit], 0, s>>>(F, P);
  return 6;
}

int stage_merge(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  const int nb_tl = (int)blocks_for(F.cap_tl, kBlock);
  k_sector_zrange<<<P.n_sectors, 256, 0, s>>>(F, P);
  k_ie_hist<<<sms * 8, kBlock, 0, s>>>(F, P);
  int k = 2;
  k += scan_exclusive(F.ie_cnt, F.ie_first, (long)P.n_sectors * P.n_rows * kMergeZ + 1,
                      F.scan_tmp, s);
  k_ie_scatter<<<sms * 8, kBlock, 0, s>>>(F);
  {
    const unsigned grid = persistent_grid(F.lc, kLMerge, sms);
    const int blk = F.lc.block[kLMerge];
    switch (F.lc.lanes[kLMerge]) {
      case 32: k_merge_best<32><<<grid, blk, 0, s>>>(F, P); break;
      case 16: k_merge_best<16><<<grid, blk, 0, s>>>(F, P); break;
      case 8: k_merge_best<8><<<grid, blk, 0, s>>>(F, P); break;
      case 4: k_merge_best<4><<<grid, blk, 0, s>>>(F, P); break;
      default: k_merge_best<1><<<grid, blk, 0, s>>>(F, P); break;
    }
  }
  k_merge_link<<<sms * 8, kBlock, 0, s>>>(F);
  if (P.ac_merge) {
    k_cross_best<<<sms * 8, kBlock, 0, s>>>(F, P);
    k_cross_link<<<sms * 8, kBlock, 0, s>>>(F);
    k += 2;
  }
  k_head_count<<<nb_tl, kBlock, 0, s>>>(F);
  k_scan_partials<<<1, 1024, 0, s>>>(F.scan_tmp, nb_tl, &F.cnt->n_merged);
  k_head_write<<<nb_tl, kBlock, 0, s>>>(F, P);
  k_head_check<<<1, 1, 0, s>>>(F);
  const int nb_ft = (int)blocks_for(F.cap_ft, kBlock);
  k_looper_count<<<nb_ft, kBlock, 0, s>>>(F);
  k_scan_partials<<<1, 1024, 0, s>>>(F.scan_tmp, nb_ft, &F.cnt->n_loopers);
  k_looper_write<<<nb_ft, kBlock, 0, s>>>(F);
  return k + 10;
}

int stage_fit12(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  k_fit_stations<<<sms * 8, kBlock, 0, s>>>(F, P);
  const unsigned g = persistent_grid(F.lc, kLFit12, sms);
  const int b = F.lc.block[kLFit12];
  // iterations 1 and 2 keep loopers and other tracks in one launch (split in
  // two parts, as iteration 3 is, they measured slower: 22.4 -> 25.1 ms per
  // batch, the two kinds of track no longer sharing the warps)
  if (F.map.on) {
    k_fit1<true, 0><<<g, b, 0, s>>>(F, P, F.map);
    k_fit2<true, 0><<<g, b, 0, s>>>(F, P, F.map);
    k_inner_cand<true><<<sms * 8, kBlock, 0, s>>>(F, P, F.map);
  } else {
    k_fit1<false, 0><<<g, b, 0, s>>>(F, P, F.map);
    k_fit2<false, 0><<<g, b, 0, s>>>(F, P, F.map);
    k_inner_cand<false><<<sms * 8, kBlock, 0, s>>>(F, P, F.map);
  }
  return 4;  // the station lists, iterations 1 and 2, the candidate search
}

int stage_ambiguity2(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  int k = 0;
  for (int r = 0; r < P.cand_k; ++r) {
    k_amb_bid<<<sms * 8, kBlock, 0, s>>>(F, P, r);
    k_amb_resolve<<<sms * 8, kBlock, 0, s>>>(F, P, r);
    k_amb_mark<<<sms * 8, kBlock, 0, s>>>(F, P, r);
    k += 3;
  }
  return k;
}

int stage_fit3(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  const unsigned g = persistent_grid(F.lc, kLFit3, sms);
  const int b = F.lc.block[kLFit3];
  if (F.map.on) {
    k_fit3<true, 0><<<g, b, 0, s>>>(F, P, F.map);
    return 1;
  }
  k_fit3<false, 1><<<g, b, 0, s>>>(F, P, F.map);
  k_fit3<false, 2><<<g, b, 0, s>>>(F, P, F.map);
  return 2;
}

int stage_output(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  const int nb = (int)blocks_for(F.cap_ft, kBlock);
  k_out_count<<<nb, kBlock, 0, s>>>(F, P);
  k_out_scan<<<1, 1024, 0, s>>>(F, nb);
  k_out_write<<<nb, kBlock, 0, s>>>(F, P);
  k_out_attach<<<sms * 8, kBlock, 0, s>>>(F, P);
  return 4;
}

}  // namespace TPC_NS
}  // namespace tpc
