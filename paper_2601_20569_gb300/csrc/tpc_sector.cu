// Sector tracking kernels (Sec. 2 of the paper): per-row cluster grids,
// cellular-automaton neighbour finding and cleaning, start hits, Kalman
// tracklet construction and ambiguity solving (with the Phase I criterion of
// Sec. 3).  This translation unit is compiled twice: with --fmad=false into
// namespace tpc::strict (bit-identical to the strict CPU evaluation) and with
// FMA contraction into tpc::fast.
#include <cuda_runtime.h>

#include <cstdint>

#include "tpc_kernels.h"
#include "tpc_model.cuh"
#include "tpc_util.cuh"

namespace tpc {
namespace TPC_NS {

namespace {

// ------------------------------------------------------------------ a1 grid
// Input cluster i: position, row and (batch) sector.  A batch call reads each
// frame in place through the frame table: the frame holding i is found by a
// binary search over the frames' offsets, and a sector outside the frame's
// range gives an out-of-range batch sector, which the grid build reports.
struct ClusterIn {
  float y, z;
  int row, sector;
};

__device__ __forceinline__ ClusterIn load_cluster(const FrameDev& F, long i) {
  if (F.nsrc == 0) return {F.y[i], F.z[i], (int)F.row[i], (int)F.sector[i]};
  int lo = 0, hi = F.nsrc - 1;  // the last frame whose offset is <= i
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (F.src[mid].off <= i) lo = mid;
    else hi = mid - 1;
  }
  const FrameSrc& S = F.src[lo];
  const long j = i - S.off;
  const int s = S.sector[j];
  return {S.y[j], S.z[j], (int)S.row[j], s < F.src_nsec ? lo * F.src_nsec + s : 0x7FFFFFFF};
}

__global__ void k_row_stats(FrameDev F, KParams P) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F.n) return;
  const ClusterIn c = load_cluster(F, i);
  const int r = c.row, s = c.sector;
  const float y = c.y, z = c.z;
  if (r >= P.n_rows || s >= P.n_sectors || !isfinite(y) || !isfinite(z)) {
    atomicOr(&F.cnt->err, kErrInput);
    return;
  }
  const int rr = s * P.n_rows + r;
  atomicAdd(&F.row_cnt[rr], 1);
  atomicMin(&F.row_zmin[rr], f2o(z));
  atomicMax(&F.row_zmax[rr], f2o(z));
}

// The same statistics with each block's share of them gathered in shared
// memory first.  A block takes kRowStatsChunk consecutive input clusters,
// which lie (all but a block at a frame boundary) in one frame, and keeps
// count, z minimum and z maximum of that frame's W rows in shared memory;
// clusters of another frame go to global memory directly.  Then one global
// update per row the block has seen.  The statistics are a sum, a minimum and
// a maximum, so the result does not depend on the order of the updates.
constexpr int kRowStatsChunk = 256 * 128;
constexpr int kRowStatsMaxRows = 6144;  // W * 12 bytes of shared memory per block
bool g_row_stats_shared = false;        // the kernel's shared-memory size is allowed

__global__ void __launch_bounds__(256) k_row_stats_sh(FrameDev F, KParams P, int W) {
  extern __shared__ unsigned rs_sh[];
  unsigned* cnt = rs_sh;
  unsigned* zlo = rs_sh + W;
  unsigned* zhi = rs_sh + 2 * W;
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    cnt[w] = 0u;
    zlo[w] = 0xFFFFFFFFu;
    zhi[w] = 0u;
  }
  const long c0 = (long)blockIdx.x * kRowStatsChunk;
  const long c1 = min((long)F.n, c0 + kRowStatsChunk);
  int f0 = 0;  // frame of the chunk's first cluster
  if (F.nsrc > 0) {
    int lo = 0, hi = F.nsrc - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (F.src[mid].off <= c0) lo = mid;
      else hi = mid - 1;
    }
    f0 = lo;
  }
  const long wb = (long)f0 * W;
  __syncthreads();
  for (long i = c0 + threadIdx.x; i < c1; i += blockDim.x) {
    const ClusterIn c = load_cluster(F, i);
    const int r = c.row, s = c.sector;
    const float y = c.y, z = c.z;
    if (r >= P.n_rows || s >= P.n_sectors || !isfinite(y) || !isfinite(z)) {
      atomicOr(&F.cnt->err, kErrInput);
      continue;
    }
    const long rr = (long)s * P.n_rows + r;
    const unsigned zo = f2o(z);
    if (rr >= wb && rr < wb + W) {
      const int w = (int)(rr - wb);
      atomicAdd(&cnt[w], 1u);
      atomicMin(&zlo[w], zo);
      atomicMax(&zhi[w], zo);
    } else {
      atomicAdd(&F.row_cnt[rr], 1);
      atomicMin(&F.row_zmin[rr], zo);
      atomicMax(&F.row_zmax[rr], zo);
    }
  }
  __syncthreads();
  for (int w = threadIdx.x; w < W; w += blockDim.x) {
    const unsigned n = cnt[w];
    if (n == 0u) continue;
    const long rr = wb + w;
    atomicAdd(&F.row_cnt[rr], (int)n);
    atomicMin(&F.row_zmin[rr], zlo[w]);
    atomicMax(&F.row_zmax[rr], zhi[w]);
  }
}

// One block: bin layout of every (sector,row) and the row/bin offsets.
__global__ void k_row_grid(FrameDev F, KParams P) {
  __shared__ int sh[32];
  __shared__ int carry_bins, carry_cl;
  const int nrr = P.n_sectors * P.n_rows;
  if (threadIdx.x == 0) carry_bins = carry_cl = 0;
  __syncthreads();
  for (int base = 0; base < nrr; base += blockDim.x) {
    const int rr = base + threadIdx.x;
    RowGrid g{};
    int nb = 0, cnt = 0;
    if (rr < nrr) {
      const int r = rr % P.n_rows;
      cnt = F.row_cnt[rr];
      const float x = F.row_x[r];
      const float ymax = x * P.tan_half + 0.5f;
      int nZ = 1;
      float zlo = 0.0f, zr = 0.0f;
      if (cnt > 0) {
        zlo = o2f(F.row_zmin[rr]);
        zr = o2f(F.row_zmax[rr]) - zlo;
      }
      // about square bins holding grid_occ clusters each (0.5), at least grid_dy
      // wide in y: the search windows (a few cm in y and in z) then cover few
      // bins and few clusters outside the window
      const float side = sqrtf(2.0f * ymax * fmaxf(zr, 1.0f) * P.grid_occ / (float)max(cnt, 1));
      int nY = (int)(2.0f * ymax / fmaxf(side, P.grid_dy));
      nY = clampi(nY, 1, 64);
      g.nY = nY;
      g.y0 = -ymax;
      g.invDy = (float)nY / (2.0f * ymax);
      if (cnt > 0) {
        const float want = ceilf((float)cnt / ((float)nY * P.grid_occ));
        const float zmax_bins = floorf(zr) + 1.0f;  // bins of at least ~1 cm
        nZ = (int)fminf(fminf(want, zmax_bins), (float)((1 << 20) / nY));
        nZ = max(nZ, 1);
      }
      g.nZ = nZ;
      g.z0 = zlo;
      g.invDz = zr > 0.0f ? (float)nZ / zr : 0.0f;
      g.ncl = cnt;
      nb = nY * nZ;
    }
    int tot_b, tot_c;
    const int ob = block_exscan(nb, sh, &tot_b);
    const int oc = block_exscan(cnt, sh, &tot_c);
    if (rr < nrr) {
      g.bin0 = carry_bins + ob;
      F.rows[rr] = g;
      F.row_first[rr] = carry_cl + oc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      carry_bins += tot_b;
      carry_cl += tot_c;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    F.row_first[nrr] = carry_cl;
    F.cnt->n_bins = carry_bins;
    if (carry_bins > F.cap_bins) atomicOr(&F.cnt->err, kErrCapBins);
  }
}

__global__ void k_bin_hist(FrameDev F, KParams P) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F.n || F.cnt->err) return;
  const ClusterIn c = load_cluster(F, i);
  const int rr = c.sector * P.n_rows + c.row;
  const RowGrid g = F.rows[rr];
  const int iy = bin_of(c.y, g.y0, g.invDy, g.nY);
  const int iz = bin_of(c.z, g.z0, g.invDz, g.nZ);
  const int b = g.bin0 + iz * g.nY + iy;
  F.cl_bin[i] = b;
  F.cl_slot[i] = atomicAdd(&F.bin_cnt[b], 1);
}

__global__ void k_scatter(FrameDev F) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= F.n || F.cnt->err) return;
  const int b = F.cl_bin[i];
  const int pos = F.bin_first[b] + F.cl_slot[i];
  const ClusterIn c = load_cluster(F, i);
  // one 16-byte record per cluster: a single scattered store
  F.srec[pos] = make_int4(__float_as_int(c.y), __float_as_int(c.z), (int)i, b);
}

// First sorted cluster of every bin: one block per row scans the row's bin
// counts from the row's first cluster (the rows' bins and clusters are both
// laid out row after row), so the scan covers the bins in use only.
__global__ void k_row_scan(FrameDev F) {
  __shared__ int sh[32];
  if (F.cnt->err) return;  // the same for the whole block
  const int rr = blockIdx.x;
  const RowGrid g = F.rows[rr];
  const int nb = g.nY * g.nZ;
  int base = F.row_first[rr];
  for (int j0 = 0; j0 < nb; j0 += blockDim.x) {
    const int j = j0 + threadIdx.x;
    const int c = j < nb ? F.bin_cnt[g.bin0 + j] : 0;
    int tot;
    const int ex = block_exscan(c, sh, &tot);
    if (j < nb) F.bin_first[g.bin0 + j] = base + ex;
    base += tot;
  }
  if (rr == gridDim.x - 1 && threadIdx.x == 0) F.bin_first[g.bin0 + nb] = base;
}

// (sector, row) of every sorted cluster: a row's clusters are contiguous in
// the sorted order, so one block per row writes its range in order (rather
// than the scatter adding another scattered store per cluster).
__global__ void k_row_fill(FrameDev F) {
  if (F.cnt->err) return;
  const int rr = blockIdx.x;
  const int lo = F.row_first[rr], hi = F.row_first[rr + 1];
  for (int k = lo + threadIdx.x; k < hi; k += blockDim.x) F.srow[k] = (uint16_t)rr;
}

// Order the clusters of each bin by input id (deterministic layout) and
// split the records into the sorted (y, z) and id arrays: one thread per
// sorted cluster, whose place in its bin is the number of the bin's clusters
// with a smaller id (bins hold about one cluster, so the work follows the
// clusters, not the bins).
__global__ void k_bin_sort(FrameDev F) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= F.n || F.cnt->err) return;
  const int4 v = F.srec[k];
  const int lo = F.bin_first[v.w], hi = F.bin_first[v.w + 1];
  int pos = lo;
  if (hi - lo > 1) {
    if (hi - lo > kMaxBinOcc) {
      atomicOr(&F.cnt->err, kErrDense);
      return;
    }
    for (int j = lo; j < hi; ++j) pos += F.srec[j].z < v.z ? 1 : 0;
  }
  F.syz[pos] = make_float2(__int_as_float(v.x), __int_as_float(v.y));
  F.sid[pos] = v.z;
}

// ------------------------------------------------------------- a2 neighbours
// Clusters of the row below inside the window are listed once (up to
// kLinkList of them; a denser window falls back to rescanning the grid for
// every upper candidate), then every upper candidate inside the window is
// paired with the list.  The best pair minimises the distance of the middle
// cluster to the straight line through the pair; ties go to the smaller
// input id of the upper, then of the lower cluster, so the result does not
// depend on the visiting order.  In the iterations after the first (kLeft)
// the clusters taken by earlier iterations neither link nor are linked to.
constexpr int kLinkList = 8;

// The best (lower, upper) pair of sorted cluster k (-1, -1: none).
template <bool kLeft>
__device__ __forceinline__ void links_one(const FrameDev& F, const KParams& P, long k, int& bu,
                                          int& bd) {
  const int rr = F.srow[k];
  const int r = rr % P.n_rows;
  bu = -1;
  bd = -1;
  if (r >= 1 && r <= P.n_rows - 2 && !(kLeft && F.sused[k])) {
    const float2 pc = F.syz[k];
    const float yc = pc.x, zc = pc.y;
    const float xd = F.row_x[r - 1], xc = F.row_x[r], xu = F.row_x[r + 1];
    const float f = (xc - xd) / (xu - xd);
    const RowGrid gu = F.rows[rr + 1], gd = F.rows[rr - 1];
    const float m = 0.01f;
    const float ylo = yc - P.link_wy - m, yhi = yc + P.link_wy + m;
    const float zlo = zc - P.link_wz - m, zhi = zc + P.link_wz + m;
    int dl[kLinkList];
    int nd = 0;
    bool dense = false;
    for_window(F.bin_first, gd, ylo, yhi, zlo, zhi, [&](int d) {
      if (kLeft && F.sused[d]) return;
      const float2 pd = F.syz[d];
      const float yd = pd.x, zd = pd.y;
      if (!(fabsf(yd - yc) <= P.link_wy && fabsf(zd - zc) <= P.link_wz)) return;
      if (nd < kLinkList)
        dl[nd++] = d;
      else
        dense = true;
    });
    float best = 0.0f;
    int buid = 0, bdid = 0;
    auto pair = [&](int u, float yu, float zu, int uid, int d) {
      const float2 pd = F.syz[d];
      const float yd = pd.x, zd = pd.y;
      const float yp = yd + (yu - yd) * f;
      const float zp = zd + (zu - zd) * f;
      const float ey = yp - yc, ez = zp - zc;
      const float d2 = ey * ey + ez * ez;
      if (!(d2 < P.link_chi2)) return;
      const int did = F.sid[d];
      if (bu < 0 || d2 < best || (d2 == best && (uid < buid || (uid == buid && did < bdid)))) {
        best = d2;
        bu = u;
        bd = d;
        buid = uid;
        bdid = did;
      }
    };
    if (nd > 0)
      for_window(F.bin_first, gu, ylo, yhi, zlo, zhi, [&](int u) {
        if (kLeft && F.sused[u]) return;
        const float2 pu = F.syz[u];
        const float yu = pu.x, zu = pu.y;
        if (!(fabsf(yu - yc) <= P.link_wy && fabsf(zu - zc) <= P.link_wz)) return;
        const int uid = F.sid[u];
        if (!dense) {
          for (int j = 0; j < nd; ++j) pair(u, yu, zu, uid, dl[j]);
        } else {
          for_window(F.bin_first, gd, ylo, yhi, zlo, zhi, [&](int d) {
            if (kLeft && F.sused[d]) return;
            const float2 pd = F.syz[d];
            const float yd = pd.x, zd = pd.y;
            if (fabsf(yd - yc) <= P.link_wy && fabsf(zd - zc) <= P.link_wz)
              pair(u, yu, zu, uid, d);
          });
        }
      });
  }
}

template <bool kLeft>
__global__ void k_links(FrameDev F, KParams P) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= F.n || F.cnt->err) return;
  int bu, bd;
  links_one<kLeft>(F, P, k, bu, bd);
  F.lup[k] = bu;
  F.ldn[k] = bd;
}

// The same search with a group of G lanes per cluster (G = 4 or 8).  The z
// strips of the window on the row below and the row above (each a contiguous
// run of sorted clusters) are dealt out to the lanes, their sizes summed by a
// group scan and their clusters tested G at a time; those inside the window
// go to per-cluster lists in shared memory.  Then the (lower, upper) pairs
// are dealt out to the lanes and the best one, by (distance, upper id, lower
// id), is found by shuffles.  A window holding more than kGroupList clusters
// on a row falls back to the one-lane search.  The result is the same.
constexpr int kGroupList = 8;

template <int G, bool kLeft>
__global__ void __launch_bounds__(256, 4) k_links_g(FrameDev F, KParams P) {
  constexpr int kGroups = 256 / G;
  __shared__ int sD[kGroups][kGroupList];
  __shared__ int sU[kGroups][kGroupList];
  const int lane = threadIdx.x & 31;
  const int gl = lane & (G - 1);
  const int grp = threadIdx.x / G;
  const unsigned gmask = ((1u << G) - 1u) << (lane & ~(G - 1));
  const unsigned below = ((1u << lane) - 1u) & gmask;
  const long k = (long)blockIdx.x * kGroups + grp;
  if (k >= F.n || F.cnt->err) return;  // the whole group
  const int NR = P.n_rows;
  const int rr = F.srow[k];
  const int r = rr % NR;
  int bu = -1, bd = -1;
  if (r >= 1 && r <= NR - 2 && !(kLeft && F.sused[k])) {
    const float2 pc = F.syz[k];
    const float yc = pc.x, zc = pc.y;
    const float xd = F.row_x[r - 1], xc = F.row_x[r], xu = F.row_x[r + 1];
    const float f = (xc - xd) / (xu - xd);
    const RowGrid gu = F.rows[rr + 1], gd = F.rows[rr - 1];
    const float m = 0.01f;
    const float ylo = yc - P.link_wy - m, yhi = yc + P.link_wy + m;
    const float zlo = zc - P.link_wz - m, zhi = zc + P.link_wz + m;
    // the window's z strips on the two rows: [0, nzd) below, [nzd, nzd + nzu) above
    int iyd0 = 0, iyd1 = -1, izd0 = 0, nzd = 0, iyu0 = 0, iyu1 = -1, izu0 = 0, nzu = 0;
    if (gd.ncl > 0) {
      iyd0 = bin_of(ylo, gd.y0, gd.invDy, gd.nY);
      iyd1 = bin_of(yhi, gd.y0, gd.invDy, gd.nY);
      izd0 = bin_of(zlo, gd.z0, gd.invDz, gd.nZ);
      nzd = bin_of(zhi, gd.z0, gd.invDz, gd.nZ) - izd0 + 1;
    }
    if (gu.ncl > 0) {
      iyu0 = bin_of(ylo, gu.y0, gu.invDy, gu.nY);
      iyu1 = bin_of(yhi, gu.y0, gu.invDy, gu.nY);
      izu0 = bin_of(zlo, gu.z0, gu.invDz, gu.nZ);
      nzu = bin_of(zhi, gu.z0, gu.invDz, gu.nZ) - izu0 + 1;
    }
    const int ns = nzd + nzu;
    int nd = 0, nu = 0;
    for (int s0 = 0; s0 < ns; s0 += G) {
      const int sx = s0 + gl;
      int lo = 0, cnt = 0, up = 0;
      if (sx < ns) {
        up = sx >= nzd;
        const RowGrid& g = up ? gu : gd;
        const int b = g.bin0 + (up ? izu0 + sx - nzd : izd0 + sx) * g.nY;
        lo = F.bin_first[b + (up ? iyu0 : iyd0)];
        cnt = F.bin_first[b + (up ? iyu1 : iyd1) + 1] - lo;
      }
      int inc = cnt;
#pragma unroll
      for (int o = 1; o < G; o <<= 1) {
        const int v = __shfl_up_sync(gmask, inc, o, G);
        if (gl >= o) inc += v;
      }
      const int total = __shfl_sync(gmask, inc, G - 1, G);
      for (int c0 = 0; c0 < total; c0 += G) {
        const int c = c0 + gl;
        int L = 0;
#pragma unroll
        for (int st = G / 2; st >= 1; st >>= 1) {
          const int v = __shfl_sync(gmask, inc, L + st - 1, G);
          if (v <= c) L += st;
        }
        const int excl = __shfl_sync(gmask, inc - cnt, L, G);
        const int lo_l = __shfl_sync(gmask, lo, L, G);
        const int up_l = __shfl_sync(gmask, up, L, G);
        int cand = -1;
        bool pass = false;
        if (c < total) {
          cand = lo_l + (c - excl);
          if (!(kLeft && F.sused[cand])) {
            const float2 pk = F.syz[cand];
            pass = fabsf(pk.x - yc) <= P.link_wy && fabsf(pk.y - zc) <= P.link_wz;
          }
        }
        const unsigned bd_ = __ballot_sync(gmask, pass && !up_l) & gmask;
        const unsigned bu_ = __ballot_sync(gmask, pass && up_l) & gmask;
        if (pass) {
          if (up_l) {
            const int q = nu + __popc(bu_ & below);
            if (q < kGroupList) sU[grp][q] = cand;
          } else {
            const int q = nd + __popc(bd_ & below);
            if (q < kGroupList) sD[grp][q] = cand;
          }
        }
        nd += __popc(bd_);
        nu += __popc(bu_);
      }
    }
    __syncwarp(gmask);
    if (nd > kGroupList || nu > kGroupList) {
      // dense window: the one-lane search, on the group's first lane
      if (gl == 0) links_one<kLeft>(F, P, k, bu, bd);
    } else {
      float best = 0.0f;
      int buid = 0, bdid = 0;
      const int np = nd * nu;
      for (int p = gl; p < np; p += G) {
        const int d = sD[grp][p / nu], u = sU[grp][p % nu];
        const float2 pd = F.syz[d], pu = F.syz[u];
        const float yp = pd.x + (pu.x - pd.x) * f;
        const float zp = pd.y + (pu.y - pd.y) * f;
        const float ey = yp - yc, ez = zp - zc;
        const float d2 = ey * ey + ez * ez;
        if (!(d2 < P.link_chi2)) continue;
        const int uid = F.sid[u], did = F.sid[d];
        if (bu < 0 || d2 < best || (d2 == best && (uid < buid || (uid == buid && did < bdid)))) {
          best = d2;
          bu = u;
          bd = d;
          buid = uid;
          bdid = did;
        }
      }
#pragma unroll
      for (int o = G / 2; o >= 1; o >>= 1) {
        const float ob = __shfl_xor_sync(gmask, best, o, G);
        const int obu = __shfl_xor_sync(gmask, bu, o, G);
        const int obd = __shfl_xor_sync(gmask, bd, o, G);
        const int ouid = __shfl_xor_sync(gmask, buid, o, G);
        const int odid = __shfl_xor_sync(gmask, bdid, o, G);
        if (obu >= 0 && (bu < 0 || ob < best ||
                         (ob == best && (ouid < buid || (ouid == buid && odid < bdid))))) {
          best = ob;
          bu = obu;
          bd = obd;
          buid = ouid;
          bdid = odid;
        }
      }
    }
  }
  if (gl == 0) {
    F.lup[k] = bu;
    F.ldn[k] = bd;
  }
}

// The same search with the candidates staged per warp.  A warp takes 32
// consecutive sorted clusters; when they lie on one pad row (the common case:
// a row holds hundreds to thousands of clusters), the clusters of the row
// below that any of the 32 windows can reach lie in one run of z strips, and
// so in one contiguous run of the sorted order (a row's bins are laid out z
// strip by z strip, all y bins of a strip together); likewise on the row
// above.  The warp copies both runs into shared memory with coalesced loads,
// and every lane tests all staged clusters against its own window: the same
// sequence of tests on all lanes, so the warp issues them without the
// divergence of the per-lane bin walk.  The clusters inside a lane's window
// are kept as bit masks and paired as in links_one.  The runs hold every
// cluster the lane's own bin walk would visit (the bin index is monotone in
// z), the window test is the same, and the best pair is a minimum under a
// total order (distance, upper id, lower id): the links are those of
// links_one, bit for bit.  A warp whose clusters span two rows, or whose runs
// exceed kStageMax clusters, takes links_one.
constexpr int kStageMax = 96;  // staged clusters per row and warp (three mask words)
constexpr int kStageWarps = 8;  // warps per block

template <bool kLeft>
__global__ void __launch_bounds__(32 * kStageWarps, 4) k_links_w(FrameDev F, KParams P) {
  __shared__ float2 sP[kStageWarps][2][kStageMax];
  __shared__ int sI[kStageWarps][2][kStageMax];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long k0 = ((long)blockIdx.x * kStageWarps + wib) * 32;
  if (k0 >= F.n || F.cnt->err) return;  // the whole warp
  const long k = k0 + lane;
  const bool valid = k < F.n;
  const int NR = P.n_rows;
  const int rr = valid ? (int)F.srow[k] : -1;
  const int rr0 = __shfl_sync(0xffffffffu, rr, 0);
  int bu = -1, bd = -1;
  const bool one_row = __all_sync(0xffffffffu, !valid || rr == rr0);
  const int r = rr0 % NR;
  if (!one_row) {
    if (valid) links_one<kLeft>(F, P, k, bu, bd);
  } else if (r >= 1 && r <= NR - 2) {
    float2 pc = make_float2(0.0f, 0.0f);
    bool live = valid;
    if (valid) {
      pc = F.syz[k];
      if (kLeft && F.sused[k]) live = false;
    }
    const float yc = pc.x, zc = pc.y;
    // z range reached by the warp's windows
    float zmin = live ? zc : __int_as_float(0x7f800000);
    float zmax = live ? zc : -__int_as_float(0x7f800000);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) {
      zmin = fminf(zmin, __shfl_xor_sync(0xffffffffu, zmin, o));
      zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    }
    const float m = 0.01f;
    const float zlo = zmin - P.link_wz - m, zhi = zmax + P.link_wz + m;
    int lo[2] = {0, 0}, cnt[2] = {0, 0};
    if (zlo <= zhi) {  // false when no lane is live
#pragma unroll
      for (int sd = 0; sd < 2; ++sd) {
        const RowGrid g = F.rows[sd == 0 ? rr0 - 1 : rr0 + 1];
        if (g.ncl > 0) {
          const int iz0 = bin_of(zlo, g.z0, g.invDz, g.nZ);
          const int iz1 = bin_of(zhi, g.z0, g.invDz, g.nZ);
          lo[sd] = F.bin_first[g.bin0 + iz0 * g.nY];
          cnt[sd] = F.bin_first[g.bin0 + (iz1 + 1) * g.nY] - lo[sd];
        }
      }
    }
    if (cnt[0] > kStageMax || cnt[1] > kStageMax) {
      if (valid) links_one<kLeft>(F, P, k, bu, bd);
    } else if (cnt[0] > 0 && cnt[1] > 0) {
#pragma unroll
      for (int sd = 0; sd < 2; ++sd)
        for (int j = lane; j < cnt[sd]; j += 32) {
          const long kk = lo[sd] + j;
          float2 p = F.syz[kk];
          // a cluster taken by an earlier iteration can lie in no window
          if (kLeft && F.sused[kk]) p.x = __int_as_float(0x7fc00000);
          sP[wib][sd][j] = p;
          sI[wib][sd][j] = F.sid[kk];
        }
      __syncwarp();
      unsigned dm[3] = {0u, 0u, 0u}, um[3] = {0u, 0u, 0u};
#pragma unroll
      for (int w = 0; w < 3; ++w) {
        unsigned mdn = 0u, mup = 0u;
        for (int jj = 0; jj < 32 && 32 * w + jj < cnt[0]; ++jj) {
          const float2 p = sP[wib][0][32 * w + jj];
          if (fabsf(p.x - yc) <= P.link_wy && fabsf(p.y - zc) <= P.link_wz) mdn |= 1u << jj;
        }
        for (int jj = 0; jj < 32 && 32 * w + jj < cnt[1]; ++jj) {
          const float2 p = sP[wib][1][32 * w + jj];
          if (fabsf(p.x - yc) <= P.link_wy && fabsf(p.y - zc) <= P.link_wz) mup |= 1u << jj;
        }
        dm[w] = live ? mdn : 0u;
        um[w] = live ? mup : 0u;
      }
      const bool anyd = (dm[0] | dm[1] | dm[2]) != 0u;
      if (anyd) {
        const float xd = F.row_x[r - 1], xc = F.row_x[r], xu = F.row_x[r + 1];
        const float f = (xc - xd) / (xu - xd);
        float best = 0.0f;
        int buid = 0, bdid = 0;
#pragma unroll
        for (int wu = 0; wu < 3; ++wu)
          for (unsigned mu = um[wu]; mu; mu &= mu - 1u) {
            const int ju = 32 * wu + __ffs(mu) - 1;
            const float2 pu = sP[wib][1][ju];
            const float yu = pu.x, zu = pu.y;
            const int uid = sI[wib][1][ju];
#pragma unroll
            for (int wd = 0; wd < 3; ++wd)
              for (unsigned md = dm[wd]; md; md &= md - 1u) {
                const int jd = 32 * wd + __ffs(md) - 1;
                const float2 pd = sP[wib][0][jd];
                const float yd = pd.x, zd = pd.y;
                const float yp = yd + (yu - yd) * f;
                const float zp = zd + (zu - zd) * f;
                const float ey = yp - yc, ez = zp - zc;
                const float d2 = ey * ey + ez * ez;
                if (!(d2 < P.link_chi2)) continue;
                const int did = sI[wib][0][jd];
                if (bu < 0 || d2 < best ||
                    (d2 == best && (uid < buid || (uid == buid && did < bdid)))) {
                  best = d2;
                  bu = lo[1] + ju;
                  bd = lo[0] + jd;
                  buid = uid;
                  bdid = did;
                }
              }
          }
      }
    }
  }
  if (valid) {
    F.lup[k] = bu;
    F.ldn[k] = bd;
  }
}

// --------------------------------------------------------------- a3 cleaner
__global__ void k_clean(FrameDev F) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= F.n || F.cnt->err) return;
  const int u = F.lup[k], d = F.ldn[k];
  F.cup[k] = (u >= 0 && F.ldn[u] == (int)k) ? u : -1;
  F.cdn[k] = (d >= 0 && F.lup[d] == (int)k) ? d : -1;
}

// ------------------------------------------------------------ a4 start hits
// Compaction without atomics: per-block counts, scan of the counts, then each
// block writes its flagged elements at its offset in order.  An iteration's
// start hits follow those of the earlier iterations (from cnt->tl_base).
constexpr int kCompactItems = 4;  // elements per thread

__device__ __forceinline__ bool is_start(const FrameDev& F, long k) {
  const int u = F.cup[k];
  return F.cdn[k] < 0 && u >= 0 && F.cup[u] >= 0;
}

__global__ void k_start_count(FrameDev F) {
  __shared__ int sh[32];
  const long base = (long)blockIdx.x * blockDim.x * kCompactItems;
  int c = 0;
  if (!F.cnt->err)
    for (int j = 0; j < kCompactItems; ++j) {
      const long k = base + (long)j * blockDim.x + threadIdx.x;
      if (k < F.n && is_start(F, k)) ++c;
    }
  int tot;
  block_exscan(c, sh, &tot);
  if (threadIdx.x == 0) F.scan_tmp[blockIdx.x] = tot;
}

__global__ void k_start_write(FrameDev F) {
  __shared__ int sh[32];
  __shared__ int off;
  if (F.cnt->err) return;
  const long base = (long)blockIdx.x * blockDim.x * kCompactItems;
  if (threadIdx.x == 0) off = F.cnt->tl_base + F.scan_tmp[blockIdx.x];
  __syncthreads();
  for (int j = 0; j < kCompactItems; ++j) {
    const long k = base + (long)j * blockDim.x + threadIdx.x;
    const int flag = (k < F.n && is_start(F, k)) ? 1 : 0;
    int tot;
    const int ex = block_exscan(flag, sh, &tot);
    const int pos = off + ex;
    if (flag && pos < F.cap_tl) F.starts[pos] = (int)k;
    __syncthreads();
    if (threadIdx.x == 0) off += tot;
    __syncthreads();
  }
}

__global__ void k_start_check(FrameDev F) {
  F.cnt->n_starts = F.cnt->tl_base + F.cnt->n_new;
  if (F.cnt->n_starts > F.cap_tl) {
    atomicOr(&F.cnt->err, kErrCapTracklets);
    atomicMax(&F.cnt->need_tracklets, F.cnt->n_starts);
  }
}

// ------------------------------------------------------------ a5 tracklets
struct Pick {
  int k;
  float chi2;
};

// Best cluster of row (s, r) with chi2 < follow_chi2 (ties: smaller input id);
// the y/z box is the widened 2x2 Mahalanobis bound of the cut.  kLeft: the
// clusters taken by earlier sector-tracking iterations are not candidates;
// kKept: nor those kept by a sector track (the edge following).
template <bool kLeft, bool kKept = false>
__device__ __forceinline__ int pick(const FrameDev& F, const KParams& P, const Trk<float>& t,
                                    const RowGrid& g, float& by, float& bz) {
  const float hy = sqrtf(P.follow_chi2 * (t.c[0] + P.sy2)) * 1.001f + 0.01f;
  const float hz = sqrtf(P.follow_chi2 * (t.c[2] + P.sz2)) * 1.001f + 0.01f;
  const float ylo = t.p[0] - hy, yhi = t.p[0] + hy;
  const float zlo = t.p[1] - hz, zhi = t.p[1] + hz;
  int best = -1, bid = 0;
  float bchi = 0.0f;
  for_window(F.bin_first, g, ylo, yhi, zlo, zhi, [&](int k) {
    if (kLeft && F.sused[k]) return;
    if (kKept && F.st_kept[k]) return;
    const float2 pk = F.syz[k];
    const float yk = pk.x, zk = pk.y;
    if (!(yk >= ylo && yk <= yhi)) return;
    if (fabsf(zk - t.p[1]) > hz) return;
    const float chi2 = chi2_of(t, yk, zk, P);
    if (!(chi2 < P.follow_chi2)) return;
    const int id = F.sid[k];
    if (best < 0 || chi2 < bchi || (chi2 == bchi && id < bid)) {
      best = k;
      bchi = chi2;
      bid = id;
      by = yk;
      bz = zk;
    }
  });
  return best;
}

// CA chain of each start hit: its length and the seed through the chain's
// first, middle (the (L-1)/2-th up-link) and last cluster, computed here for
// all tracklets at once so that the constructor's state machine only loads
// it.  tl_seed: p[5], x, (sector, row) of the start, 1 / 0 = seed valid.
__global__ void k_chain_info(FrameDev F, KParams P) {
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  for (int ti = F.cnt->tl_base + blockIdx.x * blockDim.x + threadIdx.x; ti < nst;
       ti += gridDim.x * blockDim.x) {
    const int start = F.starts[ti];
    // the chain's clusters go to the tracklet's row-indexed hit array on the
    // way (a CA link joins adjacent rows of one sector, so the i-th cluster
    // lies on row r0 + i), where the constructor reads them in row order
    const int rr0 = F.srow[start];
    int* H = F.tl_hits + (long)ti * kMaxRows;
    const int r0 = rr0 % NR;
    H[r0] = start;
    int L = 1, last = start;
    for (int nx = F.cup[start]; nx >= 0; nx = F.cup[nx]) {
      last = nx;
      H[r0 + L] = nx;
      ++L;
    }
    const int mid = H[r0 + (L - 1) / 2];  // the (L-1)/2-th up-link
    F.tl_len[ti] = L;
    float xs[3], ys[3], zs[3];
    const int sel[3] = {start, mid, last};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int rs = i == 0 ? rr0 : (int)F.srow[sel[i]];
      xs[i] = F.row_x[rs % NR];
      const float2 ps = F.syz[sel[i]];
      ys[i] = ps.x;
      zs[i] = ps.y;
    }
    Trk<float> t;
    const bool ok = seed3(xs, ys, zs, P, t);
    float* sd = F.tl_seed + (long)ti * kSeedF;
#pragma unroll
    for (int i = 0; i < 5; ++i) sd[i] = t.p[i];
    sd[5] = t.x;
    sd[6] = __int_as_float(rr0);
    sd[7] = __int_as_float(ok ? 1 : 0);
  }
}

// Tracklet constructor as per-lane state machines: every loop iteration is
// one row step (propagate, choose the row's cluster, update) of the lane's
// current tracklet, and a lane whose tracklet ends takes the next one from the
// work queue in the same loop.  The lanes of a warp therefore stay busy on
// row steps however unequal their tracklets are.  Per tracklet the sequence
// of operations is that of the constructor (Sec. 2): seed from the chain's
// first, middle and last clusters; follow the CA chain upwards (k_tl_chain);
// extend upwards by the best cluster of each row until max_miss rows in a row
// have none (k_tl_up); restart from the top with reset covariance and refit
// downwards over the found clusters (k_tl_refit); extend below the start the
// same way (k_tl_down).  Four kernels rather than one: each carries only its
// own part's code and state, and all lanes of a kernel run the same kind of
// step (the steps over known clusters then run without the divergence of the
// searches).
//
// Per-thread shared-memory state of the searching and refitting kernels: the
// state they only save and restore (downward: the state at the innermost hit;
// upward: the state and position at the top hit), field-major so that a
// warp's accesses hit distinct banks.  It keeps the kernels at 64 registers,
// four 256-thread blocks per SM.
constexpr int kTlShared = 21;  // saved state: p[5], c[15], x (or p[5], x, y_hit, z_hit)

// Tracklet states between the kernels (tl_n): 0 none yet or rejected; -2 seed
// and chain followed, state in tl_par / tl_cov / tl_seed[5] (x), position of
// the top hit in tl_chi2 / tl_x, its row in tl_rhi; -1 upward part done, the
// state at the top hit in tl_seed[0..5], its position in tl_chi2 / tl_x.
constexpr int kTlChainDone = -2;
constexpr int kTlUpDone = -1;

// The state and position of the top hit, for the downward pass.
__device__ __forceinline__ void tl_up_done(const FrameDev& F, int ti, const float* p, float x,
                                           float y, float z, int top) {
  float* sd = F.tl_seed + (long)ti * kSeedF;
#pragma unroll
  for (int i = 0; i < 5; ++i) sd[i] = p[i];
  sd[5] = x;
  F.tl_chi2[ti] = y;
  F.tl_x[ti] = z;
  F.tl_rhi[ti] = top;
  F.tl_n[ti] = kTlUpDone;
}

// Upward pass, first part: seed and CA chain.  Every chain step takes the
// chain's next cluster (a CA link always joins adjacent pad rows of one
// sector, so the chain's next row is known); the next link and the cluster's
// position are requested before the propagation.  The state after the last
// update is the state at the top hit.
__global__ void __launch_bounds__(256, 4) k_tl_chain(FrameDev F, KParams P) {
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  const int tbase = F.cnt->tl_base;
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  bool busy = false;
  int ti = 0, rcur = 0, cn = 0, left = 0;
  const int* H = nullptr;  // the chain's clusters by row (k_chain_info)
  float yt = 0.0f, zt = 0.0f;  // position of the top hit
  Trk<float> t;
  for (;;) {
    bool handover = false;
    if (!busy) {
      ti = tbase + queue_next(&F.cnt->queue[kQTracklets]);
      if (ti >= nst) break;
      H = F.tl_hits + (long)ti * kMaxRows;
      const int L = F.tl_len[ti];
      const float* sd = F.tl_seed + (long)ti * kSeedF;
      float sv[kSeedF];
#pragma unroll
      for (int i = 0; i < kSeedF; ++i) sv[i] = sd[i];
      F.tl_n[ti] = 0;
      if (__float_as_int(sv[7]) == 0) continue;  // no seed
      const int r0 = __float_as_int(sv[6]) % NR;
#pragma unroll
      for (int i = 0; i < 5; ++i) t.p[i] = sv[i];
      t.x = sv[5];
      reset_cov(t.c, P);
      // the seed passes through the start cluster: its measurement is (y, z)
      // of the seed itself
      yt = t.p[0];
      zt = t.p[1];
      update(t, residual(t, yt, zt, P));
      if (L > 1) cn = H[r0 + 1];
      rcur = r0;
      left = L - 1;  // chain steps still to take
      busy = left > 0;
      handover = !busy;
    } else {
      // ---- one chain step
      const int r = rcur + 1;
      const int k = cn;
      if (left > 1) cn = H[r + 1];
      const float2 pk = F.syz[k];
      const bool stop = r >= NR || !propagate(t, F.row_x[r], P, P.max_snp);
      if (stop) {
        tl_up_done(F, ti, t.p, t.x, yt, zt, rcur);
        busy = false;
        continue;
      }
      update(t, residual(t, pk.x, pk.y, P));
      yt = pk.x;
      zt = pk.y;
      rcur = r;
      busy = --left > 0;
      handover = !busy;
    }
    if (!handover) continue;
#pragma unroll
    for (int i = 0; i < 5; ++i) F.tl_par[(long)ti * 5 + i] = t.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) F.tl_cov[(long)ti * 15 + i] = t.c[i];
    F.tl_seed[(long)ti * kSeedF + 5] = t.x;
    F.tl_chi2[ti] = yt;
    F.tl_x[ti] = zt;
    F.tl_rhi[ti] = rcur;
    F.tl_n[ti] = kTlChainDone;
  }
}

// Upward pass, second part: extension by the best cluster of each row from
// the chain's top.  The state at the top hit and that hit's position are left
// in tl_seed[0..5], tl_chi2 and tl_x for the downward pass.
template <bool kLeft>
__global__ void __launch_bounds__(256, 4) k_tl_up(FrameDev F, KParams P) {
  extern __shared__ float tl_sh[];
  float* const S = tl_sh + threadIdx.x;
  const int BS = blockDim.x;
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  const int tbase = F.cnt->tl_base;
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  bool busy = false;
  int ti = 0, sbase = 0, top = 0, rcur = 0, miss = 0;
  int* H = nullptr;
  Trk<float> t;
  auto save_top = [&](float y, float z) {
#pragma unroll
    for (int i = 0; i < 5; ++i) S[i * BS] = t.p[i];
    S[5 * BS] = t.x;
    S[6 * BS] = y;
    S[7 * BS] = z;
  };
  for (;;) {
    if (!busy) {
      ti = tbase + queue_next(&F.cnt->queue[kQTlUp]);
      if (ti >= nst) break;
      if (F.tl_n[ti] != kTlChainDone) continue;
      H = F.tl_hits + (long)ti * kMaxRows;
      const float* sd = F.tl_seed + (long)ti * kSeedF;
#pragma unroll
      for (int i = 0; i < 5; ++i) t.p[i] = F.tl_par[(long)ti * 5 + i];
#pragma unroll
      for (int i = 0; i < 15; ++i) t.c[i] = F.tl_cov[(long)ti * 15 + i];
      t.x = sd[5];
      const int rr0 = __float_as_int(sd[6]);
      sbase = rr0 - rr0 % NR;  // sector * n_rows
      top = F.tl_rhi[ti];
      rcur = top;
      save_top(F.tl_chi2[ti], F.tl_x[ti]);
      miss = 0;
      busy = true;
      continue;
    }
    // ---- one row step (the row's grid record requested before the
    // propagation, so that its latency overlaps the arithmetic)
    const int r = rcur + 1;
    bool stop = r >= NR;
    RowGrid g;
    if (!stop) g = F.rows[sbase + r];
    if (!stop) stop = !propagate(t, F.row_x[r], P, P.max_snp);
    if (!stop) stop = fabsf(t.p[0]) > t.x * P.tan_half + P.edge_margin;
    bool miss_out = false;
    if (!stop) {
      float ky = 0.0f, kz = 0.0f;
      const int k = pick<kLeft>(F, P, t, g, ky, kz);
      if (k >= 0) {
        update(t, residual(t, ky, kz, P));
        H[r] = k;
        save_top(ky, kz);
        top = r;
        miss = 0;
      } else {
        H[r] = -1;
        miss_out = ++miss >= P.max_miss;
      }
      rcur = r;
    }
    if (!(stop || miss_out)) continue;
    // upward part done (no more rows, edge or max_miss misses)
    float pt[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) pt[i] = S[i * BS];
    tl_up_done(F, ti, pt, S[5 * BS], S[6 * BS], S[7 * BS], top);
    busy = false;
  }
}

// Ambiguity key of a tracklet (Sec. 3 Phase I: priority to a small chi2
// per degree of freedom, then to length): the ordered bits of
// score = n - w * chi2 / ndf, then the complement of the start cluster's
// input id (a unique tie-break).
__device__ __forceinline__ unsigned long long make_tl_key(int n, float chi2, unsigned sid,
                                                          const KParams& P) {
  const float score = (float)n - P.score_w * (chi2 / (float)(2 * n - 5));
  return ((unsigned long long)f2o(score) << 32) | (unsigned long long)(0xFFFFFFFFu - sid);
}

// The downward pass's result: n clusters, the state at the innermost one,
// and the tracklet's ambiguity key for the selection.
__device__ __forceinline__ void tl_down_done(const FrameDev& F, const KParams& P, int ti, int n,
                                             int rlo, int top, float chi2, const float* S,
                                             int BS) {
  if (n < P.min_hits) return;  // tl_n stays 0
  F.tl_n[ti] = n;
  F.tl_key[ti] = make_tl_key(n, chi2, (unsigned)F.sid[F.starts[ti]], P);
  F.tl_rlo[ti] = rlo;
  F.tl_rhi[ti] = top;
  F.tl_chi2[ti] = chi2;
  F.tl_x[ti] = S[20 * BS];
#pragma unroll
  for (int i = 0; i < 5; ++i) F.tl_par[(long)ti * 5 + i] = S[i * BS];
#pragma unroll
  for (int i = 0; i < 15; ++i) F.tl_cov[(long)ti * 15 + i] = S[(5 + i) * BS];
}

// Downward pass, first part: restart at the top hit with reset covariance
// and refit down over the hits found on the way up (the next stored hit is
// requested one step ahead, its position before the propagation).  The start
// row always holds a hit (the start cluster), so a tracklet that reaches it
// leaves this kernel with the state at its innermost hit: that state, chi2 and
// the count go to the extension below the start (tl_n = -3; n in tl_rlo).
constexpr int kTlRefitDone = -3;

__global__ void __launch_bounds__(256, 4) k_tl_refit(FrameDev F, KParams P) {
  extern __shared__ float tl_sh[];
  float* const S = tl_sh + threadIdx.x;
  const int BS = blockDim.x;
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  const int tbase = F.cnt->tl_base;
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  bool busy = false;
  int ti = 0, r0 = 0, top = 0, rcur = 0, hn = -1, n = 0, rlo = 0;
  const int* H = nullptr;
  float chi2 = 0.0f;
  Trk<float> t;
  auto save_inner = [&]() {
#pragma unroll
    for (int i = 0; i < 5; ++i) S[i * BS] = t.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) S[(5 + i) * BS] = t.c[i];
    S[20 * BS] = t.x;
  };
  for (;;) {
    if (!busy) {
      ti = tbase + queue_next(&F.cnt->queue[kQTlRefit]);
      if (ti >= nst) break;
      if (F.tl_n[ti] != kTlUpDone) continue;
      H = F.tl_hits + (long)ti * kMaxRows;
      const float* sd = F.tl_seed + (long)ti * kSeedF;
      float sv[kSeedF];
#pragma unroll
      for (int i = 0; i < kSeedF; ++i) sv[i] = sd[i];
      const float ty = F.tl_chi2[ti], tz = F.tl_x[ti];
      top = F.tl_rhi[ti];
      r0 = __float_as_int(sv[6]) % NR;
      F.tl_n[ti] = 0;
#pragma unroll
      for (int i = 0; i < 5; ++i) t.p[i] = sv[i];
      t.x = sv[5];
      reset_cov(t.c, P);
      const Resid R = residual(t, ty, tz, P);
      chi2 = R.chi2;
      update(t, R);
      hn = top - 1 >= r0 ? H[top - 1] : -1;
      n = 1;
      save_inner();
      rlo = top;
      rcur = top;
      busy = top > r0;
    } else {
      // ---- one stored row step
      const int r = rcur - 1;
      const int k = hn;
      hn = r - 1 >= r0 ? H[r - 1] : -1;
      float2 pk = make_float2(0.0f, 0.0f);
      if (k >= 0) pk = F.syz[k];
      bool stop = !propagate(t, F.row_x[r], P, P.max_snp);
      if (!stop) stop = fabsf(t.p[0]) > t.x * P.tan_half + P.edge_margin;
      if (stop) {
        tl_down_done(F, P, ti, n, rlo, top, chi2, S, BS);
        busy = false;
        continue;
      }
      if (k >= 0) {
        const Resid R = residual(t, pk.x, pk.y, P);
        chi2 = chi2 + R.chi2;
        update(t, R);
        ++n;
        save_inner();
        rlo = r;
      }
      rcur = r;
      busy = r > r0;
    }
    if (busy) continue;
    // at the start row, whose hit was the last update: t is the innermost state
#pragma unroll
    for (int i = 0; i < 5; ++i) F.tl_par[(long)ti * 5 + i] = t.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) F.tl_cov[(long)ti * 15 + i] = t.c[i];
    F.tl_x[ti] = t.x;
    F.tl_chi2[ti] = chi2;
    F.tl_rlo[ti] = n;
    F.tl_n[ti] = kTlRefitDone;
  }
}

// Downward pass, second part: extension below the start by the best cluster
// of each row until max_miss rows in a row have none.
template <bool kLeft>
__global__ void __launch_bounds__(256, 4) k_tl_down(FrameDev F, KParams P) {
  extern __shared__ float tl_sh[];
  float* const S = tl_sh + threadIdx.x;
  const int BS = blockDim.x;
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  const int tbase = F.cnt->tl_base;
  if (F.cnt->err) return;
  const int NR = P.n_rows;
  bool busy = false;
  int ti = 0, sbase = 0, top = 0, rcur = 0, miss = 0, n = 0, rlo = 0;
  int* H = nullptr;
  float chi2 = 0.0f;
  Trk<float> t;
  auto save_inner = [&]() {
#pragma unroll
    for (int i = 0; i < 5; ++i) S[i * BS] = t.p[i];
#pragma unroll
    for (int i = 0; i < 15; ++i) S[(5 + i) * BS] = t.c[i];
    S[20 * BS] = t.x;
  };
  for (;;) {
    if (!busy) {
      ti = tbase + queue_next(&F.cnt->queue[kQTlDown]);
      if (ti >= nst) break;
      if (F.tl_n[ti] != kTlRefitDone) continue;
      H = F.tl_hits + (long)ti * kMaxRows;
#pragma unroll
      for (int i = 0; i < 5; ++i) t.p[i] = F.tl_par[(long)ti * 5 + i];
#pragma unroll
      for (int i = 0; i < 15; ++i) t.c[i] = F.tl_cov[(long)ti * 15 + i];
      t.x = F.tl_x[ti];
      chi2 = F.tl_chi2[ti];
      n = F.tl_rlo[ti];
      top = F.tl_rhi[ti];
      const int rr0 = __float_as_int(F.tl_seed[(long)ti * kSeedF + 6]);
      const int r0 = rr0 % NR;
      sbase = rr0 - r0;
      F.tl_n[ti] = 0;
      save_inner();
      rlo = r0;
      rcur = r0;
      miss = 0;
      busy = true;
      continue;
    }
    // ---- one row step (the row's grid record before the propagation)
    const int r = rcur - 1;
    bool stop = r < 0;
    RowGrid g;
    if (!stop) g = F.rows[sbase + r];
    if (!stop) stop = !propagate(t, F.row_x[r], P, P.max_snp);
    if (!stop) stop = fabsf(t.p[0]) > t.x * P.tan_half + P.edge_margin;
    bool miss_out = false;
    if (!stop) {
      float ky = 0.0f, kz = 0.0f;
      const int k = pick<kLeft>(F, P, t, g, ky, kz);
      if (k >= 0) {
        const Resid R = residual(t, ky, kz, P);
        chi2 = chi2 + R.chi2;
        update(t, R);
        H[r] = k;
        miss = 0;
        ++n;
        save_inner();
        rlo = r;
      } else {
        H[r] = -1;
        miss_out = ++miss >= P.max_miss;
      }
      rcur = r;
    }
    if (!(stop || miss_out)) continue;
    tl_down_done(F, P, ti, n, rlo, top, chi2, S, BS);
    busy = false;
  }
}

// ------------------------------------------------------------- a6 selector
__device__ __forceinline__ unsigned long long tracklet_key(const FrameDev& F, int ti) {
  return F.tl_key[ti];
}

// One warp per tracklet: the lanes read 32 consecutive rows of the
// row-indexed hit array at once and raise those hits' owner keys together.
__global__ void k_sel_owner(FrameDev F, KParams P) {
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  if (F.cnt->err) return;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int ti = F.cnt->tl_base + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); ti < nst;
       ti += nw) {
    // (the four loads issued together; key and rows are read for every
    // tracklet and used for the finished ones)
    const int n = F.tl_n[ti];
    const unsigned long long key = tracklet_key(F, ti);
    const int rlo = F.tl_rlo[ti], rhi = F.tl_rhi[ti];
    if (n == 0) continue;
    const int* H = F.tl_hits + (long)ti * kMaxRows;
    for (int r = rlo + lane; r <= rhi; r += 32) {
      const int h = H[r];
      if (h >= 0) atomicMax(&F.owner_key[h], key);
    }
  }
}

// Outer-to-inner walk of every tracklet's hits.  The rows are taken in
// groups of kWalkGroup: their hit indices, then those hits' owner keys, are
// requested together before the (sequential) keep decisions of the group.
constexpr int kWalkGroup = 16;

__global__ void k_sel_walk(FrameDev F, KParams P) {
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  if (F.cnt->err) return;
  for (int ti = F.cnt->tl_base + blockIdx.x * blockDim.x + threadIdx.x; ti < nst;
       ti += gridDim.x * blockDim.x) {
    F.tl_acc[ti] = 0;
    F.tl_nkept[ti] = 0;
    if (F.tl_n[ti] == 0) continue;
    const unsigned long long key = tracklet_key(F, ti);
    const int* H = F.tl_hits + (long)ti * kMaxRows;
    int* K = F.tl_kept + (long)ti * kMaxRows;
    const int rlo = F.tl_rlo[ti], rhi = F.tl_rhi[ti];
    int kept = 0, shared = 0;
    unsigned owned[(kMaxRows + 31) / 32] = {};  // bit j: K[j] is owned
    for (int rg = rhi; rg >= rlo; rg -= kWalkGroup) {
      int h[kWalkGroup];
      unsigned long long ok[kWalkGroup];
#pragma unroll
      for (int j = 0; j < kWalkGroup; ++j) h[j] = rg - j >= rlo ? H[rg - j] : -1;
#pragma unroll
      for (int j = 0; j < kWalkGroup; ++j) ok[j] = h[j] >= 0 ? F.owner_key[h[j]] : 0ull;
#pragma unroll
      for (int j = 0; j < kWalkGroup; ++j) {
        const int k = h[j];
        if (k < 0) continue;
        if (ok[j] == key) {
          owned[kept >> 5] |= 1u << (kept & 31);
          K[kept++] = k;
        } else if ((float)(shared + 1) <= P.shared_frac * (float)(kept + 1)) {
          K[kept++] = k;
          ++shared;
        }
      }
    }
    if (kept >= P.min_hits) {
      F.tl_nkept[ti] = kept;
      F.tl_acc[ti] = 1;
      for (int j = 0; j < kept; ++j)
        if (owned[j >> 5] & (1u << (j & 31))) F.sec_owner[K[j]] = ti;
    }
  }
}

// ------------------------------------------- later seeding iterations
// Sec. 3 (Phase III) seeds again on the clusters left over after the ambiguity
// solving.  Between two iterations: every cluster kept by an accepted tracklet
// of the iteration just done, and its start cluster, become taken; the owner
// keys of the clusters still free are cleared for the next selection (only the
// next iteration's tracklets, which hold free clusters only, compete there).
__global__ void k_mark_used(FrameDev F) {
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  if (F.cnt->err) return;
  for (int ti = F.cnt->tl_base + blockIdx.x * blockDim.x + threadIdx.x; ti < nst;
       ti += gridDim.x * blockDim.x) {
    if (!F.tl_acc[ti]) continue;
    const int nk = F.tl_nkept[ti];
    const int* K = F.tl_kept + (long)ti * kMaxRows;
    for (int j = 0; j < nk; ++j) F.sused[K[j]] = 1;
    F.sused[F.starts[ti]] = 1;
  }
}

__global__ void k_owner_reset(FrameDev F) {
  if (F.cnt->err) return;
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < F.n;
       k += (long)gridDim.x * blockDim.x)
    if (!F.sused[k]) F.owner_key[k] = 0ull;
}

// The next iteration's tracklets follow the current ones.
__global__ void k_pass_begin(FrameDev F, int pass) {
  const int nst = min(F.cnt->n_starts, (int)F.cap_tl);
  F.cnt->tl_base = nst;
  F.cnt->pass_start[pass] = nst;
  F.cnt->queue[kQTracklets] = 0;
  F.cnt->queue[kQTlUp] = 0;
  F.cnt->queue[kQTlRefit] = 0;
  F.cnt->queue[kQTlDown] = 0;
}

// ------------------------------------------------------------ edge following
// Sec. 2: the sector tracking cannot find very short track segments, so
// tracks ending at a sector edge close to the upper or lower end of the TPC
// are propagated into the adjacent sector before the merging and followed
// there.  From each end of a sector track the end state is propagated row by
// row away from the track over at most edge_rows rows, over its sector's edge
// once (rotation into the neighbouring sector of the same side, then the
// row's x there); from the crossing on, each row's best cluster kept by no
// sector track is filtered in, until max_miss rows in a row have none.  A
// segment of at least edge_min clusters becomes a sector track of the
// neighbouring sector (a tracklet slot holds its clusters), linked to the
// track it continues before the merging.  Segment order and keys do not
// depend on scheduling: ends are numbered 2 j + (inner end), segments are
// compacted in that order, and a segment's key is its track's key plus 2^29
// (inner end) or 2^30 (outer end).

__global__ void k_edge_mark(FrameDev F) {  // one warp per sector track
  const int ns = F.cnt->n_tracks;
  if (F.cnt->err) return;
  const int lane = threadIdx.x & 31;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); j < ns; j += nw) {
    if (!F.st_ok[j]) continue;
    const int ti = F.st_tl[j];
    const int nk = F.tl_nkept[ti];
    const int* K = F.tl_kept + (long)ti * kMaxRows;
    for (int m = lane; m < nk; m += 32) F.st_kept[K[m]] = 1;
  }
}

// Can an end reach its sector's edge within the rows ahead (x1: the last of
// them)?  Along a helix sin(phi) is linear in x, so over the run |sin(phi)|
// stays below s = max(|sin(phi0)|, |sin(phi0) + kappa dx|) and |dy/dx| below
// t = s / sqrt(1 - s^2); the distance to the edge, x tan(10 deg) - |y|, can
// then shrink by at most |dx| (t -+ tan(10 deg)) (outward / inward).  A 1 cm
// margin covers the rounding; an end ruled out here would cross no edge in
// the row-by-row propagation either, so the result does not change.
__device__ __forceinline__ bool edge_reachable(const Trk<float>& t, float x1, const KParams& P) {
  const float dx = x1 - t.x;
  const float s0 = t.p[2];
  const float s = fmaxf(fabsf(s0), fabsf(s0 + t.p[4] * P.kb * dx));
  if (!(s < P.max_snp)) return true;  // the propagation decides
  const float tmax = s / sqrtf(1.0f - s * s);
  const float e0 = t.x * P.tan_half - fabsf(t.p[0]);
  const float close = fabsf(dx) * (dx > 0.0f ? tmax - P.tan_half : tmax + P.tan_half);
  return e0 - 1.0f < close;
}

// The segment beyond one end of sector track j: returns the clusters found;
// their sorted indices go to K in the order found, `first` / `last` receive
// the filter after the first and the last of them, `sec` the sector.
__device__ int edge_follow(const FrameDev& F, const KParams& P, int j, bool inner, int* K,
                           Trk<float>* first, Trk<float>* last, int& sec) {
  const int NR = P.n_rows;
  Trk<float> t;
  get_state((inner ? F.st_ie : F.st_oe) + (long)j * kStateF, t);
  sec = F.st_sector[j];
  const int dir = inner ? -1 : 1;
  const int r0 = inner ? F.st_rmin[j] : F.st_rmax[j];
  const int r_end = inner ? max(r0 - P.edge_rows, 0) : min(r0 + P.edge_rows, NR - 1);
  if (r_end == r0 || !edge_reachable(t, F.row_x[r_end], P)) return 0;
  bool crossed = false;
  int miss = 0, nh = 0;
  for (int e = 1; e <= P.edge_rows; ++e) {
    const int r = r0 + dir * e;
    if (r < 0 || r >= NR) break;
    if (!propagate(t, F.row_x[r], P, P.max_snp)) break;
    if (!crossed && fabsf(t.p[0]) > t.x * P.tan_half) {
      const int d = t.p[0] > 0.0f ? 1 : -1;
      if (!rotate(t, d, P, P.max_snp)) break;
      const int half = P.n_phi;
      sec = sec - sec % half + (sec % half + (d > 0 ? 1 : half - 1)) % half;
      if (!propagate(t, F.row_x[r], P, P.max_snp)) break;
      crossed = true;
    }
    if (fabsf(t.p[0]) > t.x * P.tan_half + P.edge_margin) break;
    if (!crossed) continue;
    float ky = 0.0f, kz = 0.0f;
    const int k = pick<false, true>(F, P, t, F.rows[sec * NR + r], ky, kz);
    if (k >= 0) {
      update(t, residual(t, ky, kz, P));
      if (K) K[nh] = k;
      if (first && nh == 0) *first = t;
      if (last) *last = t;
      ++nh;
      miss = 0;
    } else if (++miss >= P.max_miss) {
      break;
    }
  }
  return nh;
}

// Which ends find a segment (flag per end, over the whole capacity so that
// the scan behind it reads no stale flags).
__global__ void k_edge_count(FrameDev F, KParams P) {
  const int ns = F.cnt->n_tracks;
  const long m = 2 * F.cap_tl;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q <= m;
       q += (long)gridDim.x * blockDim.x) {
    int f = 0;
    const int j = (int)(q >> 1);
    if (!F.cnt->err && q < 2L * ns && F.st_ok[j]) {
      int sec;
      f = edge_follow(F, P, j, (q & 1) != 0, nullptr, nullptr, nullptr, sec) >= P.edge_min;
    }
    F.edge_flag[q] = f;
  }
}

// Room for the segments: sector-track entries after the tracks, tracklet
// slots after the tracklets.
__global__ void k_edge_commit(FrameDev F) {
  const int ns = F.cnt->n_tracks;
  const int ntl = min(F.cnt->n_starts, (int)F.cap_tl);
  const int nseg = F.edge_pos[2 * F.cap_tl];
  F.cnt->n_st0 = ns;
  F.cnt->n_tl_all = ntl;
  if (F.cnt->err) return;
  const long need = (long)max(ns, ntl) + nseg;
  if (need > F.cap_tl) {
    atomicOr(&F.cnt->err, kErrCapEdge);
    atomicMax(&F.cnt->need_tracklets, (int)need);
    return;
  }
  F.cnt->n_tracks = ns + nseg;
}

// Every segment: the following again, now keeping its clusters, states and
// links.  The outer segment of j continues j (j -> segment), the inner one
// leads into it (segment -> j); the linked ends take no part in the merging.
__global__ void k_edge_write(FrameDev F, KParams P) {
  const int ns0 = F.cnt->n_st0, ntl = F.cnt->n_tl_all;
  if (F.cnt->err) return;
  for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < 2L * ns0;
       q += (long)gridDim.x * blockDim.x) {
    if (!F.edge_flag[q]) continue;
    const int j = (int)(q >> 1);
    const bool inner = (q & 1) != 0;
    const int k = F.edge_pos[q];
    const int i = ns0 + k, ti = ntl + k;
    int H[kMaxRows];
    Trk<float> first, last;
    int sec;
    const int nh = edge_follow(F, P, j, inner, H, &first, &last, sec);
    int* K = F.tl_kept + (long)ti * kMaxRows;  // outermost first
    for (int m = 0; m < nh; ++m) K[m] = inner ? H[m] : H[nh - 1 - m];
    F.tl_nkept[ti] = nh;
    F.tl_rlo[ti] = 1;  // no tracklet hits (the seeding history of the cluster removal)
    F.tl_rhi[ti] = 0;
    F.st_tl[i] = ti;
    F.st_key[i] = F.st_key[j] + (inner ? (1 << 29) : (1 << 30));
    F.st_sector[i] = sec;
    const int r_a = F.srow[H[0]] % P.n_rows, r_b = F.srow[H[nh - 1]] % P.n_rows;
    F.st_rmin[i] = inner ? r_b : r_a;
    F.st_rmax[i] = inner ? r_a : r_b;
    put_state(F.st_ie + (long)i * kStateF, inner ? last : first, sec);
    put_state(F.st_oe + (long)i * kStateF, inner ? first : last, sec);
    F.st_ok[i] = 1;
    F.st_bestB[i] = -1;
    F.st_bestA[i] = ~0ull;
    F.st_xbestB[i] = -1;
    F.st_xbestA[i] = ~0ull;
    F.st_dz[i] = 0.0f;
    if (inner) {
      F.st_next[i] = j;
      F.st_hasprev[i] = 0;
      F.st_hasprev[j] = 1;
    } else {
      F.st_next[j] = i;
      F.st_next[i] = -1;
      F.st_hasprev[i] = 1;
    }
  }
}

// The neighbour search on 1, 4 or 8 lanes per cluster, or staged per warp
// (lanes = 32; launch slot kLLinks).
template <bool kLeft>
void launch_links(FrameDev& F, const KParams& P, long n, cudaStream_t s) {
  switch (F.lc.lanes[kLLinks]) {
    case 32: k_links_w<kLeft><<<blocks_for(n, 32 * kStageWarps), 32 * kStageWarps, 0, s>>>(F, P); break;
    case 8: k_links_g<8, kLeft><<<blocks_for(n, 256 / 8), 256, 0, s>>>(F, P); break;
    case 4: k_links_g<4, kLeft><<<blocks_for(n, 256 / 4), 256, 0, s>>>(F, P); break;
    default: k_links<kLeft><<<blocks_for(n, kBlock), kBlock, 0, s>>>(F, P); break;
  }
}

}  // namespace

// Allows the shared-memory row statistics their dynamic shared memory on
// the current device (before any launch or stream capture); without it the
// grid build takes the plain statistics kernel.
void init_attributes() {
  g_row_stats_shared = cudaFuncSetAttribute(k_row_stats_sh,
                                            cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            kRowStatsMaxRows * 12) == cudaSuccess;
}

// Stage launchers; each returns the number of kernels it enqueued.
int stage_grid(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  const long n = F.n;
  int k = 0;
  // rows of one frame: the window of the shared-memory statistics
  const int W = (F.nsrc > 0 ? F.src_nsec : P.n_sectors) * P.n_rows;
  if (n > 0 && g_row_stats_shared && W <= kRowStatsMaxRows) {
    k_row_stats_sh<<<blocks_for(n, kRowStatsChunk), 256, (size_t)W * 12, s>>>(F, P, W);
    ++k;
  } else if (n > 0) {
    k_row_stats<<<blocks_for(n, kBlock), kBlock, 0, s>>>(F, P);
    ++k;
  }
  k_row_grid<<<1, 1024, 0, s>>>(F, P); ++k;
  if (n > 0) { k_bin_hist<<<blocks_for(n, kBlock), kBlock, 0, s>>>(F, P); ++k; }
  k_row_scan<<<P.n_sectors * P.n_rows, 256, 0, s>>>(F);
  ++k;
  if (n > 0) {
    k_scatter<<<blocks_for(n, kBlock), kBlock, 0, s>>>(F);
    k_bin_sort<<<blocks_for(n, kBlock), kBlock, 0, s>>>(F);
    k_row_fill<<<P.n_sectors * P.n_rows, 128, 0, s>>>(F);
    k += 3;
  }
  return k;
}

int stage_links(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  (void)sms;
  const long n = F.n;
  if (n <= 0) return 0;
  launch_links<false>(F, P, n, s);
  k_clean<<<blocks_for(n, kBlock), kBlock, 0, s>>>(F);
  return 2;
}

int stage_starts(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  (void)P; (void)sms;
  const long n = F.n;
  const int nb = (int)blocks_for(n > 0 ? n : 1, kBlock * kCompactItems);
  k_start_count<<<nb, kBlock, 0, s>>>(F);
  k_scan_partials<<<1, 1024, 0, s>>>(F.scan_tmp, nb, &F.cnt->n_new);
  k_start_write<<<nb, kBlock, 0, s>>>(F);
  k_start_check<<<1, 1, 0, s>>>(F);
  return 4;
}

int stage_tracklets(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  k_chain_info<<<sms * 8, kBlock, 0, s>>>(F, P);
  const int tb = F.lc.block[kLTracklets];
  const size_t sh = sizeof(float) * kTlShared * tb;
  k_tl_chain<<<persistent_grid(F.lc, kLTracklets, sms), tb, 0, s>>>(F, P);
  k_tl_up<false><<<persistent_grid(F.lc, kLTracklets, sms), tb, sh, s>>>(F, P);
  k_tl_refit<<<persistent_grid(F.lc, kLTracklets, sms), tb, sh, s>>>(F, P);
  k_tl_down<false><<<persistent_grid(F.lc, kLTracklets, sms), tb, sh, s>>>(F, P);
  return 5;
}

int stage_select(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  k_sel_owner<<<sms * 8, kBlock, 0, s>>>(F, P);
  k_sel_walk<<<sms * 8, kBlock, 0, s>>>(F, P);
  return 2;
}

// Sector-tracking iterations 2..seed_iters, each on the clusters the accepted
// tracklets of the earlier ones left: the same neighbour finding, cleaning,
// start hits, tracklet construction and selection, over the free clusters.
int stage_edge(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  if (P.edge_rows <= 0) return 0;
  if (cudaMemsetAsync(F.st_kept, 0, F.n > 0 ? F.n : 1, s) != cudaSuccess) return 0;
  k_edge_mark<<<sms * 8, kBlock, 0, s>>>(F);
  k_edge_count<<<sms * 8, kBlock, 0, s>>>(F, P);
  int k = 2 + scan_exclusive(F.edge_flag, F.edge_pos, 2 * F.cap_tl + 1, F.scan_tmp, s);
  k_edge_commit<<<1, 1, 0, s>>>(F);
  k_edge_write<<<sms * 8, kBlock, 0, s>>>(F, P);
  return k + 2;
}

int stage_reseed(FrameDev& F, const KParams& P, int sms, cudaStream_t s) {
  const long n = F.n;
  if (P.seed_iters <= 1 || n <= 0) return 0;
  int k = 0;
  const int nb = (int)blocks_for(n, kBlock * kCompactItems);
  const int tb = F.lc.block[kLTracklets];
  const size_t sh = sizeof(float) * kTlShared * tb;
  for (int pass = 1; pass < P.seed_iters; ++pass) {
    k_mark_used<<<sms * 8, kBlock, 0, s>>>(F);
    k_owner_reset<<<sms * 8, kBlock, 0, s>>>(F);
    k_pass_begin<<<1, 1, 0, s>>>(F, pass);
    launch_links<true>(F, P, n, s);
    k_clean<<<blocks_for(n, kBlock), kBlock, 0, s>>>(F);
    k_start_count<<<nb, kBlock, 0, s>>>(F);
    k_scan_partials<<<1, 1024, 0, s>>>(F.scan_tmp, nb, &F.cnt->n_new);
    k_start_write<<<nb, kBlock, 0, s>>>(F);
    k_start_check<<<1, 1, 0, s>>>(F);
    k_chain_info<<<sms * 8, kBlock, 0, s>>>(F, P);
    k_tl_chain<<<persistent_grid(F.lc, kLTracklets, sms), tb, 0, s>>>(F, P);
    k_tl_up<true><<<persistent_grid(F.lc, kLTracklets, sms), tb, sh, s>>>(F, P);
    k_tl_refit<<<persistent_grid(F.lc, kLTracklets, sms), tb, sh, s>>>(F, P);
    k_tl_down<true><<<persistent_grid(F.lc, kLTracklets, sms), tb, sh, s>>>(F, P);
    k_sel_owner<<<sms * 8, kBlock, 0, s>>>(F, P);
    k_sel_walk<<<sms * 8, kBlock, 0, s>>>(F, P);
    k += 16;
  }
  return k;
}

// ------------------------------------------------------------------- scan
namespace {
constexpr int kScanItems = 8;

__global__ void k_scan_reduce(const int* in, long n, int* part) {
  __shared__ int sh[32];
  const long base = (long)blockIdx.x * blockDim.x * kScanItems;
  int s = 0;
  for (int j = 0; j < kScanItems; ++j) {
    const long i = base + (long)j * blockDim.x + threadIdx.x;
    if (i < n) s += in[i];
  }
  int tot;
  block_exscan(s, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void k_scan_apply(const int* in, int* out, long n, const int* part) {
  __shared__ int sh[32];
  __shared__ int off;
  const long base = (long)blockIdx.x * blockDim.x * kScanItems;
  if (threadIdx.x == 0) off = part[blockIdx.x];
  __syncthreads();
  for (int j = 0; j < kScanItems; ++j) {
    const long i = base + (long)j * blockDim.x + threadIdx.x;
    const int v = i < n ? in[i] : 0;
    int tot;
    const int ex = block_exscan(v, sh, &tot);
    if (i < n) out[i] = off + ex;
    __syncthreads();
    if (threadIdx.x == 0) off += tot;
    __syncthreads();
  }
}
}  // namespace

int scan_exclusive(const int* in, int* out, long n, int* tmp, cudaStream_t s) {
  const int nb = (int)blocks_for(n, kBlock * kScanItems);
  k_scan_reduce<<<nb, kBlock, 0, s>>>(in, n, tmp);
  k_scan_partials<<<1, 1024, 0, s>>>(tmp, nb, tmp + nb);
  k_scan_apply<<<nb, kBlock, 0, s>>>(in, out, n, tmp);
  return 3;
}

}  // namespace TPC_NS
}  // namespace tpc
