// Online cluster removal (Sec. 4) on the tracks of the last tracking call.
//
// Clusters inside a protective tube around physics tracks are kept; of the
// others, those inside a removal tube around secondary looper legs and
// around very-low-pT tracks are flagged for removal; the clusters of the
// tracklets a physics track was built from (its seeding history) are
// protected too.  The section gives the rules in words; the readings:
// * very low pT: |q/pT| at the innermost cluster above qpt;
// * looper legs: two looper tracks (|q/pT| > looper_qpt) of one side whose
//   |q/pT| differ by at most leg_dq relative, whose tan(lambda) are opposite
//   within leg_dtgl (legs flown inwards are parametrised outwards) and whose
//   circle centres in global coordinates lie within leg_dc; |z| grows along
//   the looper and side * z_measured differs from it by one constant of the
//   collision, so a leg linked to one with a smaller side * z at the
//   innermost cluster is a secondary leg; its parent is the first such leg
//   (smallest (side * z, key), the track key breaking exact ties);
// * tubes follow the track's clusters, with the linear interpolation from
//   the lower-row cluster on the rows between two consecutive clusters of one
//   sector; protection 1 = a wide protective and a narrow removal tube;
//   protection 2 (mode 2) scales them on the innermost rows, near the sector
//   edge and where the occupancy around the centre is high.
// Every decision is an integer or a comparison of FP32 values computed in the
// same order as the strict CPU oracle; flags are combined with atomicOr, so
// the result does not depend on the order of the threads.
#include <cuda_runtime.h>

#include "tpc_internal.h"
#include "tpc_kernels.h"
#include "tpc_util.cuh"

namespace tpc {
namespace TPC_NS {
namespace {

constexpr float kCrHalfRange = 256.0f;  // circle centres binned over [-256, 256) cm per axis

// Centre bin of a circle centre (clamped: centres outside the range share the
// edge bins, which keeps any two centres within one bin width in adjacent bins).
__device__ __forceinline__ int centre_bin(float c, const RemovalParams& R) {
  return min(R.nbx - 1, max(0, (int)floorf((c + kCrHalfRange) * R.inv_cell)));
}

__device__ __forceinline__ int out_count(const FrameDev& F) { return F.cnt->n_out; }

// Class, looper flag, leg order key and circle centre of every output track;
// loopers are counted per (side block, centre bin).
__global__ void k_cr_tracks(FrameDev F, KParams P, RemovalParams R) {
  const int nt = out_count(F);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    const float* o = F.out_par + (long)t * 5;
    const int s = F.out_sector[t];
    const float q = o[4];
    const float side = (s % R.nsec_frame) < R.half ? 1.0f : -1.0f;
    F.cr_zk[t] = side * o[1];
    F.cr_cls[t] = fabsf(q) > R.qpt ? 1 : 0;
    F.cr_parent[t] = -1;
    // the curvature centre lies 1/kappa along the left normal of the direction
    const float rk = 1.0f / (P.kb * q);
    const float sn = o[2];
    const float cs = sqrtf(1.0f - sn * sn);
    const float xc = F.out_x[t] - sn * rk, yc = o[0] + cs * rk;
    const int a = s % 18;
    const float cx = xc * R.sec_cos[a] - yc * R.sec_sin[a];
    const float cy = xc * R.sec_sin[a] + yc * R.sec_cos[a];
    F.cr_cx[t] = cx;
    F.cr_cy[t] = cy;
    if (P.looper_qpt > 0.0f && fabsf(q) > P.looper_qpt) {
      const int b = ((s / R.half) * R.nbx + centre_bin(cy, R)) * R.nbx + centre_bin(cx, R);
      atomicAdd(&F.cr_bin_cnt[b], 1);
    }
  }
}

__device__ __forceinline__ int cr_bin(const FrameDev& F, const RemovalParams& R, int t) {
  return ((F.out_sector[t] / R.half) * R.nbx + centre_bin(F.cr_cy[t], R)) * R.nbx +
         centre_bin(F.cr_cx[t], R);
}

__device__ __forceinline__ bool is_looper(const FrameDev& F, const KParams& P, int t) {
  return P.looper_qpt > 0.0f && fabsf(F.out_par[(long)t * 5 + 4]) > P.looper_qpt;
}

// Loopers into their bins (bin order is irrelevant: the leg search takes a
// minimum over the whole neighbourhood).
__global__ void k_cr_scatter(FrameDev F, KParams P, RemovalParams R) {
  const int nt = out_count(F);
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += gridDim.x * blockDim.x) {
    if (!is_looper(F, P, t)) continue;
    const int b = cr_bin(F, R, t);
    F.cr_bin_items[F.cr_bin_first[b] + atomicSub(&F.cr_bin_cnt[b], 1) - 1] = t;
  }
}

// Secondary legs: the first earlier leg among the loopers of the 3 x 3
// neighbouring centre bins (bins are at least leg_dc wide).
__global__ void k_cr_legs(FrameDev F, KParams P, RemovalParams R) {
  const int nt = out_count(F);
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nt; a += gridDim.x * blockDim.x) {
    if (!is_looper(F, P, a)) continue;
    const float qa = F.out_par[(long)a * 5 + 4], ta = F.out_par[(long)a * 5 + 3];
    const float xa = F.cr_cx[a], ya = F.cr_cy[a], za = F.cr_zk[a];
    const float aa = fabsf(qa);
    const int ka = F.out_key[a];
    const int b0 = cr_bin(F, R, a);
    const int xb = b0 % R.nbx, yb = (b0 / R.nbx) % R.nbx;
    int best = -1, bk = 0;
    float bz = 0.0f;
    for (int e = -1; e <= 1; ++e) {
      if (yb + e < 0 || yb + e >= R.nbx) continue;
      // the three x bins of centre row yb + e are contiguous
      const int x0 = max(0, xb - 1), x1 = min(R.nbx - 1, xb + 1);
      const int row0 = b0 - xb + e * R.nbx;
      const int lo = F.cr_bin_first[row0 + x0], hi = F.cr_bin_first[row0 + x1 + 1];
      for (int j = lo; j < hi; ++j) {
        const int b = F.cr_bin_items[j];
        if (b == a) continue;
        const float qb = F.out_par[(long)b * 5 + 4];
        if ((qa > 0.0f) == (qb > 0.0f)) continue;
        const float ab = fabsf(qb);
        const float mx = aa > ab ? aa : ab;
        if (!(fabsf(aa - ab) <= R.leg_dq * mx)) continue;
        if (!(fabsf(ta + F.out_par[(long)b * 5 + 3]) <= R.leg_dtgl)) continue;
        const float dx = xa - F.cr_cx[b], dy = ya - F.cr_cy[b];
        if (!(dx * dx + dy * dy <= R.leg_dc * R.leg_dc)) continue;
        const float zb = F.cr_zk[b];
        const int kb = F.out_key[b];
        if (!(zb < za || (zb == za && kb < ka))) continue;
        if (best < 0 || zb < bz || (zb == bz && kb < bk)) {
          best = b;
          bz = zb;
          bk = kb;
        }
      }
    }
    if (best >= 0) {
      F.cr_parent[a] = best;
      F.cr_cls[a] = 2;
    }
  }
}

// One tube cross-section: the clusters of batch row rr within h of (yc, zc).
// Where protection 2 depends on the occupancy, one scan of the window that
// covers both the occupancy window and the larger of the two possible tubes
// counts the occupancy and lists the tube candidates (up to kCrList; a denser
// window is scanned again once h is known).
constexpr int kCrList = 12;

__device__ __forceinline__ void cr_tube(const FrameDev& F, const KParams& P,
                                        const RemovalParams& R, int rr, float yc, float zc,
                                        bool protect) {
  const int r = rr % P.n_rows;
  const RowGrid g = F.rows[rr];
  const float h0 = protect ? R.protect : R.remove;
  const float fac = protect ? R.p2_grow : R.p2_shrink;
  const unsigned bit = protect ? 1u : 4u;
  float h = h0;
  if (R.mode >= 2) {
    if (r < P.inner_rows || fabsf(yc) > F.row_x[r] * P.tan_half - R.edge) {
      h = h0 * fac;
    } else {
      const float w = R.occ_w;
      const float hg = h0 * fac;
      const float hm = hg > h0 ? hg : h0;  // the larger tube the occupancy may select
      const float wb = hm > w ? hm : w;
      int occ = 0, nc = 0;
      bool over = false;
      int cand[kCrList];
      for_window(F.bin_first, g, yc - wb, yc + wb, zc - wb, zc + wb, [&](int k) {
        const float2 pk = F.syz[k];
        const float dy = fabsf(pk.x - yc), dz = fabsf(pk.y - zc);
        if (dy <= w && dz <= w) ++occ;
        if (dy <= hm && dz <= hm) {
          if (nc < kCrList)
            cand[nc++] = k;
          else
            over = true;
        }
      });
      if (occ > R.occ_max) h = hg;
      if (!over) {
        for (int j = 0; j < nc; ++j) {
          const float2 pk = F.syz[cand[j]];
          if (fabsf(pk.x - yc) <= h && fabsf(pk.y - zc) <= h) atomicOr(&F.cr_flags[cand[j]], bit);
        }
        return;
      }
    }
  }
  for_window(F.bin_first, g, yc - h, yc + h, zc - h, zc + h, [&](int k) {
    const float2 pk = F.syz[k];
    if (fabsf(pk.x - yc) <= h && fabsf(pk.y - zc) <= h) atomicOr(&F.cr_flags[k], bit);
  });
}

// Tubes of every output track and the seeding history of the physics ones.
__global__ void k_cr_tubes(FrameDev F, KParams P, RemovalParams R) {
  const int nf = min(F.cnt->n_merged, (int)F.cap_ft);
  const int NR = P.n_rows;
  for (int f = blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += gridDim.x * blockDim.x) {
    const int t = F.ft_outidx[f];
    if (t < 0) continue;
    const bool protect = F.cr_cls[t] == 0;
    const int n = F.ft_n[f];
    if (n <= 0) continue;
    const int* used = F.ft_used + (long)f * kMaxRows;
    int crr = F.srow[used[0]];
    float2 pc = F.syz[used[0]];
    for (int i = 0; i < n; ++i) {
      // the next cluster is requested before this one's tube is scanned
      const int d = i + 1 < n ? used[i + 1] : -1;
      const int drr = d >= 0 ? F.srow[d] : -1;
      const float2 pd = d >= 0 ? F.syz[d] : make_float2(0.0f, 0.0f);
      cr_tube(F, P, R, crr, pc.x, pc.y, protect);
      if (d < 0) break;
      if (drr / NR == crr / NR) {
        const bool cl = crr < drr;  // interpolate from the lower-row cluster
        const int rl = (cl ? crr : drr) % NR, rh = (cl ? drr : crr) % NR;
        const float2 lo = cl ? pc : pd, hi = cl ? pd : pc;
        const int base = crr - crr % NR;
        for (int r = rl + 1; r < rh; ++r) {
          const float fr = (float)(r - rl) / (float)(rh - rl);
          cr_tube(F, P, R, base + r, lo.x + (hi.x - lo.x) * fr, lo.y + (hi.y - lo.y) * fr,
                  protect);
        }
      }
      crr = drr;
      pc = pd;
    }
    if (!protect) continue;
    for (int sg = F.ft_head[f]; sg >= 0; sg = F.st_next[sg]) {
      const int ti = F.st_tl[sg];
      const int* H = F.tl_hits + (long)ti * kMaxRows;
      for (int r = F.tl_rlo[ti]; r <= F.tl_rhi[ti]; ++r)
        if (H[r] >= 0) atomicOr(&F.cr_flags[H[r]], 2u);
    }
  }
}

// Removed = in a removal tube, neither protected nor history; flags out in
// input order, removed clusters counted.
__global__ void k_cr_final(FrameDev F) {
  for (long k = (long)blockIdx.x * blockDim.x + threadIdx.x; k < F.n;
       k += (long)gridDim.x * blockDim.x) {
    unsigned fl = F.cr_flags[k];
    const bool rem = (fl & 4u) && !(fl & 3u);
    if (rem) fl |= 8u;
    F.cr_out[F.sid[k]] = (uint8_t)fl;
    const unsigned m = __ballot_sync(__activemask(), rem);
    if (rem && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(&F.cnt->n_removed, __popc(m));
  }
}

}  // namespace

int cluster_removal(FrameDev& F, const KParams& P, const RemovalParams& R, int nblk, int sms,
                    cudaStream_t s) {
  const int nbins = nblk * R.nbx * R.nbx;
  const int g = sms * 8;
  k_cr_tracks<<<g, kBlock, 0, s>>>(F, P, R);
  int k = 1 + scan_exclusive(F.cr_bin_cnt, F.cr_bin_first, nbins + 1, F.scan_tmp, s);
  k_cr_scatter<<<g, kBlock, 0, s>>>(F, P, R);
  k_cr_legs<<<g, kBlock, 0, s>>>(F, P, R);
  k_cr_tubes<<<g, kBlock, 0, s>>>(F, P, R);
  k_cr_final<<<g, kBlock, 0, s>>>(F);
  return k + 4;
}

}  // namespace TPC_NS
}  // namespace tpc
