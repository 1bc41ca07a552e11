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

constexpr float kCrHalfRange = 300.0f;  // circle centres binned over [-300, 300) cm

__device__ __forceinline__ int out_count(const FrameDev& F) { return F.cnt->n_out; }

// Class, looper flag, leg order key and circle centre of every output track;
// loopers are counted per (side block, centre-x bin).
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
      const int xb = min(R.nbx - 1, max(0, (int)floorf((cx + kCrHalfRange) * R.inv_cell)));
      atomicAdd(&F.cr_bin_cnt[(s / R.half) * R.nbx + xb], 1);
    }
  }
}

__device__ __forceinline__ int cr_bin(const FrameDev& F, const RemovalParams& R, int t) {
  const int xb = min(R.nbx - 1, max(0, (int)floorf((F.cr_cx[t] + kCrHalfRange) * R.inv_cell)));
  return (F.out_sector[t] / R.half) * R.nbx + xb;
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

// Secondary legs: the first earlier leg among the loopers of the three
// neighbouring centre-x bins (bins are at least leg_dc wide).
__global__ void k_cr_legs(FrameDev F, KParams P, RemovalParams R) {
  const int nt = out_count(F);
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < nt; a += gridDim.x * blockDim.x) {
    if (!is_looper(F, P, a)) continue;
    const float qa = F.out_par[(long)a * 5 + 4], ta = F.out_par[(long)a * 5 + 3];
    const float xa = F.cr_cx[a], ya = F.cr_cy[a], za = F.cr_zk[a];
    const float aa = fabsf(qa);
    const int ka = F.out_key[a];
    const int b0 = cr_bin(F, R, a);
    const int xb = b0 % R.nbx;
    int best = -1, bk = 0;
    float bz = 0.0f;
    for (int d = -1; d <= 1; ++d) {
      if (xb + d < 0 || xb + d >= R.nbx) continue;
      const int lo = F.cr_bin_first[b0 + d], hi = F.cr_bin_first[b0 + d + 1];
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
__device__ __forceinline__ void cr_tube(const FrameDev& F, const KParams& P,
                                        const RemovalParams& R, int rr, float yc, float zc,
                                        bool protect) {
  const int r = rr % P.n_rows;
  const RowGrid g = F.rows[rr];
  float h = protect ? R.protect : R.remove;
  if (R.mode >= 2) {
    bool dyn = r < P.inner_rows || fabsf(yc) > F.row_x[r] * P.tan_half - R.edge;
    if (!dyn) {
      const float w = R.occ_w;
      int occ = 0;
      for_window(F.bin_first, g, yc - w, yc + w, zc - w, zc + w, [&](int k) {
        const float2 pk = F.syz[k];
        if (fabsf(pk.x - yc) <= w && fabsf(pk.y - zc) <= w) ++occ;
      });
      dyn = occ > R.occ_max;
    }
    if (dyn) h = h * (protect ? R.p2_grow : R.p2_shrink);
  }
  const unsigned bit = protect ? 1u : 4u;
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
      cr_tube(F, P, R, crr, pc.x, pc.y, protect);
      if (i + 1 == n) break;
      const int d = used[i + 1];
      const int drr = F.srow[d];
      const float2 pd = F.syz[d];
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
  const int nbins = nblk * R.nbx;
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
