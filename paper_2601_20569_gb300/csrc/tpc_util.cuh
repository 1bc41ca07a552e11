// Device helpers shared by the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include "tpc_internal.h"

namespace tpc {
namespace TPC_NS {
namespace {

constexpr int kBlock = 256;

__device__ __forceinline__ unsigned f2o(float f) {
  const unsigned u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float o2f(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

__device__ __forceinline__ int bin_of(float v, float v0, float inv, int n) {
  return clampi((int)floorf((v - v0) * inv), 0, n - 1);
}

// Visit sorted clusters of a row grid whose bins cover [ylo,yhi] x [zlo,zhi]
// (a superset of the clusters inside the box: bin index is monotone in the
// coordinate).
template <typename Fn>
__device__ __forceinline__ void for_window(const int* __restrict__ bin_first, const RowGrid& g,
                                           float ylo, float yhi, float zlo, float zhi, Fn&& fn) {
  if (g.ncl == 0 || !(ylo <= yhi) || !(zlo <= zhi)) return;
  const int iy0 = bin_of(ylo, g.y0, g.invDy, g.nY), iy1 = bin_of(yhi, g.y0, g.invDy, g.nY);
  const int iz0 = bin_of(zlo, g.z0, g.invDz, g.nZ), iz1 = bin_of(zhi, g.z0, g.invDz, g.nZ);
  for (int iz = iz0; iz <= iz1; ++iz) {
    const int b = g.bin0 + iz * g.nY;
    const int lo = bin_first[b + iy0], hi = bin_first[b + iy1 + 1];
    for (int k = lo; k < hi; ++k) fn(k);
  }
}

__device__ __forceinline__ int block_exscan(int v, int* sh_warp, int* total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh_warp[wid] = x;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int w = lane < nw ? sh_warp[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    if (lane < nw) sh_warp[lane] = w;
  }
  __syncthreads();
  const int base = wid ? sh_warp[wid - 1] : 0;
  if (total) *total = sh_warp[(blockDim.x >> 5) - 1];
  __syncthreads();
  return base + x - v;
}

// Exclusive scan of the block counts in one block; writes the total.
__global__ void k_scan_partials(int* part, int nparts, int* total) {
  __shared__ int sh[32];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nparts; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nparts ? part[i] : 0;
    int tot;
    const int ex = block_exscan(v, sh, &tot);
    if (i < nparts) part[i] = carry + ex;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Device-side work queue: each call hands the calling lanes the next item
// indices of the queue (one atomic per warp), so uneven items (tracklets of
// 3..150 rows, sectors of 10x different occupancy) balance dynamically across
// a persistent grid.
__device__ __forceinline__ int queue_next(int* q) {
  const unsigned mask = __activemask();
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(mask) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(q, __popc(mask));
  base = __shfl_sync(mask, base, leader);
  return base + __popc(mask & ((1u << lane) - 1u));
}

// Scheduling order from per-item buckets: order[start of bucket b + slot] = i
// for the first min(*n, cap) items.  Every block scans the kOrdBuckets counts
// in shared memory.  The order only decides which item a thread takes next;
// no result depends on it (slots within a bucket follow atomic arrival).
__global__ void k_order_scatter(const int* __restrict__ bucket, const int* __restrict__ slot,
                                const int* __restrict__ cnt, const int* n, long cap,
                                const int* err, int* __restrict__ order) {
  __shared__ int base[kOrdBuckets];
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int b = 0; b < kOrdBuckets; ++b) {
      base[b] = acc;
      acc += cnt[b];
    }
  }
  __syncthreads();
  if (*err) return;
  const int m = (int)min((long)*n, cap);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    order[base[bucket[i]] + slot[i]] = i;
}

}  // namespace

inline unsigned blocks_for(long n, int b) { return (unsigned)((n + b - 1) / b); }

// Persistent grid of a heavy kernel for launch slot `slot`.
inline unsigned persistent_grid(const LaunchCfg& lc, int slot, int sms) {
  return (unsigned)(sms * lc.per_sm[slot]);
}

}  // namespace TPC_NS
}  // namespace tpc
