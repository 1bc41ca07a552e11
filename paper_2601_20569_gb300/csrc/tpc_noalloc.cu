// Cellular-automaton neighbour links of one frame without any device
// allocation: every working buffer lives in one file-scope device array.
//
// Who needs this: callers that must not call cudaMalloc while they run, for
// example code executing inside a memory pool or allocator callback, an
// embedding runtime whose device memory is fully reserved up front, or an
// audited real-time loop where allocation latency and fragmentation are not
// allowed.  They pass device inputs and outputs; the scratch comes from a
// static __device__ array that every GPU loading this library keeps until
// process exit.
//
// Limits and sharing: at most kNoAllocMaxClusters clusters per call and
// n_sectors * n_rows <= kNoAllocMaxRows.  All calls share the one array and
// find the previous call's contents in it; what must start at zero is cleared
// at the start of every call.  Calls whose GPU work overlaps (two streams, two
// host threads) race on the array and must be serialised by the caller.  On a
// device, the first call looks up the array's device address
// (cudaGetSymbolAddress) with that device current; make that first call
// before any stream capture.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "tpc.h"
#include "tpc_internal.h"
#include "tpc_kernels.h"

namespace tpc {
void derive(KParams& P, const tpc_options& o, float bz, const std::vector<float>& row_x);
}

using namespace tpc;

namespace {

constexpr long kNoAllocMaxClusters = TPC_NOALLOC_MAX_CLUSTERS;
constexpr long kNoAllocMaxRows = 36 * kMaxRows;  // (sector, row) pairs
constexpr long kNoAllocBins = kNoAllocMaxClusters + kNoAllocMaxRows * 65;

constexpr long align256(long b) { return (b + 255) / 256 * 256; }

// Byte layout of the scratch array.
constexpr long kOffCnt = 0;
constexpr long kOffRowX = kOffCnt + align256(sizeof(Counters));
constexpr long kOffRowCnt = kOffRowX + align256(sizeof(float) * kMaxRows);
constexpr long kOffRowZmin = kOffRowCnt + align256(sizeof(int) * kNoAllocMaxRows);
constexpr long kOffRowZmax = kOffRowZmin + align256(sizeof(unsigned) * kNoAllocMaxRows);
constexpr long kOffRows = kOffRowZmax + align256(sizeof(unsigned) * kNoAllocMaxRows);
constexpr long kOffBinCnt = kOffRows + align256(sizeof(RowGrid) * kNoAllocMaxRows);
constexpr long kOffBinFirst = kOffBinCnt + align256(sizeof(int) * (kNoAllocBins + 1));
constexpr long kOffScanTmp = kOffBinFirst + align256(sizeof(int) * (kNoAllocBins + 1));
constexpr long kScanTmpInts = kNoAllocBins / 256 + 4096;
constexpr long kOffPerCl = kOffScanTmp + align256(sizeof(int) * kScanTmpInts);
constexpr long kPerClInts = 9;  // cl_bin, cl_slot, (y, z) [two slots], sid, lup, ldn, cup, cdn
constexpr long kOffSrow = kOffPerCl + kPerClInts * align256(4 * kNoAllocMaxClusters);
constexpr long kOffSrec = kOffSrow + align256(2 * kNoAllocMaxClusters);
constexpr long kOffRowFirst = kOffSrec + align256(16 * kNoAllocMaxClusters);
constexpr long kScratchBytes = kOffRowFirst + align256(sizeof(int) * (kNoAllocMaxRows + 1));

static_assert(kScratchBytes < (16L << 20), "no-allocation scratch must stay modest");
static_assert(align256(4 * kNoAllocMaxClusters) == 4 * kNoAllocMaxClusters,
              "the (y, z) pairs span two consecutive per-cluster slots");

// The scratch.  Host code must never use the symbol's host-side address: the
// device address is looked up per device below.
static __device__ __align__(256) unsigned char g_links_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[64] = {};

// Device address of the scratch on the current device (looked up once).
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_links_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

// Sorted-order links -> caller's input-id order.  Writes nothing when the grid
// build or the neighbour finding recorded an error: those kernels then leave
// the sorted arrays partly unwritten, holding an earlier call's ids, which may
// lie beyond this call's n.
__global__ void k_links_to_ids(const Counters* __restrict__ cnt, const int* __restrict__ sid,
                               const int* __restrict__ cup, const int* __restrict__ cdn, long n,
                               int32_t* up, int32_t* dn) {
  const long k = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n || cnt->err != 0) return;
  const int id = sid[k];
  const int u = cup[k], d = cdn[k];
  up[id] = u >= 0 ? sid[u] : -1;
  dn[id] = d >= 0 ? sid[d] : -1;
}

}  // namespace

extern "C" tpc_status tpc_links_noalloc(const tpc_geometry* geo, const tpc_options* opt,
                                        const tpc_clusters* cl, int32_t* link_up,
                                        int32_t* link_dn, void* cuda_stream) {
  if (!geo || !opt || !cl || !geo->row_x || cl->n < 0) return TPC_ERR_INVALID_ARG;
  if (geo->n_rows < 4 || geo->n_rows > kMaxRows || geo->n_sectors < 1 ||
      (long)geo->n_sectors * geo->n_rows > kNoAllocMaxRows)
    return TPC_ERR_INVALID_ARG;
  if (cl->n > kNoAllocMaxClusters) return TPC_ERR_CAPACITY;
  if (cl->n > 0 && (!cl->y || !cl->z || !cl->row || !cl->sector || !link_up || !link_dn))
    return TPC_ERR_INVALID_ARG;
  for (int r = 1; r < geo->n_rows; ++r)
    if (!(geo->row_x[r] > geo->row_x[r - 1])) return TPC_ERR_INVALID_ARG;
  void* base = nullptr;
  if (scratch_address(&base) != cudaSuccess) return TPC_ERR_CUDA;
  unsigned char* b = (unsigned char*)base;
  cudaStream_t s = (cudaStream_t)cuda_stream;

  KParams P{};
  std::vector<float> rx(geo->row_x, geo->row_x + geo->n_rows);
  derive(P, *opt, opt->bz, rx);
  P.n_rows = geo->n_rows;
  P.n_sectors = geo->n_sectors;
  P.n_phi = geo->n_sectors / 2 > 0 ? geo->n_sectors / 2 : 1;

  const long n = cl->n;
  const long nrr = (long)geo->n_sectors * geo->n_rows;
  FrameDev F{};
  for (int i = 0; i < kLNum; ++i) {
    F.lc.block[i] = 128;
    F.lc.per_sm[i] = 8;
    F.lc.lanes[i] = 1;
  }
  F.y = cl->y;
  F.z = cl->z;
  F.row = cl->row;
  F.sector = cl->sector;
  F.n = n;
  F.cnt = (Counters*)(b + kOffCnt);
  F.row_x = (const float*)(b + kOffRowX);
  F.row_cnt = (int*)(b + kOffRowCnt);
  F.row_zmin = (unsigned*)(b + kOffRowZmin);
  F.row_zmax = (unsigned*)(b + kOffRowZmax);
  F.rows = (RowGrid*)(b + kOffRows);
  F.bin_cnt = (int*)(b + kOffBinCnt);
  F.bin_first = (int*)(b + kOffBinFirst);
  F.cap_bins = kNoAllocBins;
  F.scan_tmp = (int*)(b + kOffScanTmp);
  int* per[kPerClInts];
  for (long i = 0; i < kPerClInts; ++i)
    per[i] = (int*)(b + kOffPerCl + i * align256(4 * kNoAllocMaxClusters));
  F.cl_bin = per[0];
  F.cl_slot = per[1];
  F.syz = (float2*)per[2];  // spans slots 2 and 3 (8 bytes per cluster)
  F.sid = per[4];
  F.lup = per[5];
  F.ldn = per[6];
  F.cup = per[7];
  F.cdn = per[8];
  F.srow = (uint16_t*)(b + kOffSrow);
  F.srec = (int4*)(b + kOffSrec);
  F.row_first = (int*)(b + kOffRowFirst);

  // clear what the grid build accumulates into; copy the geometry
  if (cudaMemsetAsync(F.cnt, 0, sizeof(Counters), s) != cudaSuccess ||
      cudaMemsetAsync(F.row_cnt, 0, sizeof(int) * nrr, s) != cudaSuccess ||
      cudaMemsetAsync(F.row_zmin, 0xFF, sizeof(unsigned) * nrr, s) != cudaSuccess ||
      cudaMemsetAsync(F.row_zmax, 0, sizeof(unsigned) * nrr, s) != cudaSuccess ||
      cudaMemsetAsync(F.bin_cnt, 0, sizeof(int) * (kNoAllocBins + 1), s) != cudaSuccess ||
      cudaMemcpyAsync((void*)F.row_x, geo->row_x, sizeof(float) * geo->n_rows,
                      cudaMemcpyHostToDevice, s) != cudaSuccess)
    return TPC_ERR_CUDA;
  int sms = 1;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  strict::stage_grid(F, P, sms > 0 ? sms : 1, s);
  strict::stage_links(F, P, sms > 0 ? sms : 1, s);
  if (n > 0)
    k_links_to_ids<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(F.cnt, F.sid, F.cup, F.cdn, n,
                                                                link_up, link_dn);
  if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
  Counters hc;
  if (cudaMemcpyAsync(&hc, F.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return TPC_ERR_CUDA;
  if (hc.err & (kErrInput | kErrDense)) return TPC_ERR_INVALID_INPUT;
  if (hc.err & kErrCapBins) return TPC_ERR_CAPACITY;
  return TPC_OK;
}
