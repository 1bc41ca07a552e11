// Host-side launchers of the kernels.  The kernel translation units are
// compiled twice: into tpc::strict (no FMA contraction) and tpc::fast.
#pragma once

#include <cuda_runtime.h>

#include "tpc_internal.h"

namespace tpc {

// Each launcher enqueues one stage on stream s and returns its kernel count.
#define TPC_DECLARE_LAUNCHERS                                                       \
  void init_attributes();                                                          \
  int stage_grid(FrameDev& F, const KParams& P, int sms, cudaStream_t s);         \
  int stage_links(FrameDev& F, const KParams& P, int sms, cudaStream_t s);        \
  int stage_starts(FrameDev& F, const KParams& P, int sms, cudaStream_t s);       \
  int stage_tracklets(FrameDev& F, const KParams& P, int sms, cudaStream_t s);    \
  int stage_select(FrameDev& F, const KParams& P, int sms, cudaStream_t s);       \
  int stage_reseed(FrameDev& F, const KParams& P, int sms, cudaStream_t s);       \
  int stage_sector_refit(FrameDev& F, const KParams& P, int sms, cudaStream_t s);       \
  int stage_edge(FrameDev& F, const KParams& P, int sms, cudaStream_t s);               \
  int stage_merge(FrameDev& F, const KParams& P, int sms, cudaStream_t s);              \
  int stage_fit12(FrameDev& F, const KParams& P, int sms, cudaStream_t s);              \
  int stage_ambiguity2(FrameDev& F, const KParams& P, int sms, cudaStream_t s);         \
  int stage_fit3(FrameDev& F, const KParams& P, int sms, cudaStream_t s);               \
  int stage_output(FrameDev& F, const KParams& P, int sms, cudaStream_t s);             \
  int refit_forward(RefitDev& R, const KParams& P, int* steps3, int sms, cudaStream_t s); \
  int refit_backward(RefitDev& R, const KParams& P, const int* steps3, int sms,          \
                     cudaStream_t s);                                                    \
  int scan_exclusive(const int* in, int* out, long n, int* tmp, cudaStream_t s);           \
  int cluster_removal(FrameDev& F, const KParams& P, const RemovalParams& R, int nblk,     \
                      int sms, cudaStream_t s);

namespace strict {
TPC_DECLARE_LAUNCHERS
}
namespace fast {
TPC_DECLARE_LAUNCHERS
}

#undef TPC_DECLARE_LAUNCHERS

}  // namespace tpc
