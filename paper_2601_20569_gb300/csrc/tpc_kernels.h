// Host-side launchers of the kernels.  The kernel translation units are
// compiled twice: into tpc::strict (no FMA contraction) and tpc::fast.
#pragma once

#include <cuda_runtime.h>

#include "tpc_internal.h"

namespace tpc {

#define TPC_DECLARE_LAUNCHERS                                                        \
  void sector_tracking(FrameDev& F, const KParams& P, int sms, cudaStream_t s);    \
  void scan_exclusive(const int* in, int* out, long n, int* tmp, cudaStream_t s);

namespace strict {
TPC_DECLARE_LAUNCHERS
}
namespace fast {
TPC_DECLARE_LAUNCHERS
}

#undef TPC_DECLARE_LAUNCHERS

}  // namespace tpc
