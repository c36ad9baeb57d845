// Split-precision (Ozaki-style) path: internal interface used by the C ABI.
#pragma once
#include <cstddef>
#include <cuda_runtime.h>
#include "../../include/lrbatch.h"

namespace lrb {
namespace split {

struct SplitPlan;

// Builds the device work list for `count` entries at `precision`
// (LRB_PREC_SPLIT_*); fills items/grid/groups of *info.
lrb_status create(int device, int sms, const lrb_gemm_desc* descs, size_t count, int precision, SplitPlan** out,
                  lrb_plan_info* info);
cudaError_t launch(SplitPlan* p, cudaStream_t s);
void destroy(SplitPlan* p);

}  // namespace split
}  // namespace lrb
