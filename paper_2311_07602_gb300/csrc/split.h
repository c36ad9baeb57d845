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
                  lrb_plan_info* info, int test_stall = 0);
cudaError_t launch(SplitPlan* p, cudaStream_t s);
// Same launch, also writing every chunk's FP32 level sums to `dump`
// (float[chunks][S][m][n] for a single-entry plan) for the exactness test.
cudaError_t launch_dump(SplitPlan* p, float* dump, cudaStream_t s);
// Reads the plan's device status word (1 after a bounded wait expired).
int read_status(SplitPlan* p, cudaStream_t s, int* value);
int chunk_len(int precision);
int digit_count(int precision);
void destroy(SplitPlan* p);

}  // namespace split
}  // namespace lrb
