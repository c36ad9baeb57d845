// Split-precision (Ozaki-style) path: internal interface used by the C ABI.
#pragma once
#include <cstddef>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/lrbatch.h"
#include "lrb_internal.h"

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
// One 128 x 64 output tile of the split kernel with its entry's descriptor
// (64 bytes, so a tile is described by one record the kernel can prefetch).
struct STile {
    DevDesc d;
    int32_t entry, row0, col0, pad;
};
static_assert(sizeof(STile) == 64, "tile record layout");

// Tile list of a batch and the launch of the split kernel on uploaded tiles
// (used by the serving queue, whose waves live in stream-slot memory).
void build_items(const lrb_gemm_desc* descs, size_t count, std::vector<STile>& items);
cudaError_t launch_raw(int precision, const STile* d_items, int n_items, int* d_status, cudaStream_t s);
int chunk_len(int precision);
int digit_count(int precision);
void destroy(SplitPlan* p);

}  // namespace split
}  // namespace lrb
