// Split-precision path (placeholder until the tensor-core kernel lands).
#include "split.h"

namespace lrb {
namespace split {

struct SplitPlan {
    int unused;
};

lrb_status create(int, int, const lrb_gemm_desc*, size_t, int, SplitPlan** out, lrb_plan_info*) {
    *out = nullptr;
    return LRB_ERR_UNSUPPORTED;
}
cudaError_t launch(SplitPlan*, cudaStream_t) { return cudaErrorNotSupported; }
void destroy(SplitPlan* p) { delete p; }

}  // namespace split
}  // namespace lrb
