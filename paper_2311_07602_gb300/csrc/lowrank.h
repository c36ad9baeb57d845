// Producers and consumers of low-rank blocks (lowrank.cu): randomized SVD,
// expansion, rounded addition.  Each plan is a fixed sequence of batched
// kernels captured once as a CUDA graph.
#pragma once
#include "lrb_internal.h"

namespace lrb {
namespace lowrank {

struct LrPlan;

lrb_status create_rsvd(lrb_handle* h, const lrb_rsvd_desc* d, size_t count, int power_iters, LrPlan** out,
                       lrb_plan_info* info);
lrb_status create_expand(lrb_handle* h, const lrb_expand_desc* d, size_t count, LrPlan** out,
                         lrb_plan_info* info);
lrb_status create_round_add(lrb_handle* h, const lrb_round_add_desc* d, size_t count, LrPlan** out,
                            lrb_plan_info* info);
cudaError_t launch(LrPlan* p, cudaStream_t s);
// Synchronises `s` and reads the plan's status word (non-zero: a Jacobi SVD
// reached its sweep limit).  Returns 0 on success.
int read_status(LrPlan* p, cudaStream_t s, int* value);
void destroy(LrPlan* p);

}  // namespace lowrank
}  // namespace lrb
