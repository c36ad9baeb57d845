// Internal declarations shared by the library's translation units.
#pragma once
#include <cstdint>
#include <vector>
#include <cuda_runtime.h>
#include "../../include/lrbatch.h"

namespace lrb {

// Device copy of one entry; the same field layout as lrb_gemm_desc.  m, n, k
// are the product's sizes; with transposed forms lda / ldb describe the
// stored (transposed) operand.
struct DevDesc {
    const double* A;
    const double* B;
    double* C;
    int32_t m, n, k;
    int32_t lda, ldb, ldc;
};
static_assert(sizeof(DevDesc) == sizeof(lrb_gemm_desc), "descriptor layout");

// Device copy of one low-rank chain entry (same layout as lrb_lr_desc).
struct LrDesc {
    const double* AVT;
    const double* BU;
    const double* AX;
    const double* BX;
    double* G;
    int32_t ra, rb, k;
    int32_t ld_avt, ld_bu, ld_ax, ld_bx, ldg;
};
static_assert(sizeof(LrDesc) == sizeof(lrb_lr_desc), "chain descriptor layout");

// One output tile of one entry: rows [row0, row0+BM), cols [col0, col0+BN)
// of the variant's tile extent (clipped to the entry at run time).
struct Item {
    int32_t entry;
    int32_t row0;
    int32_t col0;
    int32_t variant;
};

// FP64 tile variants.  128 threads = 4 warps per CTA.
//  DFMA variants: lanes run along rows (row = lane + 32 i, i < TM), warps
//  along columns (WN groups of TN columns) and along k (SK groups that split
//  each k-step and are summed at the end).  BM = 32 TM, BN = WN TN.
//  DMMA variants: FP64 tensor-core m8n8k4 fragments; each warp owns 16 rows
//  of a 64 x BN tile.
struct Variant {
    int tm, tn, wn, sk, dmma;
    int bm() const { return dmma ? 64 : 32 * tm; }
    int bn() const { return dmma ? 8 * tn : wn * tn; }
};

constexpr int kThreads = 128;
constexpr int kBK = 16;          // k-step staged in shared memory
constexpr int kNumVariants = 10;

// Host-side copy of the variant table (same order as the device dispatch).
extern const Variant kVariants[kNumVariants];

size_t variant_smem_bytes(int v);
size_t max_smem_bytes();

// Kernel launchers (fp64_tiles.cu).
// set: the variant set of the persistent kernel (variant_set); 0 slim (5
// CTAs per SM), 1 narrow (3 CTAs, the default), 2 wide (every variant).
// ops: operand forms (bit 0 A^T, bit 1 B^T, bit 2 overwrite C), slim set only.
cudaError_t launch_persistent(const DevDesc* d_descs, const Item* d_items, int n_items,
                              int* d_head, int grid, cudaStream_t s, int set = 1, int ops = 0);
cudaError_t launch_plain_group(int variant, const DevDesc* d_descs, const int32_t* d_entries,
                               int n_entries, int tiles_m, int tiles_n, cudaStream_t s);
int persistent_blocks_per_sm(int set = 1);
int variant_set(int v);

// Fused low-rank chain (lr_chain.cu).
// rmax: the plan's largest rank (sizes the kernel's registers and staging).
size_t lr_chain_smem_bytes_for(int stage);
int lr_chain_max_rank();
cudaError_t launch_lr_chain(const LrDesc* d_descs, int count, int rmax, cudaStream_t s);

// Sets the calling thread's lrb_last_error() message (api.cu).
void set_last_error(const char* msg);

// Planner pieces (api.cu) used by the serving queue.
struct HandleInfo {
    int device, sms, blocks_per_sm, blocks_per_sm_wide, blocks_per_sm_slim;
};
HandleInfo handle_info(const lrb_handle* h);
lrb_plan_opts default_plan_opts();
lrb_status validate_descs(const lrb_gemm_desc* d, size_t count, const lrb_plan_opts& o);
// Tile variant per entry (tuned-cache lookup, else tuning or the heuristic as o.tune says).
lrb_status plan_variants(lrb_handle* h, const lrb_gemm_desc* d, size_t count, const lrb_plan_opts& o,
                         std::vector<int>& var);
// Enqueues an FP64 plan's persistent launch on `s` (no device switch: safe
// inside a stream capture); cudaErrorInvalidValue for other plan kinds.
cudaError_t enqueue_fp64_plan(lrb_plan* p, cudaStream_t s);
// The planner's tile variant for an entry when nothing is tuned (by output
// width: 64 x 8, 64 x 16, 64 x 32 or 64 x 64 tiles, variants 0..3).
int untuned_variant(int m, int n, int k);
// Output tiles of all entries, longest first.
void plan_tiles(const lrb_gemm_desc* d, size_t count, const std::vector<int>& var, std::vector<Item>& items);

}  // namespace lrb
