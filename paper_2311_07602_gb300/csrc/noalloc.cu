// lrb_launch_noalloc: the persistent FP64 batch launch without any device
// allocation, for callers that cannot call cudaMalloc.
//
// Who needs it: programs whose GPU memory is owned up front by someone else
// (a framework's caching pool, a fixed budget set at start-up), and
// latency-critical loops that must not call cudaMalloc/cudaFree because
// those calls can synchronise the whole device.  Such callers already own
// A, B and C; what the planned path still allocates is its scratch -- the
// descriptor copy, the tile list and the work counter.  Here that scratch
// is one file-scope __device__ array of fixed size, so nothing is allocated
// at call time.
//
// Limits: at most kMaxEntries entries and kMaxTiles output tiles per call
// (about 4.2 MB of scratch, held by every GPU that loads the library until
// the process exits).  Every call shares the array: calls that overlap on
// the GPU (different streams, or another thread) race on it, so callers must
// order them.  The first call on a device looks up the array's device
// address (cudaGetSymbolAddress) and sets the kernel's shared-memory limit;
// make that first call before any stream capture.
#include <algorithm>
#include <cstdio>
#include <mutex>

#include "lrb_internal.h"

namespace lrb {
namespace {

constexpr int kMaxEntries = LRB_NOALLOC_MAX_ENTRIES;
constexpr int kMaxTiles = LRB_NOALLOC_MAX_TILES;
constexpr size_t kOffHead = 0;                                      // work counter
constexpr size_t kOffDescs = 256;                                   // kMaxEntries descriptors
constexpr size_t kOffItems = kOffDescs + sizeof(DevDesc) * kMaxEntries;  // kMaxTiles tiles
constexpr size_t kScratchBytes = kOffItems + sizeof(Item) * kMaxTiles;
static_assert(kOffItems % 256 == 0, "tile list alignment");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Untuned tile choice, the same rule as the planner's (by output width n).
__host__ __device__ inline int untuned_variant(int n) {
    return n <= 8 ? 0 : n <= 16 ? 1 : n <= 32 ? 2 : 3;
}
__host__ __device__ inline int variant_bm(int) { return 64; }
__host__ __device__ inline int variant_bn(int v) { return v == 0 ? 8 : v == 1 ? 16 : v == 2 ? 32 : 64; }

// One block: per-entry tile offsets (serial prefix in shared memory), then
// every thread writes tiles; clears the work counter.
__global__ void __launch_bounds__(256) k_noalloc_tiles(const DevDesc* __restrict__ descs, int count,
                                                       Item* __restrict__ items, int* __restrict__ head) {
    __shared__ int s_off[kMaxEntries + 1];
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int e = 0; e < count; ++e) {
            s_off[e] = acc;
            const int v = untuned_variant(descs[e].n);
            acc += ((descs[e].m + variant_bm(v) - 1) / variant_bm(v)) * ((descs[e].n + variant_bn(v) - 1) / variant_bn(v));
        }
        s_off[count] = acc;
        *head = 0;
    }
    __syncthreads();
    for (int e = 0; e < count; ++e) {
        const int v = untuned_variant(descs[e].n);
        const int bm = variant_bm(v), bn = variant_bn(v);
        const int tm = (descs[e].m + bm - 1) / bm;
        const int n_t = s_off[e + 1] - s_off[e];
        for (int t = threadIdx.x; t < n_t; t += blockDim.x)
            items[s_off[e] + t] = Item{e, (t % tm) * bm, (t / tm) * bn, v};
    }
}

struct DeviceSetup {
    void* scratch = nullptr;
    int grid = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[128];

}  // namespace
}  // namespace lrb

using namespace lrb;

extern "C" lrb_status lrb_launch_noalloc(const lrb_gemm_desc* host_descs, size_t count, void* stream) {
    char msg[160];
    if (count > (size_t)kMaxEntries) {
        std::snprintf(msg, sizeof msg, "lrb_launch_noalloc: %zu entries exceed the maximum of %d", count, kMaxEntries);
        set_last_error(msg);
        return LRB_ERR_INVALID;
    }
    lrb_status st = lrb_validate(host_descs, count, nullptr);
    if (st != LRB_OK) return st;
    long long tiles = 0;
    for (size_t e = 0; e < count; ++e) {
        const int v = untuned_variant(host_descs[e].n);
        tiles += (long long)((host_descs[e].m + variant_bm(v) - 1) / variant_bm(v)) *
                 ((host_descs[e].n + variant_bn(v) - 1) / variant_bn(v));
    }
    if (tiles > kMaxTiles) {
        std::snprintf(msg, sizeof msg, "lrb_launch_noalloc: %lld output tiles exceed the maximum of %d", tiles,
                      kMaxTiles);
        set_last_error(msg);
        return LRB_ERR_INVALID;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) {
        set_last_error("lrb_launch_noalloc: no current CUDA device");
        return LRB_ERR_DEVICE;
    }
    DeviceSetup su;
    {
        std::lock_guard<std::mutex> lock(g_setup_mu);
        if (!g_setup[dev].scratch) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                set_last_error("lrb_launch_noalloc: cudaGetSymbolAddress of the scratch array failed");
                return LRB_ERR_DEVICE;
            }
            const int per_sm = persistent_blocks_per_sm();   // also sets the kernel's shared-memory limit
            int sms = 0;
            if (per_sm <= 0 || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
                set_last_error("lrb_launch_noalloc: device set-up failed");
                return LRB_ERR_DEVICE;
            }
            g_setup[dev].grid = sms * per_sm;
            g_setup[dev].scratch = p;
        }
        su = g_setup[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    char* base = (char*)su.scratch;
    int* d_head = (int*)(base + kOffHead);
    DevDesc* d_descs = (DevDesc*)(base + kOffDescs);
    Item* d_items = (Item*)(base + kOffItems);
    cudaError_t e = cudaMemcpyAsync(d_descs, host_descs, sizeof(DevDesc) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_noalloc_tiles<<<1, 256, 0, s>>>(d_descs, (int)count, d_items, d_head);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        const int grid = (int)std::max<long long>(1, std::min<long long>(su.grid, tiles));
        e = launch_persistent(d_descs, d_items, (int)tiles, d_head, grid, s);
    }
    if (e != cudaSuccess) {
        std::snprintf(msg, sizeof msg, "lrb_launch_noalloc: %s", cudaGetErrorString(e));
        set_last_error(msg);
        return LRB_ERR_DEVICE;
    }
    return LRB_OK;
}
