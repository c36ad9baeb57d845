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
// the GPU (calls on different streams) race on it, so callers must order
// them, e.g. on one stream.  A lock keeps each call's three enqueued steps
// (descriptor copy, tile kernel, persistent launch) together, so calls from
// several host threads on one stream stay whole and ordered.  The tile rule
// and tile extents are the planner's (checked on every call), so the tiles
// are those of a planned launch with untuned tiles (lrb_plan_create with
// tune = 0) on a batch big enough that the planner keeps its 64-row tiles.
// The first call on a device looks up the array's device
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

// Tile extents of the variants the untuned rule can pick (0..3), copied from
// the planner's variant table at set-up and passed to the tile kernel, so the
// tile list always matches the planner's tiles for those variants.
constexpr int kUntunedVariants = 4;
struct TileShapes {
    int bm[kUntunedVariants], bn[kUntunedVariants];
};

// One block of kTileThreads threads.  Each thread takes a run of consecutive
// entries, picks their variants (the planner's untuned rule, by output width)
// and counts their tiles; a block-wide scan of those counts gives every
// entry's first tile (kept in shared memory); then thread t writes tiles t,
// t + kTileThreads, ..., finding each tile's entry by binary search over the
// first-tile offsets, and thread 0 clears the work counter.
constexpr int kTileThreads = 256;
constexpr int kPerThread = (kMaxEntries + kTileThreads - 1) / kTileThreads;

__host__ __device__ __forceinline__ int noalloc_variant(int n) { return n <= 8 ? 0 : n <= 16 ? 1 : n <= 32 ? 2 : 3; }
inline int noalloc_variant_host(int n) { return noalloc_variant(n); }

__global__ void __launch_bounds__(kTileThreads) k_noalloc_tiles(const DevDesc* __restrict__ descs, int count,
                                                                TileShapes shp, Item* __restrict__ items,
                                                                int* __restrict__ head) {
    __shared__ int s_scan[kTileThreads];
    __shared__ int s_first[kMaxEntries + 1];
    const int t = threadIdx.x;
    const int e0 = min(count, t * kPerThread), e1 = min(count, e0 + kPerThread);
    int mine = 0;
    for (int e = e0; e < e1; ++e) {
        const int v = noalloc_variant(descs[e].n);
        mine += ((descs[e].m + shp.bm[v] - 1) / shp.bm[v]) * ((descs[e].n + shp.bn[v] - 1) / shp.bn[v]);
    }
    s_scan[t] = mine;
    __syncthreads();
    // inclusive scan (Hillis-Steele) over the per-thread tile counts
    for (int o = 1; o < kTileThreads; o <<= 1) {
        const int x = t >= o ? s_scan[t - o] : 0;
        __syncthreads();
        s_scan[t] += x;
        __syncthreads();
    }
    int first = s_scan[t] - mine;
    for (int e = e0; e < e1; ++e) {
        s_first[e] = first;
        const int v = noalloc_variant(descs[e].n);
        first += ((descs[e].m + shp.bm[v] - 1) / shp.bm[v]) * ((descs[e].n + shp.bn[v] - 1) / shp.bn[v]);
    }
    const int total = s_scan[kTileThreads - 1];
    if (t == 0) {
        s_first[count] = total;
        *head = 0;
    }
    __syncthreads();
    for (int i = t; i < total; i += kTileThreads) {
        int lo = 0, hi = count;          // the last entry e with s_first[e] <= i (entries of 0 tiles do not exist)
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (s_first[mid] <= i) lo = mid; else hi = mid;
        }
        const int e = lo, v = noalloc_variant(descs[e].n);
        const int bm = shp.bm[v], bn = shp.bn[v];
        const int tm = (descs[e].m + bm - 1) / bm, r = i - s_first[e];
        items[i] = Item{e, (r % tm) * bm, (r / tm) * bn, v};
    }
}

struct DeviceSetup {
    void* scratch = nullptr;
    int grid = 0;
};
std::mutex g_setup_mu;
DeviceSetup g_setup[128];
// Held while one call enqueues its copy, tile kernel and launch, so that two
// host threads calling on the same stream cannot interleave those three
// steps (each call's steps then stay together in stream order).
std::mutex g_enqueue_mu;

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
    TileShapes shp;
    for (int v = 0; v < kUntunedVariants; ++v) {
        shp.bm[v] = kVariants[v].bm();
        shp.bn[v] = kVariants[v].bn();
    }
    long long tiles = 0;
    for (size_t e = 0; e < count; ++e) {
        const lrb_gemm_desc& x = host_descs[e];
        const int v = untuned_variant(x.m, x.n, x.k);
        if (v < 0 || v >= kUntunedVariants || v != noalloc_variant_host(x.n)) {
            set_last_error("lrb_launch_noalloc: the planner's untuned tile rule changed; update the tile kernel");
            return LRB_ERR_UNSUPPORTED;
        }
        tiles += (long long)((x.m + shp.bm[v] - 1) / shp.bm[v]) * ((x.n + shp.bn[v] - 1) / shp.bn[v]);
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
    std::lock_guard<std::mutex> enqueue_lock(g_enqueue_mu);
    char* base = (char*)su.scratch;
    int* d_head = (int*)(base + kOffHead);
    DevDesc* d_descs = (DevDesc*)(base + kOffDescs);
    Item* d_items = (Item*)(base + kOffItems);
    cudaError_t e = cudaMemcpyAsync(d_descs, host_descs, sizeof(DevDesc) * count, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        k_noalloc_tiles<<<1, kTileThreads, 0, s>>>(d_descs, (int)count, shp, d_items, d_head);
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
