// C ABI: handles, argument validation, the planner (tiles, longest-first
// order, plain-launch groups), the tile autotuner and CUDA-graph capture.
//
// The batch is a list of independent entries, as in the paper's batched
// low-rank multiplication (Alg. 2, loop 1 runs over independent blocks).  On
// the CPU the paper splits that loop across cores and packs operands into
// caches (Alg. 3); here every entry is cut into output tiles and one
// persistent kernel pulls tiles from a device-side counter, largest first.
#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <new>
#include <queue>
#include <sstream>
#include <string>
#include <tuple>
#include <vector>

#include "lrb_internal.h"
#include "lowrank.h"
#include "split.h"

using namespace lrb;

namespace {

thread_local std::string g_err;

lrb_status fail(lrb_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

lrb_status cuda_fail(cudaError_t e, const char* what) {
    return fail(LRB_ERR_DEVICE, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LRB_CUDA(call)                                   \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
    } while (0)

lrb_plan_opts default_opts() {
    lrb_plan_opts o;
    std::memset(&o, 0, sizeof(o));
    o.precision = LRB_PREC_FP64;
    o.use_graph = 0;
    o.tune = 1;
    o.force_variant = -1;
    o.check_alias = 1;
    return o;
}

// Byte range [lo, hi) covered by a column-major rows x cols matrix.
struct Range {
    uint64_t lo, hi;
    int64_t entry;
};

bool extent(const void* p, int32_t rows, int32_t cols, int32_t ld, Range* r) {
    // last element index = ld * (cols - 1) + rows - 1, all non-negative here
    const __int128 last = (__int128)ld * (cols - 1) + rows - 1;
    const __int128 bytes = (last + 1) * 8;
    const __int128 lo = (__int128)(uintptr_t)p;
    if (bytes > ((__int128)1 << 62) || lo + bytes > ((__int128)1 << 64) - 1) return false;
    r->lo = (uint64_t)lo;
    r->hi = (uint64_t)(lo + bytes);
    return true;
}

lrb_status validate(const lrb_gemm_desc* d, size_t count, const lrb_plan_opts& o) {
    if (!d) return fail(LRB_ERR_INVALID, "host_descs is NULL");
    if (count == 0) return fail(LRB_ERR_INVALID, "count is 0");
    if (count > 0x7fffffffull) return fail(LRB_ERR_INVALID, "count exceeds 2^31-1");
    if (o.precision < LRB_PREC_FP64 || o.precision > LRB_PREC_SPLIT_FP16_S4)
        return fail(LRB_ERR_INVALID, "unknown precision");
    if (o.force_variant >= kNumVariants) return fail(LRB_ERR_INVALID, "force_variant out of range");
    if (o.trans < 0 || o.trans > 3) return fail(LRB_ERR_INVALID, "trans must be 0..3");
    if (o.overwrite < 0 || o.overwrite > 1) return fail(LRB_ERR_INVALID, "overwrite must be 0 or 1");
    const bool ta = (o.trans & 1) != 0, tb = (o.trans & 2) != 0;
    std::vector<Range> cr, ab;
    if (o.check_alias) {
        cr.reserve(count);
        ab.reserve(2 * count);
    }
    for (size_t e = 0; e < count; ++e) {
        const lrb_gemm_desc& x = d[e];
        char buf[160];
        if (!x.A || !x.B || !x.C) {
            std::snprintf(buf, sizeof buf, "entry %zu: NULL operand pointer", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        if (((uintptr_t)x.A | (uintptr_t)x.B | (uintptr_t)x.C) & 7u) {
            std::snprintf(buf, sizeof buf, "entry %zu: operand pointer not 8-byte aligned", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        if (x.m <= 0 || x.n <= 0 || x.k <= 0) {
            std::snprintf(buf, sizeof buf, "entry %zu: m, n, k must be >= 1 (got %d, %d, %d)", e, x.m, x.n, x.k);
            return fail(LRB_ERR_INVALID, buf);
        }
        // stored operands: A is m x k (k x m when transposed), B k x n (n x k)
        const int32_t ar = ta ? x.k : x.m, ac = ta ? x.m : x.k;
        const int32_t br = tb ? x.n : x.k, bc = tb ? x.k : x.n;
        if (x.lda < ar || x.ldb < br || x.ldc < x.m) {
            std::snprintf(buf, sizeof buf, "entry %zu: leading dimension below rows (lda %d, ldb %d, ldc %d)", e,
                          x.lda, x.ldb, x.ldc);
            return fail(LRB_ERR_INVALID, buf);
        }
        Range ra, rb, rc;
        if (!extent(x.A, ar, ac, x.lda, &ra) || !extent(x.B, br, bc, x.ldb, &rb) ||
            !extent(x.C, x.m, x.n, x.ldc, &rc)) {
            std::snprintf(buf, sizeof buf, "entry %zu: operand extent overflows", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        if (o.check_alias) {
            ra.entry = rb.entry = rc.entry = (int64_t)e;
            cr.push_back(rc);
            ab.push_back(ra);
            ab.push_back(rb);
        }
    }
    if (o.check_alias) {
        std::sort(cr.begin(), cr.end(), [](const Range& a, const Range& b) { return a.lo < b.lo; });
        for (size_t i = 1; i < cr.size(); ++i)
            if (cr[i].lo < cr[i - 1].hi) {
                char buf[160];
                std::snprintf(buf, sizeof buf, "C of entries %lld and %lld overlap", (long long)cr[i - 1].entry,
                              (long long)cr[i].entry);
                return fail(LRB_ERR_ALIAS, buf);
            }
        for (const Range& r : ab) {
            // first C range whose end is beyond r.lo
            auto it = std::upper_bound(cr.begin(), cr.end(), r.lo,
                                       [](uint64_t v, const Range& c) { return v < c.hi; });
            if (it != cr.end() && it->lo < r.hi) {
                char buf[160];
                std::snprintf(buf, sizeof buf, "an operand of entry %lld overlaps C of entry %lld",
                              (long long)r.entry, (long long)it->entry);
                return fail(LRB_ERR_ALIAS, buf);
            }
        }
    }
    return LRB_OK;
}

int ceil_div(int a, int b) { return (a + b - 1) / b; }

// Issued multiply-adds of one tile (rows rounded up to whole 32-row slots,
// DMMA fragments rounded to 8), the planner's cost for longest-first order.
double tile_cost(const Variant& V, int h, int w, int k) {
    if (V.dmma) return (double)(ceil_div(h, 8) * 8) * (ceil_div(w, 8) * 8) * (ceil_div(k, 4) * 4);
    return (double)(ceil_div(h, 32) * 32) * w * k;
}

struct Group {
    int variant, m, n, k, tiles_m, tiles_n;
    int offset, count;
};

void make_tiles(const lrb_gemm_desc* d, size_t count, const std::vector<int>& var, std::vector<Item>& items) {
    struct Keyed {
        double cost;
        Item it;
    };
    std::vector<Keyed> tmp;
    for (size_t e = 0; e < count; ++e) {
        const Variant& V = kVariants[var[e]];
        const int bm = V.bm(), bn = V.bn();
        for (int c0 = 0; c0 < d[e].n; c0 += bn)
            for (int r0 = 0; r0 < d[e].m; r0 += bm) {
                const int h = std::min(bm, d[e].m - r0), w = std::min(bn, d[e].n - c0);
                tmp.push_back({tile_cost(V, h, w, d[e].k), Item{(int32_t)e, r0, c0, var[e]}});
            }
    }
    std::stable_sort(tmp.begin(), tmp.end(), [](const Keyed& a, const Keyed& b) { return a.cost > b.cost; });
    items.resize(tmp.size());
    for (size_t i = 0; i < tmp.size(); ++i) items[i] = tmp[i].it;
}

int bucket(int x) { return (int)std::floor(2.0 * std::log2((double)x) + 1e-9); }
int bucket_center(int b) { return std::max(1, (int)std::lround(std::pow(2.0, (b + 0.5) / 2.0))); }

int heuristic_variant(int m, int n, int k, bool dmma_ok) {
    (void)m;
    (void)k;
    (void)dmma_ok;
    if (n <= 8) return 0;
    if (n <= 16) return 1;
    if (n <= 32) return 2;
    return 3;
}

}  // namespace

namespace {
// lrb_execute_host merges the copies of blocks that lie at most this many
// elements apart in host memory (256 bytes: the alignment padding between
// blocks laid out back to back); the bytes between them are copied in and,
// for C, written back unchanged.
constexpr ptrdiff_t kGapElems = 32;
// A shared operand region is copied in pieces of at most this many elements.
constexpr size_t kRegionChunkElems = (size_t)32 << 20;

// Summary of one timed lrb_execute_host call from per-piece intervals (ms from
// the call's start) of the three engines: 0 copies in, 1 launches, 2 copies out.
// Busy time = length of an engine's union of intervals; overlap of two engines
// = length of the intersection of their unions.
lrb_host_timing summarize_host_timing(std::vector<std::pair<double, double>> (&iv)[3], int pieces, double h2d_bytes,
                                      double d2h_bytes, double first_h2d_bytes) {
    std::vector<std::pair<double, double>> u[3];
    for (int c = 0; c < 3; ++c) {
        std::vector<std::pair<double, double>> v = iv[c];
        std::sort(v.begin(), v.end());
        for (const auto& x : v) {
            if (x.second <= x.first) continue;
            if (!u[c].empty() && x.first <= u[c].back().second)
                u[c].back().second = std::max(u[c].back().second, x.second);
            else
                u[c].push_back(x);
        }
    }
    auto length = [](const std::vector<std::pair<double, double>>& a) {
        double t = 0;
        for (const auto& x : a) t += x.second - x.first;
        return t;
    };
    auto overlap = [](const std::vector<std::pair<double, double>>& a, const std::vector<std::pair<double, double>>& b) {
        double t = 0;
        size_t i = 0, j = 0;
        while (i < a.size() && j < b.size()) {
            const double lo = std::max(a[i].first, b[j].first), hi = std::min(a[i].second, b[j].second);
            if (hi > lo) t += hi - lo;
            if (a[i].second < b[j].second) ++i; else ++j;
        }
        return t;
    };
    lrb_host_timing t{};
    t.valid = 1;
    t.pieces = pieces;
    double lo = 1e300, hi = 0;
    for (int c = 0; c < 3; ++c)
        for (const auto& x : u[c]) {
            lo = std::min(lo, x.first);
            hi = std::max(hi, x.second);
        }
    t.wall_ms = hi > lo ? hi - lo : 0.0;
    t.h2d_busy_ms = length(u[0]);
    t.compute_busy_ms = length(u[1]);
    t.d2h_busy_ms = length(u[2]);
    t.h2d_bytes = h2d_bytes;
    t.d2h_bytes = d2h_bytes;
    t.overlap_h2d_compute_ms = overlap(u[0], u[1]);
    t.overlap_d2h_compute_ms = overlap(u[2], u[1]);
    t.overlap_h2d_d2h_ms = overlap(u[0], u[2]);
    t.compute_start_ms = u[1].empty() ? 0.0 : u[1].front().first - lo;
    t.compute_end_to_last_ms = u[1].empty() ? 0.0 : hi - u[1].back().second;
    t.first_h2d_ms = iv[0].empty() ? 0.0 : iv[0].front().second - iv[0].front().first;
    t.first_h2d_bytes = first_h2d_bytes;
    return t;
}

// One host<->device copy of lrb_execute_host: a 2-D block, or a merged 1-D run.
struct HostCopy {
    const double* host;
    size_t dev;        // element offset in the arena
    int rows, cols, ld;
    size_t elems;      // contiguous run length (tight blocks)
};
}  // namespace

struct lrb_handle {
    int device = 0;
    int sms = 0;
    int blocks_per_sm = 0;        // narrow persistent kernel (variant set 1)
    int blocks_per_sm_wide = 0;   // wide persistent kernel (set 2)
    int blocks_per_sm_slim = 0;   // slim persistent kernel (set 0)
    std::string gpu_key;
    std::string cache_path;
    std::map<std::string, int> tuned;
    std::mutex mu;
    cudaStream_t stream = nullptr;   // tuning and graph capture
    void* scratch = nullptr;          // tuning buffers
    size_t scratch_bytes = 0;
    // lrb_execute_host: device arena and the plan cached for the last shape list
    void* arena = nullptr;
    size_t arena_bytes = 0;
    std::vector<lrb_gemm_desc> host_key;
    std::vector<size_t> host_cut;
    // the caller's last host descriptor array and its copy lists: a repeated
    // batch skips validation, layout and planning
    std::vector<lrb_gemm_desc> host_in;
    std::vector<std::vector<HostCopy>> host_h2d, host_d2h;
    lrb_plan_opts host_opts{};
    std::vector<lrb_plan*> host_plans;
    cudaStream_t copy_in = nullptr, copy_out = nullptr, compute2 = nullptr;
    std::vector<cudaEvent_t> ev_in, ev_done;
    cudaEvent_t ev_join = nullptr;
    // optional per-piece timing of lrb_execute_host (lrb_execute_host_set_timing):
    // per piece, start/end of its copies in, its launch and its copies out
    bool timing = false;
    std::vector<cudaEvent_t> tev;     // 6 per piece
    cudaEvent_t tev0 = nullptr;       // the call's start, on the caller's stream
    lrb_host_timing last_timing{};
};

struct lrb_multi_plan {
    std::vector<lrb_plan*> plans;     // one per handle (NULL: the part got no entries)
    std::vector<int64_t> entries;
    std::vector<int> devices;
};

struct lrb_plan {
    lrb_handle* h = nullptr;
    int precision = LRB_PREC_FP64;
    std::vector<lrb_gemm_desc> descs;
    void* dmem = nullptr;
    DevDesc* d_descs = nullptr;
    Item* d_items = nullptr;
    int32_t* d_group_entries = nullptr;
    int* d_head = nullptr;
    int n_items = 0;
    int grid = 0;
    int set = 0;         // variant set of the persistent kernel (largest set of any tile)
    int ops = 0;         // operand forms: bit 0 A^T, bit 1 B^T, bit 2 overwrite C (slim set only)
    std::vector<Group> groups;
    bool use_graph = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t last_stream = nullptr;
    bool launched = false;
    lrb_plan_info info{};
    split::SplitPlan* sp = nullptr;
    // low-rank chain plans
    int lr_kind = 0;                   // 0: none, 1: fused, 2: unfused (three batched products)
    LrDesc* d_lr = nullptr;
    int lr_count = 0;
    int lr_rmax = 0;                   // largest rank of any block (sizes the fused kernel)
    void* lr_work = nullptr;           // unfused: C_temp and E_temp of every block
    size_t lr_work_bytes = 0;
    lrb_plan* lr_stage[3] = {nullptr, nullptr, nullptr};
    // producer / consumer plans of low-rank blocks (randomized SVD, expansion, rounded addition)
    lowrank::LrPlan* lp = nullptr;
};

namespace {

std::string bucket_key(int m, int n, int k, bool dmma_ok) {
    char buf[64];
    std::snprintf(buf, sizeof buf, "m%d_n%d_k%d_%s", bucket(m), bucket(n), bucket(k), dmma_ok ? "dmma" : "dfma");
    return buf;
}

void load_cache(lrb_handle* h) {
    if (h->cache_path.empty()) return;
    std::ifstream f(h->cache_path);
    if (!f) return;
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    // {"gpu": "<key>", "buckets": {"<bucket>": <variant>, ...}}
    const std::string gk = "\"gpu\": \"" + h->gpu_key + "\"";
    if (s.find(gk) == std::string::npos) return;   // another GPU / driver / version: ignore
    size_t p = s.find("\"buckets\"");
    if (p == std::string::npos) return;
    p = s.find('{', p);
    while (p != std::string::npos) {
        size_t q0 = s.find('"', p + 1);
        if (q0 == std::string::npos) break;
        size_t q1 = s.find('"', q0 + 1);
        if (q1 == std::string::npos) break;
        size_t c = s.find(':', q1);
        if (c == std::string::npos) break;
        const int v = std::atoi(s.c_str() + c + 1);
        if (v >= 0 && v < kNumVariants) h->tuned[s.substr(q0 + 1, q1 - q0 - 1)] = v;
        p = s.find(',', c);
    }
}

void save_cache(lrb_handle* h) {
    if (h->cache_path.empty()) return;
    const std::string tmp = h->cache_path + ".tmp";
    {
        std::ofstream f(tmp);
        if (!f) return;
        f << "{\"gpu\": \"" << h->gpu_key << "\", \"buckets\": {";
        bool first = true;
        for (auto& kv : h->tuned) {
            f << (first ? "" : ", ") << "\"" << kv.first << "\": " << kv.second;
            first = false;
        }
        f << "}}\n";
    }
    std::rename(tmp.c_str(), h->cache_path.c_str());
}

// Time each candidate variant on a uniform batch of the bucket's central
// shape in the kernel a tuned plan runs -- the slim persistent kernel, 5 CTAs
// per SM, pulling tiles from a counter -- one warm-up launch and the best of
// two timed ones, and keep the fastest.  The batch has about 3 GFLOP and at
// least four waves of the persistent grid for every candidate (so tall tiles
// are not charged for a partly empty last wave that a large batch would not
// have); its operands are zeros in the handle's scratch buffer (at most 1 GB).
lrb_status tune_bucket(lrb_handle* h, int m, int n, int k, bool dmma_ok, int* best) {
    const int M = bucket_center(bucket(m)), N = bucket_center(bucket(n)), K = bucket_center(bucket(k));
    const double flops_entry = 2.0 * M * N * K;
    const double bytes_entry = 8.0 * ((double)M * K + (double)K * N + (double)M * N);
    *best = heuristic_variant(m, n, k, dmma_ok);
    std::vector<int> cand;
    for (int v = 0; v < kNumVariants; ++v) {
        const Variant& V = kVariants[v];
        if (variant_set(v) != 0) continue;   // tuned plans run in the slim persistent kernel (5 CTAs/SM)
        if (V.dmma && !dmma_ok) continue;
        // skip tiles more than twice as tall/wide as the shape needs
        if (V.bm() > 32 && V.bm() >= 2 * std::max(M, 32)) continue;
        if (V.bn() > 8 && V.bn() >= 2 * std::max(N, 8)) continue;
        cand.push_back(v);
    }
    if (cand.empty()) return LRB_OK;
    const int grid_full = std::max(1, h->sms * h->blocks_per_sm_slim);
    long long min_tiles = LLONG_MAX, max_tiles = 0;
    for (int v : cand) {
        const long long t = (long long)ceil_div(M, kVariants[v].bm()) * ceil_div(N, kVariants[v].bn());
        min_tiles = std::min(min_tiles, t);
        max_tiles = std::max(max_tiles, t);
    }
    long long E = (long long)std::ceil(3e9 / flops_entry);
    E = std::max(E, (4LL * grid_full + min_tiles - 1) / min_tiles);
    E = std::min(E, std::max(1LL, (long long)(1e9 / bytes_entry)));
    E = std::max(E, 1LL);
    const size_t op_bytes = (size_t)(bytes_entry * (double)E);
    const size_t desc_off = (op_bytes + 255) & ~(size_t)255;
    const size_t item_off = (desc_off + sizeof(DevDesc) * (size_t)E + 255) & ~(size_t)255;
    const size_t head_off = (item_off + sizeof(Item) * (size_t)(E * max_tiles) + 255) & ~(size_t)255;
    const size_t need = head_off + 256;
    if (need > h->scratch_bytes) {
        if (h->scratch) cudaFree(h->scratch);
        h->scratch = nullptr;
        h->scratch_bytes = 0;
        LRB_CUDA(cudaMalloc(&h->scratch, need));
        h->scratch_bytes = need;
    }
    char* base = (char*)h->scratch;
    LRB_CUDA(cudaMemsetAsync(base, 0, op_bytes, h->stream));
    std::vector<DevDesc> dd((size_t)E);
    double* A = (double*)base;
    double* B = A + (size_t)M * K * E;
    double* C = B + (size_t)K * N * E;
    for (long long e = 0; e < E; ++e)
        dd[e] = DevDesc{A + (size_t)M * K * e, B + (size_t)K * N * e, C + (size_t)M * N * e, M, N, K, M, K, M};
    DevDesc* d_dd = (DevDesc*)(base + desc_off);
    Item* d_items = (Item*)(base + item_off);
    int* d_head = (int*)(base + head_off);
    LRB_CUDA(cudaMemcpyAsync(d_dd, dd.data(), sizeof(DevDesc) * (size_t)E, cudaMemcpyHostToDevice, h->stream));
    cudaEvent_t e0, e1;
    LRB_CUDA(cudaEventCreate(&e0));
    LRB_CUDA(cudaEventCreate(&e1));
    auto fail_with = [&](cudaError_t ce, const char* what) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(ce, what);
    };
    float best_ms = 1e30f;
    std::vector<Item> items;
    for (int v : cand) {
        const Variant& V = kVariants[v];
        const int bm = V.bm(), bn = V.bn();
        // the tiles in the planner's order: longest first (full tiles before edge tiles)
        items.clear();
        std::vector<double> cost;
        for (long long e = 0; e < E; ++e)
            for (int c0 = 0; c0 < N; c0 += bn)
                for (int r0 = 0; r0 < M; r0 += bm) {
                    items.push_back(Item{(int32_t)e, r0, c0, v});
                    cost.push_back(tile_cost(V, std::min(bm, M - r0), std::min(bn, N - c0), K));
                }
        std::vector<size_t> order(items.size());
        for (size_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](size_t x, size_t y) { return cost[x] > cost[y]; });
        std::vector<Item> sorted(items.size());
        for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
        items.swap(sorted);
        const int n_items = (int)items.size();
        cudaError_t ce = cudaMemcpyAsync(d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice,
                                         h->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(h->stream);   // items is reused for the next candidate
        if (ce != cudaSuccess) return fail_with(ce, "tuning upload");
        const int grid = std::max(1, std::min(grid_full, n_items));
        ce = launch_persistent(d_dd, d_items, n_items, d_head, grid, h->stream, 0, 0);
        if (ce != cudaSuccess) return fail_with(ce, "tuning launch");
        float ms_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, h->stream);
            launch_persistent(d_dd, d_items, n_items, d_head, grid, h->stream, 0, 0);
            cudaEventRecord(e1, h->stream);
            ce = cudaEventSynchronize(e1);
            if (ce != cudaSuccess) return fail_with(ce, "tuning run");
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_min = std::min(ms_min, ms);
        }
        if (ms_min < best_ms) {
            best_ms = ms_min;
            *best = v;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return LRB_OK;
}

// One persistent launch of the entries with tile variants `var` (all in the
// slim set), on the entries' own A and B and a scratch C (tight, zeroed: the
// caller's C is not touched): the best of three timed launches after a
// warm-up, in ms.  Used to choose between near-tied tilings of small plans.
lrb_status time_plan_tiles(lrb_handle* h, const lrb_gemm_desc* d, size_t count, const std::vector<int>& var,
                           float* ms_out) {
    std::vector<Item> items;
    make_tiles(d, count, var, items);
    std::vector<size_t> coff(count);
    size_t c_elems = 0;
    for (size_t e = 0; e < count; ++e) {
        coff[e] = c_elems;
        c_elems += ((size_t)d[e].m * (size_t)d[e].n + 31) / 32 * 32;
    }
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    const size_t o_desc = up(8 * c_elems), o_items = o_desc + up(sizeof(DevDesc) * count);
    const size_t o_head = o_items + up(sizeof(Item) * items.size()), total = o_head + 256;
    void* mem = nullptr;
    LRB_CUDA(cudaMalloc(&mem, total));
    char* base = (char*)mem;
    double* C = (double*)base;
    std::vector<DevDesc> dd(count);
    for (size_t e = 0; e < count; ++e)
        dd[e] = DevDesc{d[e].A, d[e].B, C + coff[e], d[e].m, d[e].n, d[e].k, d[e].lda, d[e].ldb, d[e].m};
    DevDesc* d_dd = (DevDesc*)(base + o_desc);
    Item* d_items = (Item*)(base + o_items);
    int* d_head = (int*)(base + o_head);
    cudaError_t ce = cudaMemsetAsync(C, 0, 8 * c_elems, h->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_dd, dd.data(), sizeof(DevDesc) * count, cudaMemcpyHostToDevice, h->stream);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, h->stream);
    const int n_items = (int)items.size();
    const int grid = std::max(1, std::min(h->sms * h->blocks_per_sm_slim, n_items));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ce == cudaSuccess) ce = cudaEventCreate(&e0);
    if (ce == cudaSuccess) ce = cudaEventCreate(&e1);
    if (ce == cudaSuccess) ce = launch_persistent(d_dd, d_items, n_items, d_head, grid, h->stream, 0, 0);
    float best = 1e30f;
    for (int rep = 0; rep < 3 && ce == cudaSuccess; ++rep) {
        cudaEventRecord(e0, h->stream);
        ce = launch_persistent(d_dd, d_items, n_items, d_head, grid, h->stream, 0, 0);
        cudaEventRecord(e1, h->stream);
        if (ce == cudaSuccess) ce = cudaEventSynchronize(e1);
        float ms = 0;
        if (ce == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
        best = std::min(best, ms);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaStreamSynchronize(h->stream);
    cudaFree(mem);
    if (ce != cudaSuccess) return cuda_fail(ce, "timing a small plan's tiles");
    *ms_out = best;
    return LRB_OK;
}

lrb_status choose_variants(lrb_handle* h, const lrb_gemm_desc* d, size_t count, const lrb_plan_opts& o,
                           std::vector<int>& var) {
    var.resize(count);
    const bool dmma_ok = o.precision == LRB_PREC_FP64_DMMA_ALLOWED;
    std::lock_guard<std::mutex> lock(h->mu);
    bool dirty = false;
    std::map<std::string, int> local;
    for (size_t e = 0; e < count; ++e) {
        if (o.force_variant >= 0) {
            var[e] = o.force_variant;
            continue;
        }
        const std::string key = bucket_key(d[e].m, d[e].n, d[e].k, dmma_ok);
        auto it = local.find(key);
        if (it != local.end()) {
            var[e] = it->second;
            continue;
        }
        auto jt = h->tuned.find(key);
        int v;
        if (jt != h->tuned.end()) {
            v = jt->second;
        } else if (o.tune) {
            lrb_status s = tune_bucket(h, d[e].m, d[e].n, d[e].k, dmma_ok, &v);
            if (s != LRB_OK) return s;
            h->tuned[key] = v;
            dirty = true;
        } else {
            v = heuristic_variant(d[e].m, d[e].n, d[e].k, dmma_ok);
        }
        local[key] = v;
        var[e] = v;
    }
    if (dirty) save_cache(h);
    if (o.trans != 0 || o.overwrite != 0)   // those forms run in the slim persistent kernel only
        for (int& v : var)
            if (variant_set(v) != 0) v = kVariants[v].dmma ? 8 : 2;
    return LRB_OK;
}

void free_plan(lrb_plan* p) {
    if (!p) return;
    for (lrb_plan*& q : p->lr_stage)
        if (q) {
            free_plan(q);
            q = nullptr;
        }
    if (p->lr_work) cudaFree(p->lr_work);
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->sp) split::destroy(p->sp);
    if (p->lp) lowrank::destroy(p->lp);
    if (p->dmem) cudaFree(p->dmem);
    delete p;
}

}  // namespace

void lrb::set_last_error(const char* msg) { g_err = msg; }

// Planner pieces shared with the serving queue (serve.cu).
lrb_status lrb::validate_descs(const lrb_gemm_desc* d, size_t count, const lrb_plan_opts& o) {
    return validate(d, count, o);
}
lrb_status lrb::plan_variants(lrb_handle* h, const lrb_gemm_desc* d, size_t count, const lrb_plan_opts& o,
                              std::vector<int>& var) {
    return choose_variants(h, d, count, o, var);
}
void lrb::plan_tiles(const lrb_gemm_desc* d, size_t count, const std::vector<int>& var, std::vector<Item>& items) {
    make_tiles(d, count, var, items);
}
int lrb::untuned_variant(int m, int n, int k) { return heuristic_variant(m, n, k, false); }
lrb::HandleInfo lrb::handle_info(const lrb_handle* h) {
    return HandleInfo{h->device, h->sms, h->blocks_per_sm, h->blocks_per_sm_wide, h->blocks_per_sm_slim};
}
lrb_plan_opts lrb::default_plan_opts() { return default_opts(); }
cudaError_t lrb::enqueue_fp64_plan(lrb_plan* p, cudaStream_t s) {
    if (p->sp || p->lp || p->lr_kind) return cudaErrorInvalidValue;
    p->last_stream = s;
    p->launched = true;
    return launch_persistent(p->d_descs, p->d_items, p->n_items, p->d_head, p->grid, s, p->set, p->ops);
}

extern "C" {

const char* lrb_last_error(void) { return g_err.c_str(); }

int32_t lrb_variant_count(void) { return kNumVariants; }

lrb_status lrb_variant_shape(int32_t variant, int32_t* bm, int32_t* bn, int32_t* is_dmma) {
    if (variant < 0 || variant >= kNumVariants) return fail(LRB_ERR_INVALID, "variant out of range");
    if (bm) *bm = kVariants[variant].bm();
    if (bn) *bn = kVariants[variant].bn();
    if (is_dmma) *is_dmma = kVariants[variant].dmma;
    return LRB_OK;
}

lrb_status lrb_validate(const lrb_gemm_desc* host_descs, size_t count, const lrb_plan_opts* opts) {
    const lrb_plan_opts o = opts ? *opts : default_opts();
    return validate(host_descs, count, o);
}

lrb_status lrb_plan_tiles_host(const lrb_gemm_desc* host_descs, size_t count, int32_t variant, int32_t* out,
                               size_t cap, size_t* n_items) {
    lrb_plan_opts o = default_opts();
    o.check_alias = 0;
    lrb_status s = validate(host_descs, count, o);
    if (s != LRB_OK) return s;
    if (variant < 0 || variant >= kNumVariants) return fail(LRB_ERR_INVALID, "variant out of range");
    if (!n_items) return fail(LRB_ERR_INVALID, "n_items is NULL");
    std::vector<int> var(count, variant);
    std::vector<Item> items;
    make_tiles(host_descs, count, var, items);
    *n_items = items.size();
    if (out) {
        const Variant& V = kVariants[variant];
        for (size_t i = 0; i < items.size() && i < cap; ++i) {
            const lrb_gemm_desc& d = host_descs[items[i].entry];
            out[5 * i + 0] = items[i].entry;
            out[5 * i + 1] = items[i].row0;
            out[5 * i + 2] = items[i].col0;
            out[5 * i + 3] = std::min(V.bm(), d.m - items[i].row0);
            out[5 * i + 4] = std::min(V.bn(), d.n - items[i].col0);
        }
    }
    return LRB_OK;
}

lrb_status lrb_create(lrb_handle** out, int device) {
    if (!out) return fail(LRB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(LRB_ERR_INVALID, "device ordinal out of range");
    LRB_CUDA(cudaSetDevice(device));
    lrb_handle* h = new (std::nothrow) lrb_handle();
    if (!h) return fail(LRB_ERR_NOMEM, "handle allocation");
    h->device = device;
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaGetDeviceProperties");
    }
    h->sms = prop.multiProcessorCount;
    h->blocks_per_sm = persistent_blocks_per_sm(1);
    h->blocks_per_sm_wide = persistent_blocks_per_sm(2);
    h->blocks_per_sm_slim = persistent_blocks_per_sm(0);
    if (h->blocks_per_sm <= 0 || h->blocks_per_sm_wide <= 0 || h->blocks_per_sm_slim <= 0) {
        delete h;
        return fail(LRB_ERR_DEVICE, "persistent kernel does not fit on this device");
    }
    int drv = 0;
    cudaDriverGetVersion(&drv);
    char key[256];
    std::snprintf(key, sizeof key, "%s|cc%d%d|drv%d|lib2", prop.name, prop.major, prop.minor, drv);
    h->gpu_key = key;
    if (const char* p = std::getenv("LRB_TUNE_CACHE")) h->cache_path = p;
    load_cache(h);
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete h;
        return cuda_fail(e, "cudaStreamCreate");
    }
    *out = h;
    return LRB_OK;
}

lrb_status lrb_destroy(lrb_handle* h) {
    if (!h) return fail(LRB_ERR_INVALID, "handle is NULL");
    cudaSetDevice(h->device);
    cudaDeviceSynchronize();
    for (lrb_plan* p : h->host_plans) free_plan(p);
    for (cudaEvent_t e : h->ev_in) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_done) cudaEventDestroy(e);
    if (h->copy_in) cudaStreamDestroy(h->copy_in);
    if (h->copy_out) cudaStreamDestroy(h->copy_out);
    if (h->compute2) cudaStreamDestroy(h->compute2);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    for (cudaEvent_t e : h->tev) cudaEventDestroy(e);
    if (h->tev0) cudaEventDestroy(h->tev0);
    if (h->arena) cudaFree(h->arena);
    if (h->scratch) cudaFree(h->scratch);
    if (h->stream) cudaStreamDestroy(h->stream);
    delete h;
    return LRB_OK;
}

lrb_status lrb_plan_create(lrb_handle* h, const lrb_gemm_desc* host_descs, size_t count, const lrb_plan_opts* opts,
                           lrb_plan** out) {
    if (!h) return fail(LRB_ERR_INVALID, "handle is NULL");
    if (!out) return fail(LRB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    const lrb_plan_opts o = opts ? *opts : default_opts();
    lrb_status s = validate(host_descs, count, o);
    if (s != LRB_OK) return s;
    LRB_CUDA(cudaSetDevice(h->device));

    lrb_plan* p = new (std::nothrow) lrb_plan();
    if (!p) return fail(LRB_ERR_NOMEM, "plan allocation");
    p->h = h;
    p->precision = o.precision;
    p->descs.assign(host_descs, host_descs + count);
    double flops = 0, bytes = 0;
    for (size_t e = 0; e < count; ++e) {
        const double m = host_descs[e].m, n = host_descs[e].n, k = host_descs[e].k;
        flops += 2 * m * n * k;
        bytes += 8 * (m * k + k * n + 2 * m * n);
    }
    p->info.entries = (int64_t)count;
    p->info.flops = flops;
    p->info.alg_bytes = bytes;
    p->info.precision = o.precision;

    if (o.precision >= LRB_PREC_SPLIT_BF16_S3 && (o.trans != 0 || o.overwrite != 0)) {
        free_plan(p);
        return fail(LRB_ERR_UNSUPPORTED, "split-precision plans take A and B as stored and accumulate into C");
    }
    p->ops = o.trans | (o.overwrite ? 4 : 0);
    if (o.precision >= LRB_PREC_SPLIT_BF16_S3) {
        s = split::create(h->device, h->sms, p->descs.data(), count, o.precision, &p->sp, &p->info, o.test_stall);
        if (s != LRB_OK) {
            free_plan(p);
            return s;
        }
        *out = p;
        return LRB_OK;
    }

    std::vector<int> var;
    s = choose_variants(h, host_descs, count, o, var);
    if (s != LRB_OK) {
        free_plan(p);
        return s;
    }
    std::vector<Item> items;
    make_tiles(host_descs, count, var, items);
    if (o.force_variant < 0 && items.size() < 2 * (size_t)h->sms * (size_t)h->blocks_per_sm_slim) {
        // Fewer tiles than two waves of the persistent grid: the last wave
        // would leave most CTA slots idle.  Halve the tile height where a
        // 32-row k-split counterpart exists (64x8 -> 32x8, 64x32 -> 32x32),
        // doubling those entries' tiles.
        bool changed = false;
        for (int& v : var) {
            if (v == 0 || v == 2) {
                v = v == 0 ? 6 : 7;
                changed = true;
            }
        }
        if (changed) make_tiles(host_descs, count, var, items);
    } else if (o.tune && o.force_variant < 0 && o.trans == 0 && o.overwrite == 0 &&
               items.size() < 8 * (size_t)h->sms * (size_t)h->blocks_per_sm_slim) {
        // Two to eight waves: the last wave's share of the time is large, and
        // the bucket tuner (which times full waves) cannot see it.  Narrower
        // tiles (64x16 and 64x32 -> 64x8: the same per-element k order, so
        // the same results) give more, shorter tiles for the tail; time both
        // tilings on this plan's own operands and keep the faster (the
        // narrower one only if it gains 1 % or more).
        bool all_slim = true, narrowable = false;
        for (int v : var) {
            all_slim = all_slim && variant_set(v) == 0;
            narrowable = narrowable || v == 1 || v == 2;
        }
        if (all_slim && narrowable) {
            std::vector<int> alt(var);
            for (int& v : alt)
                if (v == 1 || v == 2) v = 0;
            float t_cur = 0, t_alt = 0;
            lrb_status st = time_plan_tiles(h, host_descs, count, var, &t_cur);
            if (st == LRB_OK) st = time_plan_tiles(h, host_descs, count, alt, &t_alt);
            if (st != LRB_OK) {
                free_plan(p);
                return st;
            }
            if (t_alt < 0.99f * t_cur) {
                var.swap(alt);
                make_tiles(host_descs, count, var, items);
            }
        }
    }
    if (items.size() > 0x7fffffffull) {
        free_plan(p);
        return fail(LRB_ERR_INVALID, "too many tiles");
    }
    // plain-launch groups: entries sharing (variant, m, n, k), in first-seen order
    std::map<std::tuple<int, int, int, int>, int> gid;
    std::vector<std::vector<int32_t>> members;
    for (size_t e = 0; e < count; ++e) {
        auto key = std::make_tuple(var[e], host_descs[e].m, host_descs[e].n, host_descs[e].k);
        auto it = gid.find(key);
        int g;
        if (it == gid.end()) {
            g = (int)members.size();
            gid[key] = g;
            members.emplace_back();
            const Variant& V = kVariants[var[e]];
            p->groups.push_back(Group{var[e], host_descs[e].m, host_descs[e].n, host_descs[e].k,
                                      ceil_div(host_descs[e].m, V.bm()), ceil_div(host_descs[e].n, V.bn()), 0, 0});
        } else {
            g = it->second;
        }
        members[g].push_back((int32_t)e);
    }
    std::vector<int32_t> flat;
    flat.reserve(count);
    for (size_t g = 0; g < members.size(); ++g) {
        p->groups[g].offset = (int)flat.size();
        p->groups[g].count = (int)members[g].size();
        flat.insert(flat.end(), members[g].begin(), members[g].end());
    }

    // one device allocation: descriptors | items | group entries | counter
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_desc = 0;
    const size_t o_items = align(o_desc + sizeof(DevDesc) * count);
    const size_t o_grp = align(o_items + sizeof(Item) * std::max<size_t>(items.size(), 1));
    const size_t o_head = align(o_grp + sizeof(int32_t) * count);
    const size_t total = o_head + 256;
    cudaError_t ce = cudaMalloc(&p->dmem, total);
    if (ce != cudaSuccess) {
        free_plan(p);
        return fail(LRB_ERR_NOMEM, std::string("plan device memory: ") + cudaGetErrorString(ce));
    }
    char* base = (char*)p->dmem;
    p->d_descs = (DevDesc*)(base + o_desc);
    p->d_items = (Item*)(base + o_items);
    p->d_group_entries = (int32_t*)(base + o_grp);
    p->d_head = (int*)(base + o_head);
    p->n_items = (int)items.size();
    ce = cudaMemcpy(p->d_descs, host_descs, sizeof(DevDesc) * count, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && !items.empty())
        ce = cudaMemcpy(p->d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->d_group_entries, flat.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice);
    if (ce == cudaSuccess) ce = cudaMemset(p->d_head, 0, 256);
    if (ce != cudaSuccess) {
        free_plan(p);
        return cuda_fail(ce, "plan upload");
    }
    for (size_t e = 0; e < count; ++e) p->set = std::max(p->set, variant_set(var[e]));
    const int per_sm = p->set == 0 ? h->blocks_per_sm_slim : p->set == 1 ? h->blocks_per_sm : h->blocks_per_sm_wide;
    p->grid = std::max(1, std::min(h->sms * per_sm, p->n_items));
    p->info.items = p->n_items;
    p->info.dmma_items = 0;
    for (const Item& it : items) p->info.dmma_items += kVariants[it.variant].dmma ? 1 : 0;
    p->info.groups = (int64_t)p->groups.size();
    p->info.grid = p->grid;

    if (o.use_graph) {
        cudaStream_t cs = h->stream;
        ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (ce == cudaSuccess) {
            cudaError_t le =
                launch_persistent(p->d_descs, p->d_items, p->n_items, p->d_head, p->grid, cs, p->set, p->ops);
            ce = cudaStreamEndCapture(cs, &p->graph);
            if (le != cudaSuccess) ce = le;
        }
        if (ce == cudaSuccess) ce = cudaGraphInstantiate(&p->exec, p->graph, 0);
        if (ce != cudaSuccess) {
            free_plan(p);
            return cuda_fail(ce, "graph capture");
        }
        p->use_graph = true;
    }
    *out = p;
    return LRB_OK;
}

lrb_status lrb_launch(lrb_plan* p, void* stream) {
    if (!p) return fail(LRB_ERR_INVALID, "plan is NULL");
    cudaStream_t s = (cudaStream_t)stream;
    LRB_CUDA(cudaSetDevice(p->h->device));
    p->last_stream = s;
    p->launched = true;
    if (p->sp) {
        cudaError_t e = split::launch(p->sp, s);
        return e == cudaSuccess ? LRB_OK : cuda_fail(e, "split launch");
    }
    if (p->lp) {
        cudaError_t e = lowrank::launch(p->lp, s);
        return e == cudaSuccess ? LRB_OK : cuda_fail(e, "low-rank plan launch");
    }
    if (p->lr_kind == 1) {
        cudaError_t e = launch_lr_chain(p->d_lr, p->lr_count, p->lr_rmax, s);
        return e == cudaSuccess ? LRB_OK : cuda_fail(e, "low-rank chain launch");
    }
    if (p->lr_kind == 2) {
        // the three products write their outputs (overwrite form): nothing to clear
        for (lrb_plan* q : p->lr_stage) {
            lrb_status st = lrb_launch(q, stream);
            if (st != LRB_OK) return st;
        }
        return LRB_OK;
    }
    cudaError_t e = p->use_graph ? cudaGraphLaunch(p->exec, s)
                                 : launch_persistent(p->d_descs, p->d_items, p->n_items, p->d_head, p->grid, s,
                                                     p->set, p->ops);
    if (e != cudaSuccess) return cuda_fail(e, "persistent launch");
    return LRB_OK;
}

lrb_status lrb_launch_plain(lrb_plan* p, void* stream) {
    if (!p) return fail(LRB_ERR_INVALID, "plan is NULL");
    if (p->sp) return fail(LRB_ERR_UNSUPPORTED, "split-precision plans have no plain launch");
    if (p->lr_kind) return fail(LRB_ERR_UNSUPPORTED, "low-rank chain plans have no plain launch");
    if (p->ops) return fail(LRB_ERR_UNSUPPORTED, "transposed or overwriting plans have no plain launch");
    if (p->lp) return fail(LRB_ERR_UNSUPPORTED, "low-rank producer/consumer plans have no plain launch");
    cudaStream_t s = (cudaStream_t)stream;
    LRB_CUDA(cudaSetDevice(p->h->device));
    p->last_stream = s;
    p->launched = true;
    for (const Group& g : p->groups) {
        cudaError_t e = launch_plain_group(g.variant, p->d_descs, p->d_group_entries + g.offset, g.count, g.tiles_m,
                                           g.tiles_n, s);
        if (e != cudaSuccess) return cuda_fail(e, "plain launch");
    }
    return LRB_OK;
}

lrb_status lrb_execute_host(lrb_handle* h, const lrb_gemm_desc* host_descs, size_t count, const lrb_plan_opts* opts,
                            void* stream) {
    if (!h) return fail(LRB_ERR_INVALID, "handle is NULL");
    const lrb_plan_opts o = opts ? *opts : default_opts();
    if (!host_descs || count == 0) return validate(host_descs, count, o);
    if (o.trans != 0 || o.overwrite != 0)
        return fail(LRB_ERR_UNSUPPORTED, "the host-buffer path takes A and B as stored and accumulates into C");
    lrb_status st = LRB_OK;
    LRB_CUDA(cudaSetDevice(h->device));
    cudaStream_t s = (cudaStream_t)stream;

    const bool cached = !h->host_plans.empty() && h->host_in.size() == count &&
                        std::memcmp(h->host_in.data(), host_descs, sizeof(lrb_gemm_desc) * count) == 0 &&
                        std::memcmp(&h->host_opts, &o, sizeof(o)) == 0;
    if (!cached) {
        st = validate(host_descs, count, o);
        if (st != LRB_OK) return st;
        // Pieces: contiguous entry ranges of about equal bytes (at most 64, at
        // least 64 MB each).  Piece p's copies in, its launch and its copies out
        // run on three streams joined by events, so piece p+1 moves in while p
        // computes and p-1 moves out.  The first piece's copy in and the last
        // one's copy out are not hidden, so more pieces shorten the step until
        // the launches' tails dominate (66 GB sweep: 16 pieces 1102, 32 pieces
        // 1150, 64 pieces 1192 GFLOP/s).
        std::vector<double> eb(count);
        double total = 0;
        for (size_t e = 0; e < count; ++e) {
            const lrb_gemm_desc& x = host_descs[e];
            eb[e] = 8.0 * ((double)x.m * x.k + (double)x.k * x.n + 2.0 * x.m * x.n);
            total += eb[e];
        }
        const int npieces = (int)std::max(1.0, std::min(64.0, std::floor(total / (64.0 * (1 << 20)))));
        std::vector<size_t> cut(1, 0);
        {
            double acc = 0;
            for (size_t e = 0; e < count; ++e) {
                acc += eb[e];
                if ((int)cut.size() < npieces && acc >= total * (double)cut.size() / npieces && e + 1 < count)
                    cut.push_back(e + 1);
            }
            cut.push_back(count);
        }
        const int P = (int)cut.size() - 1;

        // Shared regions: A and B operands whose host byte ranges overlap
        // another A or B operand's (views into one operand pool, or one block
        // used by several entries) are served from a single copy of the union
        // of those ranges, made by the first piece that uses it; those entries
        // keep their leading dimensions.  Read-only operands may overlap, so
        // this copies each host byte once.
        struct Span {
            uintptr_t lo, hi;
            size_t op;   // 2 e + 0 (A) or 1 (B)
        };
        struct Region {
            uintptr_t lo, hi;
            size_t dev;
            int first_piece;
        };
        std::vector<Span> spans(2 * count);
        for (size_t e = 0; e < count; ++e) {
            const lrb_gemm_desc& x = host_descs[e];
            spans[2 * e] = Span{(uintptr_t)x.A, (uintptr_t)x.A + 8 * ((size_t)x.lda * (x.k - 1) + x.m), 2 * e};
            spans[2 * e + 1] = Span{(uintptr_t)x.B, (uintptr_t)x.B + 8 * ((size_t)x.ldb * (x.n - 1) + x.k), 2 * e + 1};
        }
        std::sort(spans.begin(), spans.end(), [](const Span& a, const Span& b) { return a.lo < b.lo; });
        std::vector<int> region_of(2 * count, -1);
        std::vector<Region> regions;
        for (size_t i = 0; i < spans.size();) {
            size_t j = i + 1;
            uintptr_t hi = spans[i].hi;
            while (j < spans.size() && spans[j].lo < hi) hi = std::max(hi, spans[j++].hi);
            if (j - i >= 2) {
                for (size_t t = i; t < j; ++t) region_of[spans[t].op] = (int)regions.size();
                regions.push_back(Region{spans[i].lo, hi, 0, -1});
            }
            i = j;
        }
        std::vector<size_t> piece_of(count);
        for (int pc = 0; pc < P; ++pc)
            for (size_t e = cut[pc]; e < cut[pc + 1]; ++e) piece_of[e] = (size_t)pc;
        for (size_t op = 0; op < 2 * count; ++op)
            if (region_of[op] >= 0 && regions[region_of[op]].first_piece < 0)
                regions[region_of[op]].first_piece = (int)piece_of[op / 2];

        // Device layout, piece by piece: the shared regions the piece is first
        // to use, then its other A blocks, B blocks and C blocks, each packed
        // with ld = rows (runs of host-contiguous tight blocks move in one copy).
        using Copy = HostCopy;
        std::vector<lrb_gemm_desc> dd(host_descs, host_descs + count);
        std::vector<std::vector<Copy>> h2d(P), d2h(P);
        std::vector<size_t> wa(count), wb(count), wc(count);
        size_t cursor = 0;
        for (int pc = 0; pc < P; ++pc) {
            for (Region& r : regions)
                if (r.first_piece == pc) {
                    const size_t elems = (r.hi - r.lo) / 8;
                    r.dev = cursor;
                    for (size_t o = 0; o < elems; o += kRegionChunkElems)   // in chunks of 256 MB
                        h2d[pc].push_back(Copy{(const double*)r.lo + o, cursor + o, 0, -1, 0,
                                               std::min(kRegionChunkElems, elems - o)});
                    cursor += elems;
                }
            for (int cls = 0; cls < 3; ++cls) {
                std::vector<Copy>& list = h2d[pc];
                const size_t cls_start = list.size();   // runs never merge across operand classes
                for (size_t e = cut[pc]; e < cut[pc + 1]; ++e) {
                    const lrb_gemm_desc& x = host_descs[e];
                    const double* ptr = cls == 0 ? x.A : cls == 1 ? x.B : x.C;
                    const int rows = cls == 0 ? x.m : cls == 1 ? x.k : x.m;
                    const int cols = cls == 0 ? x.k : cls == 1 ? x.n : x.n;
                    const int ld = cls == 0 ? x.lda : cls == 1 ? x.ldb : x.ldc;
                    std::vector<size_t>& where = cls == 0 ? wa : cls == 1 ? wb : wc;
                    if (cls < 2 && region_of[2 * e + cls] >= 0) {
                        const Region& r = regions[region_of[2 * e + cls]];
                        where[e] = r.dev + ((uintptr_t)ptr - r.lo) / 8;
                        continue;
                    }
                    const size_t elems = (size_t)rows * cols;
                    if (list.size() > cls_start && ld == rows) {
                        // extend the previous run when this block starts at most
                        // kGapElems elements after it in host memory; the device
                        // layout keeps the same gap, so one 1-D copy moves both
                        Copy& b = list.back();
                        const ptrdiff_t gap = ptr - (b.host + b.elems);
                        if ((b.cols < 0 || b.ld == b.rows) && gap >= 0 && gap < kGapElems && b.dev + b.elems == cursor) {
                            cursor += (size_t)gap;
                            where[e] = cursor;
                            b.elems += (size_t)gap + elems;
                            b.cols = -1;   // merged run: a 1-D copy
                            cursor += elems;
                            continue;
                        }
                    }
                    where[e] = cursor;
                    list.push_back(Copy{ptr, cursor, rows, cols, ld, elems});
                    cursor += elems;
                }
                if (cls == 2) d2h[pc].assign(list.begin() + cls_start, list.end());
            }
        }

        const size_t need = cursor * 8 + 256;
        if (need > h->arena_bytes) {
            for (lrb_plan* p : h->host_plans) free_plan(p);
            h->host_plans.clear();
            cudaStreamSynchronize(s);
            if (h->arena) cudaFree(h->arena);
            h->arena = nullptr;
            h->arena_bytes = 0;
            cudaError_t ce = cudaMalloc(&h->arena, need);
            if (ce != cudaSuccess) return fail(LRB_ERR_NOMEM, std::string("host-run arena: ") + cudaGetErrorString(ce));
            h->arena_bytes = need;
            h->host_key.clear();
        }
        if (!h->copy_in) {
            LRB_CUDA(cudaStreamCreateWithFlags(&h->copy_in, cudaStreamNonBlocking));
            LRB_CUDA(cudaStreamCreateWithFlags(&h->copy_out, cudaStreamNonBlocking));
            LRB_CUDA(cudaStreamCreateWithFlags(&h->compute2, cudaStreamNonBlocking));
            LRB_CUDA(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
        }
        while ((int)h->ev_in.size() < P) {
            cudaEvent_t a, b;
            LRB_CUDA(cudaEventCreateWithFlags(&a, cudaEventDisableTiming));
            LRB_CUDA(cudaEventCreateWithFlags(&b, cudaEventDisableTiming));
            h->ev_in.push_back(a);
            h->ev_done.push_back(b);
        }
        double* base = (double*)h->arena;
        for (size_t e = 0; e < count; ++e) {
            dd[e].A = base + wa[e];
            dd[e].B = base + wb[e];
            dd[e].C = base + wc[e];
            if (region_of[2 * e] < 0) dd[e].lda = dd[e].m;       // packed; a shared region keeps the caller's ld
            if (region_of[2 * e + 1] < 0) dd[e].ldb = dd[e].k;
            dd[e].ldc = dd[e].m;
        }
        const bool same = !h->host_plans.empty() && h->host_key.size() == count && h->host_cut == cut &&
                          std::memcmp(h->host_key.data(), dd.data(), sizeof(lrb_gemm_desc) * count) == 0 &&
                          std::memcmp(&h->host_opts, &o, sizeof(o)) == 0;
        if (!same) {
            cudaStreamSynchronize(s);
            for (lrb_plan* p : h->host_plans) free_plan(p);
            h->host_plans.clear();
            for (int pc = 0; pc < P; ++pc) {
                lrb_plan* p = nullptr;
                lrb_plan_opts po = o;
                po.check_alias = 0;   // checked above on the caller's host ranges
                st = lrb_plan_create(h, dd.data() + cut[pc], cut[pc + 1] - cut[pc], &po, &p);
                if (st != LRB_OK) {
                    for (lrb_plan* q : h->host_plans) free_plan(q);
                    h->host_plans.clear();
                    return st;
                }
                h->host_plans.push_back(p);
            }
            h->host_key = dd;
            h->host_cut = cut;
            h->host_opts = o;
        }

        h->host_in.assign(host_descs, host_descs + count);
        h->host_h2d = h2d;
        h->host_d2h = d2h;
    }
    const int P = (int)h->host_h2d.size();
    const std::vector<std::vector<HostCopy>>& h2d = h->host_h2d;
    const std::vector<std::vector<HostCopy>>& d2h = h->host_d2h;
    double* base = (double*)h->arena;
    auto copy = [&](const HostCopy& c, bool to_dev, cudaStream_t cs) -> cudaError_t {
        double* dptr = base + c.dev;
        if (c.cols < 0 || c.ld == c.rows) {
            const size_t bytes = c.elems * 8;
            return to_dev ? cudaMemcpyAsync(dptr, c.host, bytes, cudaMemcpyHostToDevice, cs)
                          : cudaMemcpyAsync((void*)c.host, dptr, bytes, cudaMemcpyDeviceToHost, cs);
        }
        return to_dev ? cudaMemcpy2DAsync(dptr, (size_t)c.rows * 8, c.host, (size_t)c.ld * 8, (size_t)c.rows * 8,
                                          c.cols, cudaMemcpyHostToDevice, cs)
                      : cudaMemcpy2DAsync((void*)c.host, (size_t)c.ld * 8, dptr, (size_t)c.rows * 8,
                                          (size_t)c.rows * 8, c.cols, cudaMemcpyDeviceToHost, cs);
    };
    const bool timed = h->timing;
    if (timed) {
        if (!h->tev0) LRB_CUDA(cudaEventCreate(&h->tev0));
        while ((int)h->tev.size() < 6 * P) {
            cudaEvent_t ev;
            LRB_CUDA(cudaEventCreate(&ev));
            h->tev.push_back(ev);
        }
        LRB_CUDA(cudaEventRecord(h->tev0, s));
    }
    // per piece: tev[6 pc + 0/1] copies in start/end, + 2/3 launch, + 4/5 copies out
    auto mark = [&](int pc, int which, cudaStream_t cs) -> cudaError_t {
        return timed ? cudaEventRecord(h->tev[6 * pc + which], cs) : cudaSuccess;
    };
    // the copy and compute streams start after work already queued on the
    // caller's stream
    LRB_CUDA(cudaEventRecord(h->ev_done[0], s));
    LRB_CUDA(cudaStreamWaitEvent(h->copy_in, h->ev_done[0], 0));
    LRB_CUDA(cudaStreamWaitEvent(h->compute2, h->ev_done[0], 0));
    // Each piece's copies in, launch and copies out are enqueued together, so
    // that when the host blocks in a copy call (a stream holds a bounded
    // number of pending operations) every earlier piece's launch is already
    // queued.  Pieces alternate between the caller's stream and a second
    // compute stream, so one piece's last tiles overlap the next piece's first.
    for (int pc = 0; pc < P; ++pc) {
        LRB_CUDA(mark(pc, 0, h->copy_in));
        for (const HostCopy& c : h2d[pc]) LRB_CUDA(copy(c, true, h->copy_in));
        LRB_CUDA(cudaEventRecord(h->ev_in[pc], h->copy_in));
        LRB_CUDA(mark(pc, 1, h->copy_in));
        cudaStream_t cs = (pc & 1) ? h->compute2 : s;
        LRB_CUDA(cudaStreamWaitEvent(cs, h->ev_in[pc], 0));
        LRB_CUDA(mark(pc, 2, cs));
        st = lrb_launch(h->host_plans[pc], (void*)cs);
        if (st != LRB_OK) return st;
        LRB_CUDA(mark(pc, 3, cs));
        LRB_CUDA(cudaEventRecord(h->ev_done[pc], cs));
        LRB_CUDA(cudaStreamWaitEvent(h->copy_out, h->ev_done[pc], 0));
        LRB_CUDA(mark(pc, 4, h->copy_out));
        for (const HostCopy& c : d2h[pc]) LRB_CUDA(copy(c, false, h->copy_out));
        LRB_CUDA(mark(pc, 5, h->copy_out));
    }
    // the caller's stream ends after everything, as before
    LRB_CUDA(cudaEventRecord(h->ev_join, h->copy_out));
    LRB_CUDA(cudaStreamWaitEvent(s, h->ev_join, 0));
    LRB_CUDA(cudaStreamSynchronize(h->copy_out));
    LRB_CUDA(cudaStreamSynchronize(s));
    if (timed) {
        std::vector<std::pair<double, double>> iv[3];
        for (int pc = 0; pc < P; ++pc)
            for (int cls = 0; cls < 3; ++cls) {
                float a = 0.f, b = 0.f;
                LRB_CUDA(cudaEventElapsedTime(&a, h->tev0, h->tev[6 * pc + 2 * cls]));
                LRB_CUDA(cudaEventElapsedTime(&b, h->tev0, h->tev[6 * pc + 2 * cls + 1]));
                iv[cls].emplace_back(a, b);
            }
        double bytes[2] = {0.0, 0.0}, first = 0.0;
        for (int pc = 0; pc < P; ++pc) {
            for (const HostCopy& c : h2d[pc]) bytes[0] += 8.0 * (double)c.elems;
            for (const HostCopy& c : d2h[pc]) bytes[1] += 8.0 * (double)c.elems;
        }
        for (const HostCopy& c : h2d[0]) first += 8.0 * (double)c.elems;
        h->last_timing = summarize_host_timing(iv, P, bytes[0], bytes[1], first);
    }
    return LRB_OK;
}

lrb_status lrb_execute_host_set_timing(lrb_handle* h, int32_t enable) {
    if (!h) return fail(LRB_ERR_INVALID, "handle is NULL");
    h->timing = enable != 0;
    return LRB_OK;
}

lrb_status lrb_execute_host_get_timing(const lrb_handle* h, lrb_host_timing* out) {
    if (!h || !out) return fail(LRB_ERR_INVALID, "handle or out is NULL");
    if (!h->last_timing.valid) return fail(LRB_ERR_INVALID, "no timed lrb_execute_host call yet");
    *out = h->last_timing;
    return LRB_OK;
}

lrb_status lrb_partition_lpt(const double* cost, size_t count, int32_t parts, int32_t* part_of, double* part_load) {
    if (!cost || !part_of || count == 0 || parts < 1)
        return fail(LRB_ERR_INVALID, "lrb_partition_lpt: NULL array, count == 0 or parts < 1");
    for (size_t i = 0; i < count; ++i)
        if (!(cost[i] >= 0.0) || !std::isfinite(cost[i])) return fail(LRB_ERR_INVALID, "lrb_partition_lpt: bad cost");
    std::vector<size_t> order(count);
    for (size_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return cost[a] > cost[b]; });
    // min-heap of (load, part): the least-loaded part, lower part index on ties
    using Slot = std::pair<double, int32_t>;
    std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
    for (int32_t r = 0; r < parts; ++r) heap.push(Slot(0.0, r));
    std::vector<double> load(parts, 0.0);
    for (size_t i : order) {
        Slot s = heap.top();
        heap.pop();
        part_of[i] = s.second;
        s.first = s.first + cost[i];
        load[s.second] = s.first;
        heap.push(s);
    }
    if (part_load)
        for (int32_t r = 0; r < parts; ++r) part_load[r] = load[r];
    return LRB_OK;
}

lrb_status lrb_multi_plan_create(lrb_handle* const* handles, int32_t n_handles, const lrb_gemm_desc* host_descs,
                                 size_t count, const lrb_plan_opts* opts, lrb_multi_plan** out) {
    if (!out) return fail(LRB_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!handles || n_handles < 1) return fail(LRB_ERR_INVALID, "no handles");
    for (int32_t i = 0; i < n_handles; ++i)
        if (!handles[i]) return fail(LRB_ERR_INVALID, "a handle is NULL");
    const lrb_plan_opts o = opts ? *opts : default_opts();
    lrb_status st = validate(host_descs, count, o);
    if (st != LRB_OK) return st;
    std::vector<double> cost(count);
    for (size_t e = 0; e < count; ++e)
        cost[e] = 2.0 * (double)host_descs[e].m * (double)host_descs[e].n * (double)host_descs[e].k;
    std::vector<int32_t> part(count);
    st = lrb_partition_lpt(cost.data(), count, n_handles, part.data(), nullptr);
    if (st != LRB_OK) return st;
    lrb_multi_plan* mp = new (std::nothrow) lrb_multi_plan();
    if (!mp) return fail(LRB_ERR_NOMEM, "multi-plan allocation");
    mp->plans.assign(n_handles, nullptr);
    mp->entries.assign(n_handles, 0);
    mp->devices.resize(n_handles);
    for (int32_t i = 0; i < n_handles; ++i) {
        mp->devices[i] = handles[i]->device;
        std::vector<lrb_gemm_desc> mine;
        for (size_t e = 0; e < count; ++e)
            if (part[e] == i) mine.push_back(host_descs[e]);
        mp->entries[i] = (int64_t)mine.size();
        if (mine.empty()) continue;
        st = lrb_plan_create(handles[i], mine.data(), mine.size(), &o, &mp->plans[i]);
        if (st != LRB_OK) {
            lrb_multi_plan_destroy(mp);
            return st;
        }
    }
    *out = mp;
    return LRB_OK;
}

lrb_status lrb_multi_launch(lrb_multi_plan* mp, void* const* streams) {
    if (!mp) return fail(LRB_ERR_INVALID, "multi-plan is NULL");
    for (size_t i = 0; i < mp->plans.size(); ++i) {
        if (!mp->plans[i]) continue;
        lrb_status st = lrb_launch(mp->plans[i], streams ? streams[i] : nullptr);
        if (st != LRB_OK) return st;
    }
    return LRB_OK;
}

lrb_status lrb_multi_plan_part(const lrb_multi_plan* mp, int32_t part, lrb_plan_info* info) {
    if (!mp || !info) return fail(LRB_ERR_INVALID, "multi-plan or info is NULL");
    if (part < 0 || part >= (int32_t)mp->plans.size()) return fail(LRB_ERR_INVALID, "part out of range");
    if (!mp->plans[part]) {
        std::memset(info, 0, sizeof(*info));
        return LRB_OK;
    }
    return lrb_plan_get_info(mp->plans[part], info);
}

lrb_status lrb_multi_plan_destroy(lrb_multi_plan* mp) {
    if (!mp) return fail(LRB_ERR_INVALID, "multi-plan is NULL");
    lrb_status st = LRB_OK;
    for (lrb_plan* p : mp->plans)
        if (p) {
            lrb_status s2 = lrb_plan_destroy(p);
            if (st == LRB_OK) st = s2;
        }
    delete mp;
    return st;
}

lrb_status lrb_plan_status(lrb_plan* p) {
    if (!p) return fail(LRB_ERR_INVALID, "plan is NULL");
    LRB_CUDA(cudaSetDevice(p->h->device));
    if (p->launched) LRB_CUDA(p->last_stream ? cudaStreamSynchronize(p->last_stream) : cudaDeviceSynchronize());
    if (p->sp) {
        int v = 0;
        if (split::read_status(p->sp, p->last_stream, &v) != 0) return fail(LRB_ERR_DEVICE, "reading plan status");
        if (v) return fail(LRB_ERR_TIMEOUT, "a bounded device wait expired in a split-precision launch");
    }
    if (p->lp) {
        int v = 0;
        if (lowrank::read_status(p->lp, p->last_stream, &v) != 0) return fail(LRB_ERR_DEVICE, "reading plan status");
        if (v) return fail(LRB_ERR_TIMEOUT, "a Jacobi SVD reached its sweep limit without converging");
    }
    return LRB_OK;
}

namespace {
lrb_status wrap_lowrank(lrb_handle* h, lowrank::LrPlan* lp, const lrb_plan_info& info, lrb_plan** out) {
    lrb_plan* p = new (std::nothrow) lrb_plan();
    if (!p) {
        lowrank::destroy(lp);
        return fail(LRB_ERR_NOMEM, "plan allocation");
    }
    p->h = h;
    p->lp = lp;
    p->info = info;
    *out = p;
    return LRB_OK;
}
}  // namespace

lrb_status lrb_rsvd_plan_create(lrb_handle* h, const lrb_rsvd_desc* d, size_t count, int32_t power_iters,
                                lrb_plan** out) {
    if (!h || !out) return fail(LRB_ERR_INVALID, "NULL argument");
    *out = nullptr;
    LRB_CUDA(cudaSetDevice(h->device));
    lowrank::LrPlan* lp = nullptr;
    lrb_plan_info info{};
    lrb_status s = lowrank::create_rsvd(h, d, count, power_iters, &lp, &info);
    return s != LRB_OK ? s : wrap_lowrank(h, lp, info, out);
}

lrb_status lrb_expand_plan_create(lrb_handle* h, const lrb_expand_desc* d, size_t count, lrb_plan** out) {
    if (!h || !out) return fail(LRB_ERR_INVALID, "NULL argument");
    *out = nullptr;
    LRB_CUDA(cudaSetDevice(h->device));
    lowrank::LrPlan* lp = nullptr;
    lrb_plan_info info{};
    lrb_status s = lowrank::create_expand(h, d, count, &lp, &info);
    return s != LRB_OK ? s : wrap_lowrank(h, lp, info, out);
}

lrb_status lrb_round_add_plan_create(lrb_handle* h, const lrb_round_add_desc* d, size_t count, lrb_plan** out) {
    if (!h || !out) return fail(LRB_ERR_INVALID, "NULL argument");
    *out = nullptr;
    LRB_CUDA(cudaSetDevice(h->device));
    lowrank::LrPlan* lp = nullptr;
    lrb_plan_info info{};
    lrb_status s = lowrank::create_round_add(h, d, count, &lp, &info);
    return s != LRB_OK ? s : wrap_lowrank(h, lp, info, out);
}

lrb_status lrb_split_dump_levels(lrb_plan* p, float* dump, void* stream) {
    if (!p || !dump) return fail(LRB_ERR_INVALID, "NULL argument");
    if (!p->sp || p->descs.size() != 1) return fail(LRB_ERR_UNSUPPORTED, "needs a split-precision plan of one entry");
    cudaStream_t s = (cudaStream_t)stream;
    LRB_CUDA(cudaSetDevice(p->h->device));
    p->last_stream = s;
    p->launched = true;
    cudaError_t e = split::launch_dump(p->sp, dump, s);
    return e == cudaSuccess ? LRB_OK : cuda_fail(e, "split dump launch");
}

lrb_status lrb_lr_plan_create(lrb_handle* h, const lrb_lr_desc* d, size_t count, int32_t fused, lrb_plan** out) {
    if (!h || !out) return fail(LRB_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (!d) return fail(LRB_ERR_INVALID, "host_descs is NULL");
    if (count == 0) return fail(LRB_ERR_INVALID, "count is 0");
    if (count > 0x7fffffffull) return fail(LRB_ERR_INVALID, "count exceeds 2^31-1");
    double flops = 0, bytes = 0;
    for (size_t e = 0; e < count; ++e) {
        const lrb_lr_desc& x = d[e];
        char buf[160];
        if (!x.AVT || !x.BU || !x.AX || !x.BX || !x.G) {
            std::snprintf(buf, sizeof buf, "entry %zu: NULL operand pointer", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        if (((uintptr_t)x.AVT | (uintptr_t)x.BU | (uintptr_t)x.AX | (uintptr_t)x.BX | (uintptr_t)x.G) & 7u) {
            std::snprintf(buf, sizeof buf, "entry %zu: operand pointer not 8-byte aligned", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        if (x.ra <= 0 || x.rb <= 0 || x.k <= 0 || x.ld_avt < x.ra || x.ld_bu < x.k || x.ld_ax < x.ra ||
            x.ld_bx < x.rb || x.ldg < x.ra) {
            std::snprintf(buf, sizeof buf, "entry %zu: bad dimension or leading dimension", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        Range r;
        if (!extent(x.AVT, x.ra, x.k, x.ld_avt, &r) || !extent(x.BU, x.k, x.rb, x.ld_bu, &r) ||
            !extent(x.AX, x.ra, x.ra, x.ld_ax, &r) || !extent(x.BX, x.rb, x.rb, x.ld_bx, &r) ||
            !extent(x.G, x.ra, x.rb, x.ldg, &r)) {
            std::snprintf(buf, sizeof buf, "entry %zu: operand extent overflows", e);
            return fail(LRB_ERR_INVALID, buf);
        }
        if (fused && (x.ra > lr_chain_max_rank() || x.rb > lr_chain_max_rank()))
            return fail(LRB_ERR_UNSUPPORTED, "fused low-rank chain supports ranks up to 64");
        const double ra = x.ra, rb = x.rb, k = x.k;
        flops += ra * rb * (2 * k + 2 * ra + 2 * rb);
        bytes += 8 * (ra * k + k * rb + ra * ra + rb * rb + ra * rb);
    }
    LRB_CUDA(cudaSetDevice(h->device));
    lrb_plan* p = new (std::nothrow) lrb_plan();
    if (!p) return fail(LRB_ERR_NOMEM, "plan allocation");
    p->h = h;
    p->lr_kind = fused ? 1 : 2;
    p->lr_count = (int)count;
    for (size_t e = 0; e < count; ++e) p->lr_rmax = std::max({p->lr_rmax, (int)d[e].ra, (int)d[e].rb});
    p->info.entries = (int64_t)count;
    p->info.flops = flops;
    p->info.alg_bytes = bytes;
    p->info.precision = LRB_PREC_FP64;
    p->info.grid = (int)count;
    cudaError_t ce = cudaMalloc(&p->dmem, sizeof(LrDesc) * count);
    if (ce == cudaSuccess) ce = cudaMemcpy(p->dmem, d, sizeof(LrDesc) * count, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        free_plan(p);
        return cuda_fail(ce, "chain plan upload");
    }
    p->d_lr = (LrDesc*)p->dmem;
    if (!fused) {
        size_t elems = 0;
        for (size_t e = 0; e < count; ++e) elems += 2 * (size_t)d[e].ra * d[e].rb;
        p->lr_work_bytes = elems * 8;
        ce = cudaMalloc(&p->lr_work, p->lr_work_bytes);
        if (ce != cudaSuccess) {
            free_plan(p);
            return fail(LRB_ERR_NOMEM, "chain temporaries");
        }
        std::vector<lrb_gemm_desc> s1(count), s2(count), s3(count);
        double* w = (double*)p->lr_work;
        for (size_t e = 0; e < count; ++e) {
            const lrb_lr_desc& x = d[e];
            double* Ct = w;
            double* Et = w + (size_t)x.ra * x.rb;
            w += 2 * (size_t)x.ra * x.rb;
            s1[e] = lrb_gemm_desc{x.AVT, x.BU, Ct, x.ra, x.rb, x.k, x.ld_avt, x.ld_bu, x.ra};
            s2[e] = lrb_gemm_desc{x.AX, Ct, Et, x.ra, x.rb, x.ra, x.ld_ax, x.ra, x.ra};
            s3[e] = lrb_gemm_desc{Et, x.BX, x.G, x.ra, x.rb, x.rb, x.ra, x.ld_bx, x.ldg};
        }
        lrb_plan_opts o = default_opts();
        o.use_graph = 1;
        o.check_alias = 0;
        o.overwrite = 1;   // C_temp, E_temp and G are written, as Alg. 1 assigns them
        const std::vector<lrb_gemm_desc>* st[3] = {&s1, &s2, &s3};
        for (int i = 0; i < 3; ++i) {
            lrb_status r = lrb_plan_create(h, st[i]->data(), count, &o, &p->lr_stage[i]);
            if (r != LRB_OK) {
                free_plan(p);
                return r;
            }
        }
        p->info.items = p->lr_stage[0]->info.items + p->lr_stage[1]->info.items + p->lr_stage[2]->info.items;
        p->info.groups = 3;
    }
    *out = p;
    return LRB_OK;
}

lrb_status lrb_plan_get_info(const lrb_plan* p, lrb_plan_info* info) {
    if (!p || !info) return fail(LRB_ERR_INVALID, "NULL argument");
    *info = p->info;
    return LRB_OK;
}

lrb_status lrb_plan_destroy(lrb_plan* p) {
    if (!p) return fail(LRB_ERR_INVALID, "plan is NULL");
    cudaSetDevice(p->h->device);
    if (p->launched) {
        cudaError_t e = p->last_stream ? cudaStreamSynchronize(p->last_stream) : cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            free_plan(p);
            return cuda_fail(e, "synchronise before free");
        }
    }
    free_plan(p);
    return LRB_OK;
}

}  // extern "C"
