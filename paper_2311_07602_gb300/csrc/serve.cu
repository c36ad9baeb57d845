// Serving queue: continuous batching of multiplication requests.
//
// A request is a small batch of entries (device operands, caller-owned).
// Submission is non-blocking: it validates the request, checks it against
// the queue's HBM budget (the bytes of its operands and results plus the
// planner's per-entry workspace) and appends it to a FIFO, or refuses it
// (LRB_ERR_BUDGET: larger than the whole budget; LRB_ERR_QUEUE_FULL: the
// FIFO is at its limit -- back-pressure).  One worker thread:
//   * retires finished waves (cudaEventQuery on each stream slot), marks
//     their requests done, releases their budget and records latency from
//     submission to the moment the completion was observed;
//   * for every free stream slot forms the next wave from the head of the
//     FIFO -- as many requests as fit in the budget left (FIFO order, no
//     overtaking) -- and launches it as one persistent tile-queue launch on
//     that slot's stream (tiles of every request in one list, longest
//     first).  Requests that arrive while earlier waves run join the next
//     wave as soon as a slot and budget free up; waves on different slots
//     overlap on the device.
// Tile variants come from the handle's tuned cache (else the untuned
// heuristic), and depend only on an entry's shape, so a request's result is
// bitwise the same alone or in any mix.  Every wait is bounded.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "lrb_internal.h"
#include "split.h"

using Clock = std::chrono::steady_clock;
using namespace lrb;

namespace {

enum ReqState { kWaiting = 0, kRunning = 1, kDone = 2, kFailed = 3 };

struct Request {
    uint64_t ticket = 0;
    std::vector<lrb_gemm_desc> descs;
    size_t bytes = 0;
    double flops = 0;
    Clock::time_point t_submit;
    ReqState state = kWaiting;
    double latency_ms = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* dmem = nullptr;
    size_t dmem_bytes = 0;
    int* h_status = nullptr;   // pinned: split-kernel status of the wave in flight
    bool split = false;        // the wave in flight runs in split precision
    std::vector<Request*> reqs;
    bool busy = false;
};

double ms_between(Clock::time_point a, Clock::time_point b) {
    return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t request_bytes(const lrb_gemm_desc* d, size_t n) {
    size_t b = 0;
    for (size_t e = 0; e < n; ++e)
        b += 8ull * ((size_t)d[e].m * d[e].k + (size_t)d[e].k * d[e].n + (size_t)d[e].m * d[e].n) + 64;
    return b;
}

}  // namespace

struct lrb_queue {
    lrb_handle* h = nullptr;
    HandleInfo hi{};
    size_t budget = 0;
    size_t reserved = 0;
    size_t peak_reserved = 0;
    size_t max_waiting = 4096;
    size_t max_wave_entries = 1 << 16;
    int precision = LRB_PREC_FP64;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> waiting;
    std::unordered_map<uint64_t, Request*> reqs;
    uint64_t next_ticket = 1;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    bool abandon = false;
    // statistics
    uint64_t accepted = 0, rejected_budget = 0, rejected_full = 0, rejected_invalid = 0;
    uint64_t completed = 0, failed = 0, waves = 0, wave_entries = 0, max_concurrent_waves = 0;
    std::vector<double> lat;
    double flops_done = 0;
    Clock::time_point t_first{}, t_last{};
    bool any = false;
    std::string worker_error;
};

namespace {

// Build and launch one wave on slot s (called without the queue lock).
lrb_status launch_split_wave(lrb_queue* q, Slot& s, const std::vector<lrb_gemm_desc>& all, int precision) {
    (void)q;
    std::vector<split::STile> items;
    split::build_items(all.data(), all.size(), items);
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_items = 0;
    const size_t o_status = o_items + align(sizeof(split::STile) * std::max<size_t>(items.size(), 1));
    const size_t need = o_status + 256;
    if (need > s.dmem_bytes) {
        if (s.dmem) cudaFreeAsync(s.dmem, s.stream);
        s.dmem = nullptr;
        s.dmem_bytes = 0;
        const size_t want = need + need / 2;
        if (cudaMallocAsync(&s.dmem, want, s.stream) != cudaSuccess) return LRB_ERR_NOMEM;
        s.dmem_bytes = want;
    }
    char* base = (char*)s.dmem;
    int* d_status = (int*)(base + o_status);
    cudaError_t e = cudaMemcpyAsync(base + o_items, items.data(), sizeof(split::STile) * items.size(),
                                    cudaMemcpyHostToDevice, s.stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, sizeof(int), s.stream);
    if (e == cudaSuccess)
        e = split::launch_raw(precision, (const split::STile*)(base + o_items), (int)items.size(), d_status,
                              s.stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(s.h_status, d_status, sizeof(int), cudaMemcpyDeviceToHost, s.stream);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    return e == cudaSuccess ? LRB_OK : LRB_ERR_DEVICE;
}

lrb_status launch_wave(lrb_queue* q, Slot& s, int precision) {
    std::vector<lrb_gemm_desc> all;
    for (Request* r : s.reqs) all.insert(all.end(), r->descs.begin(), r->descs.end());
    if (precision >= LRB_PREC_SPLIT_BF16_S3) return launch_split_wave(q, s, all, precision);
    lrb_plan_opts o = default_plan_opts();
    o.tune = 0;
    o.check_alias = 0;
    std::vector<int> var;
    lrb_status st = plan_variants(q->h, all.data(), all.size(), o, var);
    if (st != LRB_OK) return st;
    std::vector<Item> items;
    plan_tiles(all.data(), all.size(), var, items);
    int set = 0;
    for (int v : var) set = std::max(set, variant_set(v));
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t o_items = align(sizeof(DevDesc) * all.size());
    const size_t o_head = o_items + align(sizeof(Item) * std::max<size_t>(items.size(), 1));
    const size_t need = o_head + 256;
    if (need > s.dmem_bytes) {
        if (s.dmem) cudaFreeAsync(s.dmem, s.stream);
        s.dmem = nullptr;
        s.dmem_bytes = 0;
        const size_t want = need + need / 2;
        if (cudaMallocAsync(&s.dmem, want, s.stream) != cudaSuccess) return LRB_ERR_NOMEM;
        s.dmem_bytes = want;
    }
    char* base = (char*)s.dmem;
    DevDesc* d_descs = (DevDesc*)base;
    Item* d_items = (Item*)(base + o_items);
    int* d_head = (int*)(base + o_head);
    cudaError_t e = cudaMemcpyAsync(d_descs, all.data(), sizeof(DevDesc) * all.size(), cudaMemcpyHostToDevice,
                                    s.stream);
    if (e == cudaSuccess && !items.empty())
        e = cudaMemcpyAsync(d_items, items.data(), sizeof(Item) * items.size(), cudaMemcpyHostToDevice, s.stream);
    // pageable sources: the copies above are staged before they return, so
    // the host vectors may go out of scope
    const int per_sm = set == 0 ? q->hi.blocks_per_sm_slim : set == 1 ? q->hi.blocks_per_sm : q->hi.blocks_per_sm_wide;
    const int grid = std::max(1, std::min(q->hi.sms * per_sm, (int)items.size()));
    if (e == cudaSuccess) e = launch_persistent(d_descs, d_items, (int)items.size(), d_head, grid, s.stream, set);
    if (e == cudaSuccess) e = cudaEventRecord(s.done, s.stream);
    return e == cudaSuccess ? LRB_OK : LRB_ERR_DEVICE;
}

void worker_main(lrb_queue* q) {
    cudaSetDevice(q->hi.device);
    std::unique_lock<std::mutex> lk(q->mu);
    for (;;) {
        if (q->abandon) break;
        bool progressed = false;
        // retire finished waves
        uint64_t busy = 0;
        for (Slot& s : q->slots) {
            if (!s.busy) continue;
            cudaError_t e = cudaEventQuery(s.done);
            if (e == cudaErrorNotReady) {
                ++busy;
                continue;
            }
            const Clock::time_point now = Clock::now();
            const bool wait_expired = e == cudaSuccess && s.split && *s.h_status != 0;
            for (Request* r : s.reqs) {
                q->reserved -= r->bytes;
                r->latency_ms = ms_between(r->t_submit, now);
                if (e == cudaSuccess && !wait_expired) {
                    r->state = kDone;
                    ++q->completed;
                    q->lat.push_back(r->latency_ms);
                    q->flops_done += r->flops;
                } else {
                    r->state = kFailed;
                    ++q->failed;
                }
            }
            if (e != cudaSuccess) q->worker_error = cudaGetErrorString(e);
            if (wait_expired) q->worker_error = "a bounded device wait expired in a split-precision wave";
            s.reqs.clear();
            s.busy = false;
            q->t_last = now;
            progressed = true;
        }
        if (progressed) q->cv_done.notify_all();
        // admit the next waves
        for (Slot& s : q->slots) {
            if (s.busy || q->waiting.empty()) continue;
            size_t wave_bytes = 0, entries = 0;
            while (!q->waiting.empty()) {
                Request* r = q->waiting.front();
                if (q->reserved + wave_bytes + r->bytes > q->budget) break;
                if (!s.reqs.empty() && entries + r->descs.size() > q->max_wave_entries) break;
                s.reqs.push_back(r);
                wave_bytes += r->bytes;
                entries += r->descs.size();
                q->waiting.pop_front();
            }
            if (s.reqs.empty()) break;   // the head request waits for budget
            q->reserved += wave_bytes;
            q->peak_reserved = std::max(q->peak_reserved, q->reserved);
            for (Request* r : s.reqs) r->state = kRunning;
            const int precision = q->precision;
            s.split = precision >= LRB_PREC_SPLIT_BF16_S3;
            s.busy = true;
            ++busy;
            q->max_concurrent_waves = std::max<uint64_t>(q->max_concurrent_waves, busy);
            ++q->waves;
            q->wave_entries += entries;
            lk.unlock();
            const lrb_status st = launch_wave(q, s, precision);
            lk.lock();
            if (st != LRB_OK) {
                for (Request* r : s.reqs) {
                    q->reserved -= r->bytes;
                    r->state = kFailed;
                    ++q->failed;
                }
                q->worker_error = "wave launch failed";
                s.reqs.clear();
                s.busy = false;
                q->cv_done.notify_all();
            }
            progressed = true;
        }
        if (q->stop && q->waiting.empty()) {
            bool idle = true;
            for (Slot& s : q->slots) idle = idle && !s.busy;
            if (idle) break;
        }
        if (!progressed) q->cv_work.wait_for(lk, std::chrono::microseconds(50));
    }
}

lrb_status qfail(lrb_status s, const char* msg) {
    set_last_error(msg);
    return s;
}

}  // namespace

extern "C" {

lrb_status lrb_queue_create(lrb_handle* h, size_t hbm_budget_bytes, int max_inflight, lrb_queue** out) {
    if (!h || !out) return qfail(LRB_ERR_INVALID, "NULL argument");
    *out = nullptr;
    if (hbm_budget_bytes == 0) return qfail(LRB_ERR_INVALID, "hbm_budget_bytes is 0");
    if (max_inflight < 1 || max_inflight > 16) return qfail(LRB_ERR_INVALID, "max_inflight must be in 1..16");
    lrb_queue* q = new lrb_queue();
    q->h = h;
    q->hi = handle_info(h);
    q->budget = hbm_budget_bytes;
    if (cudaSetDevice(q->hi.device) != cudaSuccess) {
        delete q;
        return qfail(LRB_ERR_DEVICE, "cudaSetDevice");
    }
    q->slots.resize(max_inflight);
    for (Slot& s : q->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaMallocHost((void**)&s.h_status, sizeof(int)) != cudaSuccess) {
            for (Slot& t : q->slots) {
                if (t.done) cudaEventDestroy(t.done);
                if (t.stream) cudaStreamDestroy(t.stream);
                if (t.h_status) cudaFreeHost(t.h_status);
            }
            delete q;
            return qfail(LRB_ERR_DEVICE, "stream/event creation");
        }
    }
    q->worker = std::thread(worker_main, q);
    *out = q;
    return LRB_OK;
}

lrb_status lrb_queue_set_limits(lrb_queue* q, size_t max_waiting, size_t max_wave_entries) {
    if (!q || max_waiting == 0 || max_wave_entries == 0) return qfail(LRB_ERR_INVALID, "bad queue limits");
    std::lock_guard<std::mutex> lk(q->mu);
    q->max_waiting = max_waiting;
    q->max_wave_entries = max_wave_entries;
    return LRB_OK;
}

lrb_status lrb_queue_set_precision(lrb_queue* q, int32_t precision) {
    if (!q) return qfail(LRB_ERR_INVALID, "NULL queue");
    if (precision != LRB_PREC_FP64 && precision != LRB_PREC_FP64_DMMA_ALLOWED &&
        (precision < LRB_PREC_SPLIT_BF16_S3 || precision > LRB_PREC_SPLIT_FP16_S4))
        return qfail(LRB_ERR_INVALID, "unknown precision");
    std::lock_guard<std::mutex> lk(q->mu);
    q->precision = precision;
    return LRB_OK;
}

lrb_status lrb_queue_submit(lrb_queue* q, const lrb_gemm_desc* descs, size_t n, uint64_t* ticket) {
    if (!q || !ticket) return qfail(LRB_ERR_INVALID, "NULL argument");
    lrb_plan_opts o = default_plan_opts();
    lrb_status st = validate_descs(descs, n, o);
    if (st != LRB_OK) {
        std::lock_guard<std::mutex> lk(q->mu);
        ++q->rejected_invalid;
        return st;
    }
    const size_t bytes = request_bytes(descs, n);
    double flops = 0;
    for (size_t e = 0; e < n; ++e) flops += 2.0 * descs[e].m * descs[e].n * descs[e].k;
    std::lock_guard<std::mutex> lk(q->mu);
    if (bytes > q->budget) {
        ++q->rejected_budget;
        return qfail(LRB_ERR_BUDGET, "request alone exceeds the queue's HBM budget");
    }
    if (q->waiting.size() >= q->max_waiting) {
        ++q->rejected_full;
        return qfail(LRB_ERR_QUEUE_FULL, "too many requests waiting");
    }
    Request* r = new Request();
    r->ticket = q->next_ticket++;
    r->descs.assign(descs, descs + n);
    r->bytes = bytes;
    r->flops = flops;
    r->t_submit = Clock::now();
    if (!q->any) {
        q->any = true;
        q->t_first = r->t_submit;
    }
    q->reqs[r->ticket] = r;
    q->waiting.push_back(r);
    ++q->accepted;
    *ticket = r->ticket;
    q->cv_work.notify_one();
    return LRB_OK;
}

lrb_status lrb_queue_poll(lrb_queue* q, uint64_t ticket) {
    if (!q) return qfail(LRB_ERR_INVALID, "NULL queue");
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->reqs.find(ticket);
    if (it == q->reqs.end()) return qfail(LRB_ERR_INVALID, "unknown ticket");
    if (it->second->state == kDone) return LRB_OK;
    if (it->second->state == kFailed) return qfail(LRB_ERR_DEVICE, "request failed on the device");
    return LRB_ERR_TIMEOUT;
}

lrb_status lrb_queue_wait(lrb_queue* q, uint64_t ticket, int timeout_ms) {
    if (!q) return qfail(LRB_ERR_INVALID, "NULL queue");
    std::unique_lock<std::mutex> lk(q->mu);
    auto it = q->reqs.find(ticket);
    if (it == q->reqs.end()) return qfail(LRB_ERR_INVALID, "unknown ticket");
    Request* r = it->second;
    const int ms = timeout_ms < 0 ? 600000 : timeout_ms;
    const bool ok = q->cv_done.wait_for(lk, std::chrono::milliseconds(ms),
                                        [r] { return r->state == kDone || r->state == kFailed; });
    if (!ok) return qfail(LRB_ERR_TIMEOUT, "request not complete within the timeout");
    if (r->state == kFailed) return qfail(LRB_ERR_DEVICE, "request failed on the device");
    return LRB_OK;
}

lrb_status lrb_queue_latency(lrb_queue* q, uint64_t ticket, double* latency_ms) {
    if (!q || !latency_ms) return qfail(LRB_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    auto it = q->reqs.find(ticket);
    if (it == q->reqs.end()) return qfail(LRB_ERR_INVALID, "unknown ticket");
    if (it->second->state != kDone) return qfail(LRB_ERR_TIMEOUT, "request not complete");
    *latency_ms = it->second->latency_ms;
    return LRB_OK;
}

lrb_status lrb_queue_stats(lrb_queue* q, lrb_queue_stats_t* out) {
    if (!q || !out) return qfail(LRB_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(q->mu);
    std::memset(out, 0, sizeof(*out));
    out->accepted = q->accepted;
    out->rejected_budget = q->rejected_budget;
    out->rejected_full = q->rejected_full;
    out->rejected_invalid = q->rejected_invalid;
    out->completed = q->completed;
    out->failed = q->failed;
    out->waiting = q->waiting.size();
    out->waves = q->waves;
    out->max_concurrent_waves = q->max_concurrent_waves;
    out->mean_wave_entries = q->waves ? (double)q->wave_entries / (double)q->waves : 0.0;
    out->reserved_bytes = q->reserved;
    out->peak_reserved_bytes = q->peak_reserved;
    out->budget_bytes = q->budget;
    if (!q->lat.empty()) {
        std::vector<double> v = q->lat;
        std::sort(v.begin(), v.end());
        auto pct = [&](double p) {
            const double pos = p * (double)(v.size() - 1);
            const size_t i = (size_t)pos;
            const double f = pos - (double)i;
            return i + 1 < v.size() ? v[i] * (1 - f) + v[i + 1] * f : v[i];
        };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
        out->max_ms = v.back();
        double s = 0;
        for (double x : v) s += x;
        out->mean_ms = s / (double)v.size();
    }
    if (q->any && q->completed) {
        const double secs = ms_between(q->t_first, q->t_last) / 1e3;
        out->gflops = secs > 0 ? q->flops_done / secs / 1e9 : 0.0;
    }
    out->flops_done = q->flops_done;
    return LRB_OK;
}

lrb_status lrb_queue_destroy(lrb_queue* q, int timeout_ms) {
    if (!q) return qfail(LRB_ERR_INVALID, "NULL queue");
    lrb_status st = LRB_OK;
    {
        std::unique_lock<std::mutex> lk(q->mu);
        q->stop = true;
        q->cv_work.notify_all();
        const int ms = timeout_ms < 0 ? 600000 : timeout_ms;
        const bool drained = q->cv_done.wait_for(lk, std::chrono::milliseconds(ms), [q] {
            if (!q->waiting.empty()) return false;
            for (Slot& s : q->slots)
                if (s.busy) return false;
            return true;
        });
        if (!drained) {
            q->abandon = true;   // the worker stops polling; in-flight waves are left to finish
            st = qfail(LRB_ERR_TIMEOUT, "queue did not drain within the timeout");
        }
        q->cv_work.notify_all();
    }
    q->worker.join();
    for (Slot& s : q->slots) {
        if (!q->abandon) {
            if (s.dmem) cudaFreeAsync(s.dmem, s.stream);
            cudaStreamSynchronize(s.stream);
        }
        cudaEventDestroy(s.done);
        cudaStreamDestroy(s.stream);
        if (!q->abandon) cudaFreeHost(s.h_status);
    }
    for (auto& kv : q->reqs) delete kv.second;
    delete q;
    return st;
}

}  // extern "C"
