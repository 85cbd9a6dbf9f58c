// Serving loop with continuous batching.
//
// Requests (device keys, n, type) are submitted from any thread and admitted
// against an HBM budget: a request reserves the device memory its sort needs
// (staging plus temporary buffers) and releases it on completion; one that
// could never fit is refused at submission.  Two worker lanes run on their own
// streams and contexts, so their work overlaps on the GPU:
//   - the batch lane folds every admitted request below the large-request
//     cutoff into one batched launch (gathered into a staging arena, sorted
//     by the batched path, scattered back), and keeps folding new arrivals
//     into the next batch while one is on the GPU;
//   - the large lane sorts big requests one by one with the single-array path.
// Latency is measured on the host from submission to completion.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ctx.h"
#include "internal.h"

// The workload module's device generators (linked into the library), used for
// requests whose keys the library generates (AHS_REQ_GENERATE).
extern "C" {
int gen_uniform_u32(void* out, unsigned long long n, unsigned long long seed,
                    unsigned long long stream, unsigned long long m, unsigned long long start,
                    void* st);
int gen_zipf_u32(void* out, unsigned long long n, unsigned long long seed, unsigned long long stream,
                 const void* d_cdf, const void* d_values, unsigned nv, unsigned long long start,
                 void* st);
int gen_replace_u32(void* a, unsigned long long n, unsigned long long seed, unsigned long long stream,
                    unsigned long long thresh53, void* st);
void gen_zipf_cdf_host(double* out, unsigned nv, double s);
void gen_zipf_values_host(uint32_t* out, unsigned long long seed, unsigned long long stream,
                          unsigned nv);
}

namespace ahs {
ahs_status run_batch(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin, uint32_t* vout,
                     const uint64_t* offs, uint32_t n_seg, KeyDesc kd, cudaStream_t st,
                     ahs_batch_info_t* info);

namespace {
using clock = std::chrono::steady_clock;

// Requests at or above this size go to the large lane.
constexpr uint64_t kLargeKeys = 1ull << 22;
// A batch folds requests up to this many keys (bounded arena).
constexpr uint64_t kBatchKeys = 1ull << 27;

struct Request {
    uint64_t ticket;
    ahs_request_t req;
    uint64_t reserve;
    clock::time_point submitted, admitted;
    bool large;
    bool payload() const { return req.d_vals_in != nullptr; }
    const void* keys_src() const {
        return (req.flags & AHS_REQ_GENERATE) ? req.d_keys_out : req.d_keys_in;
    }
};

// Generated requests: Zipf(1.1) over 1,024 values, 1% replacements.
constexpr unsigned kGenZipfValues = 1024;
constexpr double kGenZipfS = 1.1;
constexpr unsigned long long kGenReplace53 = 90071992547410ull;
unsigned long long gen_stream(uint64_t id, unsigned part) { return (1ull << 40) + 4ull * id + part; }

// Per-lane generator tables: the Zipf CDF (constant) and one request's values.
struct LaneGen {
    double* d_cdf = nullptr;
    uint32_t* d_vals = nullptr;
    uint32_t* h_vals = nullptr;   // pinned
    ~LaneGen() {
        if (d_cdf) cudaFree(d_cdf);
        if (h_vals) cudaFreeHost(h_vals);
    }
    cudaError_t init() {
        if (d_cdf) return cudaSuccess;
        cudaError_t e = cudaMalloc(&d_cdf, kGenZipfValues * (sizeof(double) + sizeof(uint32_t)));
        if (e != cudaSuccess) return e;
        d_vals = reinterpret_cast<uint32_t*>(d_cdf + kGenZipfValues);
        e = cudaHostAlloc(&h_vals, kGenZipfValues * sizeof(double), cudaHostAllocDefault);
        if (e != cudaSuccess) return e;
        gen_zipf_cdf_host(reinterpret_cast<double*>(h_vals), kGenZipfValues, kGenZipfS);
        e = cudaMemcpy(d_cdf, h_vals, kGenZipfValues * sizeof(double), cudaMemcpyHostToDevice);
        return e;
    }
};

// Write a generated request's keys into its output buffer (sorted in place
// afterwards).  Kind 3 sorts uniform keys with the lane's context first.
ahs_status generate_keys(ahs_ctx* c, const ahs_request_t& r, cudaStream_t st, LaneGen& g) {
    cudaError_t e = g.init();
    if (e != cudaSuccess) return cuda_status(c, e);
    const unsigned long long n = r.n, seed = r.gen_seed;
    const unsigned long long s0 = gen_stream(r.gen_id, 0);
    int rc = 0;
    switch (r.gen_kind) {
    case 0: rc = gen_uniform_u32(r.d_keys_out, n, seed, s0, 4096, 0, st); break;
    case 1:
        gen_zipf_values_host(g.h_vals, seed, gen_stream(r.gen_id, 1), kGenZipfValues);
        e = cudaMemcpyAsync(g.d_vals, g.h_vals, kGenZipfValues * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // h_vals is reused next
        if (e != cudaSuccess) return cuda_status(c, e);
        rc = gen_zipf_u32(r.d_keys_out, n, seed, s0, g.d_cdf, g.d_vals, kGenZipfValues, 0, st);
        break;
    case 2: rc = gen_uniform_u32(r.d_keys_out, n, seed, s0, 1ull << 32, 0, st); break;
    case 3: {
        rc = gen_uniform_u32(r.d_keys_out, n, seed, s0, 1ull << 32, 0, st);
        if (rc) break;
        ahs_status as = ahs_sort(c, r.d_keys_out, r.d_keys_out, nullptr, nullptr, n, AHS_U32,
                                 AHS_AUTO, st, nullptr);
        if (as != AHS_OK) return as;
        rc = gen_replace_u32(r.d_keys_out, n, seed, gen_stream(r.gen_id, 2), kGenReplace53, st);
        break;
    }
    default: return AHS_ERR_INVALID_ARG;
    }
    return rc ? cuda_status(c, (cudaError_t)rc) : AHS_OK;
}

struct Done {
    ahs_result_t res;
};

uint64_t reserve_for(const ahs_request_t& r) {
    const uint64_t w = ((r.type == AHS_U32 || r.type == AHS_I32) ? 4 : 8) + (r.d_vals_in ? 4 : 0);
    // Temporary keys (and payload) + partition metadata (about n/4 bytes) + a
    // fixed part; batched requests also occupy the staging arena (in + out).
    return r.n * w * 3 + r.n / 4 + (1ull << 20);
}

}  // namespace

struct ServeState {
    ahs_serve_config_t cfg{};
    ahs_ctx* batch_ctx = nullptr;   // own workspace per lane
    ahs_ctx* large_ctx = nullptr;
    cudaStream_t batch_stream = nullptr, large_stream = nullptr;
    int device = 0;

    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::deque<Request> queue;            // submitted, waiting for admission
    std::deque<Request> batch_ready, large_ready;
    std::unordered_map<uint64_t, Done> done;
    uint64_t next_ticket = 1;
    uint64_t reserved = 0, peak_reserved = 0;
    uint32_t inflight = 0;
    bool stopping = false;

    std::vector<double> latencies;
    uint64_t completed = 0, keys = 0, batches = 0;

    // Staging arena of the batch lane (device), grown on demand.
    void* arena = nullptr;
    size_t arena_bytes = 0;
    LaneGen batch_gen, large_gen;
    CopyItem* copy_items = nullptr;   // pinned gather / scatter lists of the batch lane
    size_t copy_cap = 0;
    std::thread batch_thread, large_thread;

    // Move queued requests into the lanes while budget and slots allow (FIFO).
    void admit_locked() {
        while (!queue.empty()) {
            Request& r = queue.front();
            if (inflight >= cfg.max_inflight || reserved + r.reserve > cfg.budget_bytes) break;
            reserved += r.reserve;
            peak_reserved = std::max(peak_reserved, reserved);
            ++inflight;
            r.admitted = clock::now();
            (r.large ? large_ready : batch_ready).push_back(r);
            queue.pop_front();
        }
    }

    void finish_locked(const Request& r, ahs_status st, ahs_strategy strategy) {
        const auto now = clock::now();
        Done d{};
        d.res.status = st;
        d.res.strategy = strategy;
        d.res.latency_ms = std::chrono::duration<double, std::milli>(now - r.submitted).count();
        d.res.queue_ms = std::chrono::duration<double, std::milli>(r.admitted - r.submitted).count();
        done[r.ticket] = d;
        reserved -= r.reserve;
        --inflight;
        if (st == AHS_OK) {
            latencies.push_back(d.res.latency_ms);
            ++completed;
            keys += r.req.n;
        }
        admit_locked();
    }

    void large_loop() {
        cudaSetDevice(device);
        for (;;) {
            Request r;
            {
                std::unique_lock<std::mutex> lk(mu);
                work_cv.wait(lk, [&] { return stopping || !large_ready.empty(); });
                if (large_ready.empty()) return;
                r = large_ready.front();
                large_ready.pop_front();
            }
            ahs_sort_info_t info{};
            ahs_status st = AHS_OK;
            if (r.req.flags & AHS_REQ_GENERATE) st = generate_keys(large_ctx, r.req, large_stream, large_gen);
            if (st == AHS_OK)
                st = ahs_sort(large_ctx, r.keys_src(), r.req.d_keys_out, r.req.d_vals_in,
                              r.req.d_vals_out, r.req.n, r.req.type, AHS_AUTO, large_stream, &info);
            std::lock_guard<std::mutex> lk(mu);
            finish_locked(r, st, info.strategy);
            done_cv.notify_all();
            work_cv.notify_all();
        }
    }

    void batch_loop() {
        cudaSetDevice(device);
        for (;;) {
            std::vector<Request> batch;
            {
                std::unique_lock<std::mutex> lk(mu);
                work_cv.wait_for(lk, std::chrono::microseconds(cfg.tick_us ? cfg.tick_us : 200),
                                 [&] { return stopping || !batch_ready.empty(); });
                if (batch_ready.empty()) {
                    if (stopping) return;
                    continue;
                }
                // Fold every ready request of one key type (with or without a
                // payload), up to the arena bound.
                uint64_t nk = 0;
                const ahs_key_type t = batch_ready.front().req.type;
                const bool pay = batch_ready.front().payload();
                for (auto it = batch_ready.begin(); it != batch_ready.end();) {
                    if (it->req.type == t && it->payload() == pay &&
                        (batch.empty() || nk + it->req.n <= kBatchKeys)) {
                        nk += it->req.n;
                        batch.push_back(*it);
                        it = batch_ready.erase(it);
                    } else {
                        ++it;
                    }
                }
            }
            const ahs_status st = run_one_batch(batch);
            std::lock_guard<std::mutex> lk(mu);
            ++batches;
            for (const Request& r : batch) finish_locked(r, st, AHS_AUTO);
            done_cv.notify_all();
            work_cv.notify_all();
        }
    }

    ahs_status run_one_batch(const std::vector<Request>& batch) {
        const KeyDesc kd = key_desc(batch[0].req.type);
        const bool pay = batch[0].payload();
        std::vector<uint64_t> offs(batch.size() + 1, 0);
        for (size_t i = 0; i < batch.size(); ++i) offs[i + 1] = offs[i] + batch[i].req.n;
        const uint64_t n = offs.back();
        for (const Request& r : batch) {
            if (!(r.req.flags & AHS_REQ_GENERATE)) continue;
            const ahs_status gs = generate_keys(batch_ctx, r.req, batch_stream, batch_gen);
            if (gs != AHS_OK) return gs;
        }
        const size_t kbytes = (n * kd.bytes + 255) & ~size_t(255);
        const size_t vbytes = pay ? ((n * 4 + 255) & ~size_t(255)) : 0;
        const size_t need = 2 * (kbytes + vbytes);
        if (need > arena_bytes) {
            if (arena) cudaFree(arena);
            arena = nullptr;
            arena_bytes = 0;
            if (cudaMalloc(&arena, need + need / 2) != cudaSuccess) {
                cudaGetLastError();
                return AHS_ERR_OOM;
            }
            arena_bytes = need + need / 2;
        }
        char* in = static_cast<char*>(arena);
        char* out = in + kbytes;
        uint32_t* vin = pay ? reinterpret_cast<uint32_t*>(out + kbytes) : nullptr;
        uint32_t* vout = pay ? reinterpret_cast<uint32_t*>(out + kbytes + vbytes) : nullptr;
        // Gather every request into the arena with one launch (items read
        // in place from pinned host memory; the lane waits for the batch
        // before it rewrites them).
        std::vector<CopyItem> items;
        auto add = [&](void* d, const void* src, uint64_t words) {
            for (uint64_t o = 0; o < words; o += kCopyItemWords)
                items.push_back({static_cast<uint32_t*>(d) + o, static_cast<const uint32_t*>(src) + o,
                                 std::min(kCopyItemWords, words - o)});
        };
        for (size_t i = 0; i < batch.size(); ++i) {
            add(in + offs[i] * kd.bytes, batch[i].keys_src(), batch[i].req.n * kd.bytes / 4);
            if (pay) add(vin + offs[i], batch[i].req.d_vals_in, batch[i].req.n);
        }
        const size_t n_gather = items.size();
        for (size_t i = 0; i < batch.size(); ++i) {
            add(batch[i].req.d_keys_out, out + offs[i] * kd.bytes, batch[i].req.n * kd.bytes / 4);
            if (pay) add(batch[i].req.d_vals_out, vout + offs[i], batch[i].req.n);
        }
        cudaError_t e = cudaSuccess;
        if (items.size() > copy_cap) {
            if (copy_items) cudaFreeHost(copy_items);
            copy_items = nullptr;
            copy_cap = 0;
            e = cudaHostAlloc(reinterpret_cast<void**>(&copy_items), items.size() * 2 * sizeof(CopyItem),
                              cudaHostAllocDefault);
            if (e != cudaSuccess) {
                copy_items = nullptr;
                return cuda_status(batch_ctx, e);
            }
            copy_cap = items.size() * 2;
        }
        std::memcpy(copy_items, items.data(), items.size() * sizeof(CopyItem));
        e = launch_copy_list(copy_items, (uint32_t)n_gather, n * (kd.bytes / 4 + (pay ? 1 : 0)),
                             batch_ctx->sms, batch_stream);
        if (e != cudaSuccess) return cuda_status(batch_ctx, e);
        ahs_batch_info_t info;
        ahs_status st = run_batch(batch_ctx, in, out, vin, vout, offs.data(),
                                  (uint32_t)batch.size(), kd, batch_stream, &info);
        if (st != AHS_OK) return st;
        e = launch_copy_list(copy_items + n_gather, (uint32_t)(items.size() - n_gather),
                             n * (kd.bytes / 4 + (pay ? 1 : 0)), batch_ctx->sms, batch_stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(batch_stream);
        return cuda_status(batch_ctx, e);
    }
};

}  // namespace ahs

using ahs::ServeState;

extern "C" {

ahs_status ahs_serve_start(ahs_ctx* ctx, const ahs_serve_config_t* cfg) {
    if (!ctx || ctx->device < 0 || !cfg || cfg->budget_bytes == 0 || cfg->max_inflight == 0)
        return AHS_ERR_INVALID_ARG;
    if (ctx->serve) return AHS_ERR_INVALID_ARG;
    auto* s = new (std::nothrow) ServeState();
    if (!s) return AHS_ERR_OOM;
    s->cfg = *cfg;
    s->device = ctx->device;
    ahs_config_t c = ctx->cfg;
    c.timing = 0;
    ahs_status rc = ahs_create(&s->batch_ctx, &c);
    if (rc == AHS_OK) rc = ahs_create(&s->large_ctx, &c);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (rc == AHS_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->batch_stream, cudaStreamNonBlocking);
    if (rc == AHS_OK && e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->large_stream, cudaStreamNonBlocking);
    if (rc == AHS_OK && e != cudaSuccess) rc = ahs::cuda_status(ctx, e);
    if (rc != AHS_OK) {
        if (s->batch_ctx) ahs_destroy(s->batch_ctx);
        if (s->large_ctx) ahs_destroy(s->large_ctx);
        if (s->batch_stream) cudaStreamDestroy(s->batch_stream);
        if (s->large_stream) cudaStreamDestroy(s->large_stream);
        delete s;
        return rc;
    }
    ctx->serve = s;
    s->batch_thread = std::thread([s] { s->batch_loop(); });
    s->large_thread = std::thread([s] { s->large_loop(); });
    return AHS_OK;
}

ahs_status ahs_serve_submit(ahs_ctx* ctx, const ahs_request_t* req, uint64_t* ticket) {
    if (!ctx || !req || !ticket) return AHS_ERR_INVALID_ARG;
    ServeState* s = ctx->serve;
    if (!s) return AHS_ERR_INVALID_ARG;
    if (req->type < AHS_U32 || req->type > AHS_I64) return AHS_ERR_DTYPE;
    if (req->flags & ~AHS_REQ_GENERATE) return AHS_ERR_INVALID_ARG;
    const bool gen = (req->flags & AHS_REQ_GENERATE) != 0;
    if (gen && (req->type != AHS_U32 || req->d_vals_in || req->gen_kind > 3))
        return AHS_ERR_INVALID_ARG;
    if (req->n && (!req->d_keys_out || (!gen && !req->d_keys_in))) return AHS_ERR_INVALID_ARG;
    if (req->n && req->d_vals_in && !req->d_vals_out) return AHS_ERR_INVALID_ARG;
    ahs::Request r{};
    r.req = *req;
    r.reserve = ahs::reserve_for(*req);
    r.large = req->n >= ahs::kLargeKeys;
    r.submitted = ahs::clock::now();
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stopping) return AHS_ERR_INVALID_ARG;
    if (r.reserve > s->cfg.budget_bytes) return AHS_ERR_BUDGET;
    r.ticket = s->next_ticket++;
    *ticket = r.ticket;
    if (req->n == 0) {
        ahs::Done d{};
        d.res.status = AHS_OK;
        d.res.strategy = AHS_IDENTITY;
        s->done[r.ticket] = d;
        return AHS_OK;
    }
    s->queue.push_back(r);
    s->admit_locked();
    s->work_cv.notify_all();
    return AHS_OK;
}

ahs_status ahs_serve_poll(ahs_ctx* ctx, uint64_t ticket, int32_t timeout_ms, ahs_result_t* out) {
    if (!ctx || !out) return AHS_ERR_INVALID_ARG;
    ServeState* s = ctx->serve;
    if (!s) return AHS_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return AHS_ERR_NOT_FOUND;
    auto ready = [&] { return s->done.count(ticket) != 0; };
    if (!ready() && timeout_ms > 0)
        s->done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) return AHS_ERR_AGAIN;
    *out = it->second.res;
    s->done.erase(it);
    return AHS_OK;
}

ahs_status ahs_serve_stats(ahs_ctx* ctx, ahs_serve_stats_t* out) {
    if (!ctx || !out || !ctx->serve) return AHS_ERR_INVALID_ARG;
    ServeState* s = ctx->serve;
    std::lock_guard<std::mutex> lk(s->mu);
    std::memset(out, 0, sizeof(*out));
    out->completed = s->completed;
    out->keys = s->keys;
    out->peak_reserved_bytes = s->peak_reserved;
    out->batches = s->batches;
    if (!s->latencies.empty()) {
        std::vector<double> v = s->latencies;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (v.size() - 1) + 0.5))]; };
        out->p50_ms = pct(0.50);
        out->p99_ms = pct(0.99);
    }
    return AHS_OK;
}

ahs_status ahs_serve_stop(ahs_ctx* ctx) {
    if (!ctx) return AHS_ERR_INVALID_ARG;
    ServeState* s = ctx->serve;
    if (!s) return AHS_OK;
    {
        std::unique_lock<std::mutex> lk(s->mu);
        // Drain: wait until everything submitted has completed.
        s->done_cv.wait(lk, [&] { return s->queue.empty() && s->inflight == 0; });
        s->stopping = true;
    }
    s->work_cv.notify_all();
    if (s->batch_thread.joinable()) s->batch_thread.join();
    if (s->large_thread.joinable()) s->large_thread.join();
    cudaSetDevice(s->device);
    if (s->arena) cudaFree(s->arena);
    if (s->copy_items) cudaFreeHost(s->copy_items);
    cudaStreamDestroy(s->batch_stream);
    cudaStreamDestroy(s->large_stream);
    ahs_destroy(s->batch_ctx);
    ahs_destroy(s->large_ctx);
    delete s;
    ctx->serve = nullptr;
    return AHS_OK;
}

}  // extern "C"
