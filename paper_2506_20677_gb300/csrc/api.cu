// C ABI entry points: context, workspace, features, selection, single-array sort.
#include <cstdio>
#include <cstring>
#include <new>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "select.h"

using namespace ahs;

namespace ahs {

thread_local Tracer* g_tracer = nullptr;

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t features_region(int sms) { return align256(features_scratch_bytes(sms)); }

static FeatureScratch carve_features(ahs_ctx* ctx) {
    FeatureScratch s{};
    char* p = static_cast<char*>(ctx->ws);
    s.rec = ctx->d_rec;
    s.k1_partials = reinterpret_cast<unsigned long long*>(p);
    p += align256(3 * sizeof(unsigned long long) * 4 * (size_t)ctx->sms);
    s.slabs = reinterpret_cast<uint32_t*>(p);
    p += align256((size_t)ctx->sms * kMaxBins * sizeof(uint32_t));
    s.hist = reinterpret_cast<unsigned long long*>(p);
    p += align256(kMaxBins * sizeof(unsigned long long));
    s.ent_partials = reinterpret_cast<double*>(p);
    return s;
}

ahs_status cuda_status(ahs_ctx* ctx, cudaError_t e) {
    if (e == cudaSuccess) return AHS_OK;
    if (ctx) ctx->last_cuda_error = cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return AHS_ERR_OOM;
    return AHS_ERR_CUDA;
}

ahs_status ensure_workspace(ahs_ctx* ctx, size_t bytes) {
    bytes = align256(bytes);
    if (bytes <= ctx->ws_bytes) return AHS_OK;
    if (ctx->cfg.workspace_limit && bytes > ctx->cfg.workspace_limit) return AHS_ERR_OOM;
    if (ctx->ws) {
        cudaError_t e = cudaFree(ctx->ws);   // synchronises the device
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    // Grow geometrically to amortise reallocations.
    size_t want = bytes + bytes / 4;
    if (ctx->cfg.workspace_limit && want > ctx->cfg.workspace_limit) want = bytes;
    cudaError_t e = cudaMalloc(&ctx->ws, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        e = cudaMalloc(&ctx->ws, bytes);
        want = bytes;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return cuda_status(ctx, e);
    }
    ctx->ws_bytes = want;
    return AHS_OK;
}

void to_public(const DevFeatures& r, KeyDesc kd, ahs_features_t* out) {
    std::memset(out, 0, sizeof(*out));
    out->n = r.n;
    out->min_bits = r.min_ord ^ kd.flip;
    out->max_bits = r.max_ord ^ kd.flip;
    out->span = r.span;
    out->hist_shift = r.shift;
    out->nbins = r.nbins;
    out->entropy_bits = r.entropy;
    out->entropy_norm = r.entropy_norm;
    out->descents = r.descents;
    out->ascents = r.ascents;
}

ahs_status run_features(ahs_ctx* ctx, const void* d_keys, uint64_t n, KeyDesc kd,
                        cudaStream_t st, ahs_features_t* out, uint32_t skip_sorted) {
    // Room for the counting sort's prefix too: that strategy reads the
    // histogram in place, and growing the workspace would not keep it.
    ahs_status rc = ensure_workspace(ctx, features_region(ctx->sms) + align256((kMaxBins + 1) * 8));
    if (rc != AHS_OK) return rc;
    FeatureScratch s = carve_features(ctx);
    // K3 writes the record and the histogram into the pinned mirrors.
    s.host_rec = ctx->h_rec;
    s.host_hist = ctx->h_hist;
    s.skip_sorted = skip_sorted;
    const size_t mark = ctx->tracer.records.size();
    cudaError_t e = launch_features(d_keys, n, kd, s, ctx->sms, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    // A packed histogram counter wrapped: count again in the exact layout.
    if (e == cudaSuccess && (ctx->h_rec->k2_wrapped || (ctx->cfg.debug_flags & AHS_DEBUG_K2_SPLIT))) {
        e = launch_features_split_retry(d_keys, n, kd, s, ctx->sms, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
    if (e != cudaSuccess) return cuda_status(ctx, e);
    // The histogram kernel returned at once for an input found presorted: its
    // trace entry processed no keys.
    const DevFeatures& r = *ctx->h_rec;
    const bool skipped = ((skip_sorted & kSkipOrdered) && r.descents == 0) ||
                         ((skip_sorted & kSkipReversed) && r.ascents == 0) ||
                         ((skip_sorted & kSkipStrictReversed) && r.n >= 2 && r.descents == r.n - 1);
    if (skipped)
        for (size_t i = mark; i < ctx->tracer.records.size(); ++i)
            if (std::strcmp(ctx->tracer.records[i].name, "features_histogram") == 0)
                ctx->tracer.records[i].items = 0;
    to_public(*ctx->h_rec, kd, out);
    return AHS_OK;
}

uint32_t radix_digit_bits(const ahs_ctx* ctx, uint32_t key_bytes, bool payload, uint64_t span) {
    return ctx->tuning.radix_digit_bits(key_bytes, payload, bitlen64(span));
}

// Whether AUTO selection under the context's profile returns an input already
// in order as it is (IDENTITY) whatever its entropy.
bool sorted_identity(const ahs_ctx* ctx) {
    switch (ctx->cfg.select_mode) {
    case AHS_SEL_CUSTOM:
        return ctx->custom.sorted_identity != 0;
    case AHS_SEL_MODEL:   // ordered inputs take the rules (GB300 profile) before the trees
        return true;
    default: {
        ahs_thresholds_t t;
        return profile_thresholds(ctx->cfg.select_mode, &t) == AHS_OK && t.sorted_identity != 0;
    }
    }
}

bool reversed_input(const ahs_features_t& f, bool payload) {
    return f.n >= 2 && f.descents > 0 && f.ascents == 0 && (!payload || f.descents == f.n - 1);
}

ahs_strategy choose(const ahs_ctx* ctx, const ahs_features_t& f, uint32_t key_bytes, bool payload,
                    bool allow_reverse) {
    if (allow_reverse && reversed_input(f, payload)) return AHS_REVERSE;
    ahs_thresholds_t t;
    ahs_strategy s;
    switch (ctx->cfg.select_mode) {
    case AHS_SEL_MODEL:
        s = select_model(ctx->model, f, key_bytes, payload ? 1 : 0);
        break;
    case AHS_SEL_CUSTOM:
        s = select_fsm(f, ctx->custom);
        break;
    case AHS_SEL_LEMMA32:
        profile_thresholds(AHS_SEL_LEMMA32, &t);
        s = select_lemma32(f, t);
        break;
    default:
        profile_thresholds(ctx->cfg.select_mode, &t);
        s = select_fsm(f, t);
        break;
    }
    // Insertion-sort sized inputs run in one CTA; a profile whose n_t exceeds
    // that capacity sends the rest to the general path.
    if (s == AHS_SMALL && f.n > blocksort_capacity(key_bytes, payload)) s = AHS_GENERAL;
    // The counting sort reads the feature histogram (k <= 2^16): a counting
    // pick over a wider range runs the radix path, whose partition sizes are
    // the counts of the leading 16 bits.
    if (s == AHS_COUNTING && f.span >= kMaxBinsCounting) s = AHS_RADIX;
    return s;
}

ahs_status ensure_aux(ahs_ctx* ctx, size_t bytes) {
    bytes = align256(bytes);
    if (bytes <= ctx->aux_bytes) return AHS_OK;
    if (ctx->aux) {
        cudaError_t e = cudaFree(ctx->aux);
        ctx->aux = nullptr;
        ctx->aux_bytes = 0;
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    const size_t want = bytes + bytes / 2;
    cudaError_t e = cudaMalloc(&ctx->aux, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->aux = nullptr;
        return cuda_status(ctx, e);
    }
    ctx->aux_bytes = want;
    return AHS_OK;
}

ahs_status ensure_stage(ahs_ctx* ctx, size_t bytes) {
    bytes = align256(bytes);
    if (bytes <= ctx->h_stage_bytes) return AHS_OK;
    if (ctx->h_stage) {
        cudaError_t e = cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->h_stage_bytes = 0;
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    const size_t want = bytes + bytes / 2;
    cudaError_t e = cudaHostAlloc(&ctx->h_stage, want, cudaHostAllocDefault);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->h_stage = nullptr;
        return cuda_status(ctx, e);
    }
    ctx->h_stage_bytes = want;
    return AHS_OK;
}

ahs_status check_device_error(ahs_ctx* ctx, cudaStream_t st) {
    cudaError_t e = launch_transfer(ctx->h_err, ctx->d_err, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    const uint32_t code = *ctx->h_err;
    if (code == kDevOk) return AHS_OK;
    e = cudaMemsetAsync(ctx->d_err, 0, sizeof(uint32_t), st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    return (code == kDevLookbackTimeout || code == kDevCopyTimeout) ? AHS_ERR_DEVICE_TIMEOUT
                                                                     : AHS_ERR_CUDA;
}

// The feature histogram's nbins counts: the pinned mirror that the feature
// pass filled (it stays valid when the workspace grows).
static ahs_status host_histogram(ahs_ctx* ctx, const ahs_features_t& f, cudaStream_t,
                                 HistView* out) {
    if (f.nbins > kMaxBins) return AHS_ERR_INVALID_ARG;
    out->counts = ctx->h_hist;
    out->nbins = f.nbins;
    return AHS_OK;
}

ahs_status run_strategy(ahs_ctx* ctx, ahs_strategy s, const void* kin, void* kout,
                        const uint32_t* vin, uint32_t* vout, uint64_t n, KeyDesc kd,
                        const ahs_features_t& f, cudaStream_t st, uint32_t* passes,
                        uint32_t* buckets) {
    const size_t freg = features_region(ctx->sms);
    cudaError_t e = cudaSuccess;
    *passes = 0;
    *buckets = 0;
    const uint64_t min_ord = f.min_bits ^ kd.flip;
    switch (s) {
    case AHS_IDENTITY: {
        e = launch_copy32(kout, kin, n * kd.bytes / 4, ctx->sms, st);
        if (e == cudaSuccess && vin) e = launch_copy32(vout, vin, n, ctx->sms, st);
        return cuda_status(ctx, e);
    }
    case AHS_REVERSE: {
        // Only chosen for a reversed input (no ascents; strictly decreasing
        // with a payload, so that the reversal keeps equal keys stable).
        if (!reversed_input(f, vin != nullptr)) return AHS_ERR_INVALID_ARG;
        e = launch_reverse(kout, kin, n, kd.bytes, ctx->sms, st);
        if (e == cudaSuccess && vin) e = launch_reverse(vout, vin, n, 4, ctx->sms, st);
        *passes = 1;
        return cuda_status(ctx, e);
    }
    case AHS_SMALL: {
        if (n > blocksort_capacity(kd.bytes, vin != nullptr)) return AHS_ERR_RANGE;
        e = launch_blocksort_single(kin, kout, vin, vout, n, kd, st);
        return cuda_status(ctx, e);
    }
    case AHS_COUNTING: {
        if (f.span > 65535) return AHS_ERR_RANGE;   // k <= 2^16: bins are values
        if (!vin) {
            ahs_status rc = ensure_workspace(ctx, freg + align256((kMaxBins + 1) * 8));
            if (rc != AHS_OK) return rc;
            FeatureScratch fs = carve_features(ctx);
            unsigned long long* prefix =
                reinterpret_cast<unsigned long long*>(static_cast<char*>(ctx->ws) + freg);
            e = launch_counting_fill(kout, n, kd, ctx->d_rec, fs.hist, prefix, min_ord, f.nbins,
                                     ctx->sms, st);
            *passes = 1;
            return cuda_status(ctx, e);
        }
        // With a payload the stable rank-scatter of Listing 2 is the radix
        // pass machinery with digits spanning the whole (<= 16-bit) range.
        [[fallthrough]];
    }
    case AHS_RADIX: {
        if (s == AHS_RADIX && !vin && f.hist_shift > 0 && n >= 2 && n <= 0xffffffffull) {
            // Keys only: most significant digit first, unstable partitions.
            HistView hist;
            ahs_status rc = host_histogram(ctx, f, st, &hist);
            if (rc != AHS_OK) return rc;
            if (sparse_radix_fits(n, kd.bytes, f.span, hist)) {
                bool done = false;
                rc = run_sparse_radix(ctx, kin, kout, n, kd, min_ord, st, &done, buckets);
                if (rc != AHS_OK) return rc;
                if (done) {
                    *passes = 1;
                    return AHS_OK;
                }
            }
            const size_t need = samplesort_scratch_bytes(n, kd.bytes, false);
            rc = ensure_workspace(ctx, freg + need);
            if (rc != AHS_OK) return rc;
            return run_msd_radix(ctx, kin, kout, n, kd, min_ord, hist, f.hist_shift, group_slots(f),
                                 static_cast<char*>(ctx->ws) + freg, st, passes, buckets);
        }
        const RadixPlan plan = radix_plan(f.span, radix_digit_bits(ctx, kd.bytes, vin != nullptr, f.span));
        if (plan.passes == 0) {
            e = launch_copy32(kout, kin, n * kd.bytes / 4, ctx->sms, st);
            if (e == cudaSuccess && vin) e = launch_copy32(vout, vin, n, ctx->sms, st);
            return cuda_status(ctx, e);
        }
        if (n >= (1ull << 30)) return AHS_ERR_UNIMPLEMENTED;
        const size_t need = radix_scratch_bytes(n, kd.bytes, vin != nullptr, plan);
        ahs_status rc = ensure_workspace(ctx, freg + need);
        if (rc != AHS_OK) return rc;
        RadixScratch rs = radix_carve(static_cast<char*>(ctx->ws) + freg, n, kd.bytes,
                                      vin != nullptr, plan);
        e = launch_radix_sort(kin, kout, vin, vout, n, kd, min_ord, plan, rs, ctx->d_rec,
                              ctx->d_err, ctx->sms, st,
                              (ctx->cfg.debug_flags & AHS_DEBUG_STALL_ONE_TILE) ? 1u : ~0u);
        *passes = plan.passes;
        return cuda_status(ctx, e);
    }
    case AHS_GENERAL: {
        if (n >= (1ull << 32)) return AHS_ERR_UNIMPLEMENTED;
        HistView hist;
        const bool use_hist = !vin && f.nbins > 256;
        if (use_hist) {
            ahs_status rc = host_histogram(ctx, f, st, &hist);
            if (rc != AHS_OK) return rc;
        }
        const size_t need = samplesort_scratch_bytes(n, kd.bytes, vin != nullptr);
        ahs_status rc = ensure_workspace(ctx, freg + need);
        if (rc != AHS_OK) return rc;
        return run_samplesort(ctx, kin, kout, vin, vout, n, kd, static_cast<char*>(ctx->ws) + freg,
                              st, passes, buckets, use_hist ? &hist : nullptr, min_ord,
                              f.hist_shift, group_slots(f));
    }
    default:
        return AHS_ERR_INVALID_ARG;
    }
}

}  // namespace ahs

// ===================================================================== C ABI

extern "C" {

void ahs_default_config(ahs_config_t* cfg) {
    if (!cfg) return;
    std::memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->select_mode = AHS_SEL_GB300;
    profile_thresholds(AHS_SEL_GB300, &cfg->thresholds);
}

ahs_status ahs_profile_thresholds(ahs_select_mode mode, ahs_thresholds_t* out) {
    if (mode == AHS_SEL_CUSTOM || mode == AHS_SEL_LEMMA32) return AHS_ERR_INVALID_ARG;
    return profile_thresholds(mode, out);
}

const char* ahs_status_str(ahs_status s) {
    switch (s) {
    case AHS_OK: return "ok";
    case AHS_ERR_INVALID_ARG: return "invalid argument";
    case AHS_ERR_DTYPE: return "keys must be 32- or 64-bit integers";
    case AHS_ERR_OOM: return "device workspace allocation failed";
    case AHS_ERR_BUDGET: return "request exceeds the HBM budget";
    case AHS_ERR_CUDA: return "CUDA error";
    case AHS_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
    case AHS_ERR_AGAIN: return "not finished";
    case AHS_ERR_NOT_FOUND: return "not found";
    case AHS_ERR_UNIMPLEMENTED: return "not implemented for these arguments";
    case AHS_ERR_RANGE: return "forced strategy cannot handle this range or size";
    }
    return "unknown status";
}

ahs_status ahs_create(ahs_ctx** out, const ahs_config_t* cfg) {
    if (!out) return AHS_ERR_INVALID_ARG;
    *out = nullptr;
    ahs_ctx* ctx = new (std::nothrow) ahs_ctx();
    if (!ctx) return AHS_ERR_OOM;
    if (cfg) ctx->cfg = *cfg;
    else ahs_default_config(&ctx->cfg);
    if (ctx->cfg.select_mode < AHS_SEL_PAPER || ctx->cfg.select_mode > AHS_SEL_LEMMA32) {
        delete ctx;
        return AHS_ERR_INVALID_ARG;
    }
    ctx->custom = ctx->cfg.thresholds;
    ctx->device = ctx->cfg.device;
    if (ctx->cfg.tuning_path) {
        std::string why;
        if (!ctx->tuning.load(ctx->cfg.tuning_path, &why)) {
            delete ctx;
            return AHS_ERR_NOT_FOUND;
        }
    }
    if (ctx->device < 0) {
        // Host-only context: selection and model loading, no device work.
        if (ctx->cfg.model_path) {
            std::string why;
            if (!ctx->model.load(ctx->cfg.model_path, &why)) {
                delete ctx;
                return AHS_ERR_NOT_FOUND;
            }
        }
        *out = ctx;
        return AHS_OK;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    const size_t persist = 256 + 256;
    void* d = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d, persist);
    if (e == cudaSuccess) e = cudaMemset(d, 0, persist);
    void* h = nullptr;
    if (e == cudaSuccess) e = cudaHostAlloc(&h, persist + kMaxBins * sizeof(unsigned long long),
                                            cudaHostAllocDefault);
    for (int i = 0; e == cudaSuccess && i < 4; ++i) e = cudaEventCreate(&ctx->ev[i]);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        ahs_status rc = cuda_status(ctx, e);
        if (d) cudaFree(d);
        if (h) cudaFreeHost(h);
        delete ctx;
        return rc;
    }
    ctx->d_rec = static_cast<DevFeatures*>(d);
    ctx->d_err = reinterpret_cast<uint32_t*>(static_cast<char*>(d) + 256);
    ctx->h_rec = static_cast<DevFeatures*>(h);
    ctx->h_err = reinterpret_cast<uint32_t*>(static_cast<char*>(h) + 256);
    ctx->h_hist = reinterpret_cast<unsigned long long*>(static_cast<char*>(h) + persist);
    if (ctx->cfg.model_path) {
        std::string why;
        if (!ctx->model.load(ctx->cfg.model_path, &why)) {
            ahs_destroy(ctx);
            return AHS_ERR_NOT_FOUND;
        }
    }
    *out = ctx;
    return AHS_OK;
}

ahs_status ahs_serve_stop(ahs_ctx* ctx);

void ahs_destroy(ahs_ctx* ctx) {
    if (!ctx) return;
    if (ctx->device < 0) {
        delete ctx;
        return;
    }
    if (ctx->serve) ahs_serve_stop(ctx);
    cudaSetDevice(ctx->device);
    if (ctx->host_pipe) destroy_host_pipe(ctx->host_pipe);
    cudaDeviceSynchronize();
    for (auto& ev : ctx->ev)
        if (ev) cudaEventDestroy(ev);
    for (auto& r : ctx->tracer.records) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto& e : ctx->tracer.pool) cudaEventDestroy(e);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->aux) cudaFree(ctx->aux);
    if (ctx->side) cudaFree(ctx->side);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->h_coarse) cudaFreeHost(ctx->h_coarse);
    if (ctx->d_rec) cudaFree(ctx->d_rec);
    if (ctx->h_rec) cudaFreeHost(ctx->h_rec);
    delete ctx;
}

ahs_status ahs_trace_enable(ahs_ctx* ctx, int32_t on) {
    if (!ctx) return AHS_ERR_INVALID_ARG;
    ctx->tracer.on = on != 0;
    return AHS_OK;
}

ahs_status ahs_trace_collect(ahs_ctx* ctx, ahs_trace_entry_t* out, uint32_t cap, uint32_t* count) {
    if (!ctx || !count || (cap && !out)) return AHS_ERR_INVALID_ARG;
    cudaSetDevice(ctx->device);
    uint32_t k = 0;
    for (auto& r : ctx->tracer.records) {
        cudaError_t e = cudaEventSynchronize(r.b);
        if (e != cudaSuccess) return cuda_status(ctx, e);
        if (k < cap) {
            out[k].kernel = r.name;
            out[k].items = r.items;
            float ms = 0.f, start = 0.f;
            cudaEventElapsedTime(&ms, r.a, r.b);
            cudaEventElapsedTime(&start, ctx->tracer.records.front().a, r.a);
            out[k].ms = ms;
            out[k].start_ms = start;
        }
        ++k;
        ctx->tracer.pool.push_back(r.a);
        ctx->tracer.pool.push_back(r.b);
    }
    ctx->tracer.records.clear();
    *count = k;
    return AHS_OK;
}

const char* ahs_last_cuda_error(const ahs_ctx* ctx) {
    return ctx ? ctx->last_cuda_error.c_str() : "";
}

ahs_status ahs_load_tuning(ahs_ctx* ctx, const char* path) {
    if (!ctx) return AHS_ERR_INVALID_ARG;
    if (!path) {
        ctx->tuning.clear();
        return AHS_OK;
    }
    std::string why;
    return ctx->tuning.load(path, &why) ? AHS_OK : AHS_ERR_NOT_FOUND;
}

ahs_status ahs_tuned_radix_bits(const ahs_ctx* ctx, uint32_t key_bytes, int32_t has_payload,
                                uint64_t span, uint32_t* passes, uint32_t* digit_bits) {
    if (!ctx || !passes || !digit_bits || (key_bytes != 4 && key_bytes != 8))
        return AHS_ERR_INVALID_ARG;
    const RadixPlan p = radix_plan(span, radix_digit_bits(ctx, key_bytes, has_payload != 0, span));
    *passes = p.passes;
    *digit_bits = p.passes ? p.bits[0] : 0;
    return AHS_OK;
}

ahs_status ahs_load_model(ahs_ctx* ctx, const char* path) {
    if (!ctx || !path) return AHS_ERR_INVALID_ARG;
    std::string why;
    return ctx->model.load(path, &why) ? AHS_OK : AHS_ERR_NOT_FOUND;
}

static bool valid_type(ahs_key_type t) { return t >= AHS_U32 && t <= AHS_I64; }

ahs_status ahs_features(ahs_ctx* ctx, const void* d_keys, uint64_t n, ahs_key_type type,
                        void* stream, ahs_features_t* h_out) {
    if (!ctx || !h_out || ctx->device < 0) return AHS_ERR_INVALID_ARG;
    if (!valid_type(type)) return AHS_ERR_DTYPE;
    if (n && !d_keys) return AHS_ERR_INVALID_ARG;
    if (n == 0) {
        std::memset(h_out, 0, sizeof(*h_out));
        return AHS_OK;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    TracerGuard tg(&ctx->tracer);
    return run_features(ctx, d_keys, n, key_desc(type), static_cast<cudaStream_t>(stream), h_out);
}

ahs_status ahs_select_fsm(const ahs_features_t* f, const ahs_thresholds_t* t, ahs_strategy* out) {
    if (!f || !t || !out) return AHS_ERR_INVALID_ARG;
    *out = select_fsm(*f, *t);
    return AHS_OK;
}

ahs_status ahs_select(const ahs_ctx* ctx, const ahs_features_t* f, ahs_select_mode mode,
                      uint32_t key_bytes, int32_t has_payload, ahs_strategy* out) {
    if (!ctx || !f || !out) return AHS_ERR_INVALID_ARG;
    ahs_thresholds_t t;
    switch (mode) {
    case AHS_SEL_MODEL:
        *out = select_model(ctx->model, *f, key_bytes, has_payload);
        return AHS_OK;
    case AHS_SEL_CUSTOM:
        *out = select_fsm(*f, ctx->custom);
        return AHS_OK;
    case AHS_SEL_LEMMA32:
        profile_thresholds(AHS_SEL_LEMMA32, &t);
        *out = select_lemma32(*f, t);
        return AHS_OK;
    default:
        if (profile_thresholds(mode, &t) != AHS_OK) return AHS_ERR_INVALID_ARG;
        *out = select_fsm(*f, t);
        return AHS_OK;
    }
}

uint64_t ahs_small_capacity(ahs_key_type type, int32_t has_payload) {
    if (!valid_type(type)) return 0;
    return blocksort_capacity(key_desc(type).bytes, has_payload != 0);
}

ahs_status ahs_sort(ahs_ctx* ctx, const void* d_keys_in, void* d_keys_out,
                    const uint32_t* d_vals_in, uint32_t* d_vals_out, uint64_t n,
                    ahs_key_type type, ahs_strategy force, void* stream, ahs_sort_info_t* info) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!ctx || ctx->device < 0) return AHS_ERR_INVALID_ARG;
    if (!valid_type(type)) return AHS_ERR_DTYPE;
    if (force < AHS_AUTO || force > AHS_GENERAL) return AHS_ERR_INVALID_ARG;
    if (n && (!d_keys_in || !d_keys_out)) return AHS_ERR_INVALID_ARG;
    if (n && d_vals_in && !d_vals_out) return AHS_ERR_INVALID_ARG;
    if (n == 0) {
        if (info) info->strategy = AHS_IDENTITY;
        return AHS_OK;
    }
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const KeyDesc kd = key_desc(type);
    const bool timing = ctx->cfg.timing != 0;
    TracerGuard tg(&ctx->tracer);

    if (timing) cudaEventRecord(ctx->ev[0], st);
    ahs_features_t f;
    // A profile that returns presorted inputs by a copy (in order as they
    // are, in reverse order reversed) needs no histogram for one: the feature
    // pass skips it when K1 finds no descent, or no ascent (strictly
    // decreasing keys with a payload).
    const bool presorted = force == AHS_AUTO && sorted_identity(ctx);
    const uint32_t skip = presorted ? (kSkipOrdered | (d_vals_in ? kSkipStrictReversed : kSkipReversed)) : 0u;
    ahs_status rc = run_features(ctx, d_keys_in, n, kd, st, &f, skip);
    if (rc != AHS_OK) return rc;
    if (timing) cudaEventRecord(ctx->ev[1], st);

    const ahs_strategy s =
        force == AHS_AUTO ? choose(ctx, f, kd.bytes, d_vals_in != nullptr, presorted) : force;
    uint32_t passes = 0, buckets = 0;
    rc = run_strategy(ctx, s, d_keys_in, d_keys_out, d_vals_in, d_vals_out, n, kd, f, st, &passes,
                      &buckets);
    if (rc != AHS_OK) return rc;
    if (timing) cudaEventRecord(ctx->ev[2], st);
    rc = check_device_error(ctx, st);
    if (info) {
        info->strategy = s;
        info->features_valid = 1;
        info->features = f;
        info->passes = passes;
        info->buckets = buckets;
        info->workspace_bytes = ctx->ws_bytes;
        if (timing) {
            cudaEventElapsedTime(&info->ms_features, ctx->ev[0], ctx->ev[1]);
            cudaEventElapsedTime(&info->ms_sort, ctx->ev[1], ctx->ev[2]);
        }
    }
    return rc;
}

}  // extern "C"
