// The library context (opaque to callers as ahs_ctx).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "internal.h"
#include "select.h"
#include "trace.h"
#include "tuning.h"

namespace ahs {
struct ServeState;   // serve.cpp
struct HostPipe;     // host_sort.cu
void destroy_host_pipe(HostPipe* p);
}

struct ahs_ctx {
    int device = 0;
    int sms = 152;   // replaced by the device's SM count at creation
    ahs_config_t cfg{};
    ahs_thresholds_t custom{};

    // Persistent device block: feature record + error word (zeroed at create).
    ahs::DevFeatures* d_rec = nullptr;
    uint32_t* d_err = nullptr;
    // Pinned host mirror of the persistent block, and of the feature histogram.
    ahs::DevFeatures* h_rec = nullptr;
    uint32_t* h_err = nullptr;
    unsigned long long* h_hist = nullptr;   // kMaxBins counts

    // Growable device workspace.
    void* ws = nullptr;
    size_t ws_bytes = 0;
    // Growable auxiliary device buffer (work lists) and pinned host staging.
    void* aux = nullptr;
    size_t aux_bytes = 0;
    void* h_stage = nullptr;
    size_t h_stage_bytes = 0;
    // Growable side buffer of the exact-entropy mode (its sorted copy).
    void* side = nullptr;
    size_t side_bytes = 0;
    // Growable pinned host buffer of the batched form's coarse histograms.
    void* h_coarse = nullptr;
    size_t h_coarse_bytes = 0;

    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    std::string last_cuda_error;
    ahs::TreeModel model;
    ahs::Tuning tuning;
    ahs::Tracer tracer;

    ahs::ServeState* serve = nullptr;   // owned; released by ahs_serve_stop
    ahs::HostPipe* host_pipe = nullptr; // ahs_sort_host's streams and buffers (owned)
};

namespace ahs {

// Grow the workspace to at least `bytes` (synchronises the device when it
// reallocates).  Returns AHS_ERR_OOM beyond cfg.workspace_limit or on failure.
ahs_status ensure_workspace(ahs_ctx* ctx, size_t bytes);
ahs_status cuda_status(ahs_ctx* ctx, cudaError_t e);
// Features into ctx->h_rec (synchronises the stream); scratch at ctx->ws.
// skip_sorted (kSkip* flags): an input found presorted gets no histogram
// (entropy NaN); for callers that then return it by a copy.
ahs_status run_features(ahs_ctx* ctx, const void* d_keys, uint64_t n, KeyDesc kd,
                        cudaStream_t st, ahs_features_t* out, uint32_t skip_sorted = 0);
void to_public(const DevFeatures& r, KeyDesc kd, ahs_features_t* out);
// Reversed input: no ascents, at least one descent; with a payload strictly
// decreasing (then reversing it is the stable sort).
bool reversed_input(const ahs_features_t& f, bool payload);
// The AUTO pick under the context's profile.  allow_reverse (single-array
// sorts under a profile that returns presorted inputs by a copy): a reversed
// input is returned reversed (AHS_REVERSE) before the profile's rules.
ahs_strategy choose(const ahs_ctx* ctx, const ahs_features_t& f, uint32_t key_bytes, bool payload,
                    bool allow_reverse = false);
// Whether AUTO under the context's profile returns an input in order as it is.
bool sorted_identity(const ahs_ctx* ctx);
// Run one strategy on device-resident inputs whose features are in ctx->d_rec
// and whose feature scratch (histogram) is at the start of ctx->ws.
ahs_status run_strategy(ahs_ctx* ctx, ahs_strategy s, const void* kin, void* kout,
                        const uint32_t* vin, uint32_t* vout, uint64_t n, KeyDesc kd,
                        const ahs_features_t& f, cudaStream_t st, uint32_t* passes,
                        uint32_t* buckets);
size_t features_region(int sms);
// Largest digit width of the stable LSD passes for this key range (tuned).
uint32_t radix_digit_bits(const ahs_ctx* ctx, uint32_t key_bytes, bool payload, uint64_t span);
ahs_status check_device_error(ahs_ctx* ctx, cudaStream_t st);
// Grow the auxiliary device buffer / pinned host staging (may synchronise).
ahs_status ensure_aux(ahs_ctx* ctx, size_t bytes);
ahs_status ensure_stage(ahs_ctx* ctx, size_t bytes);
// The host copy of the feature histogram (pinned, owned by the context).
struct HistView {
    const unsigned long long* counts = nullptr;
    uint32_t nbins = 0;
    size_t size() const { return nbins; }
    bool empty() const { return nbins == 0; }
    unsigned long long operator[](size_t i) const { return counts[i]; }
};

// General path: stable sample sort with shared-memory bucket sorts.  scratch is
// samplesort_scratch_bytes() of workspace.  Synchronises `st` once per level.
// Keys only, with `hist` (the host copy of the feature histogram, bins of
// (ord(x) - min_ord) >> shift): the first two levels take their splitters from
// the histogram's bin boundaries (exact bucket sizes, no counting pass).
// group: group_slots() of the input, the levels whose partition passes take
// warp-aggregated slots.
ahs_status run_samplesort(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                          uint32_t* vout, uint64_t n, KeyDesc kd, void* scratch, cudaStream_t st,
                          uint32_t* levels_out, uint32_t* buckets_out,
                          const HistView* hist = nullptr,
                          uint64_t min_ord = 0, uint32_t shift = 0, uint32_t group = 0);

// Keys-only radix sort, most significant digit first: partition passes by the
// feature histogram's bin -- level 1 by the bin's high byte, or by runs of
// consecutive bins of about n / 256 keys when the blocks of 256 bins are
// unbalanced (a heavy bin is then a bucket after one pass), level 2 by the
// single bin -- with exact bucket sizes from `hist` (the host copy of the
// histogram, bin = (ord(x) - min_ord) >> shift), then per-bin shared-memory
// sorts.  scratch: samplesort_scratch_bytes().
ahs_status run_msd_radix(ahs_ctx* ctx, const void* kin, void* kout, uint64_t n, KeyDesc kd,
                         uint64_t min_ord, const HistView& hist,
                         uint32_t shift, uint32_t group, void* scratch, cudaStream_t st,
                         uint32_t* levels_out, uint32_t* buckets_out);

// Keys-only radix sort of an input with few distinct values: the values are
// counted in hash tables (one read of the keys), ranked, and the output is
// filled run by run.  Tried when the histogram has at most kSparseMaxBins
// non-empty bins (a lower bound on the distinct values) and n is at least
// kSparseMinKeys; *done is false when the tables overflowed (more distinct
// values than they hold), and the output is then untouched.  Synchronises
// `st` once.
constexpr uint64_t kSparseMinKeys = 1ull << 18;
constexpr uint32_t kSparseMaxBins = 2048;
bool sparse_radix_fits(uint64_t n, uint32_t key_bytes, uint64_t span, const HistView& hist);
ahs_status run_sparse_radix(ahs_ctx* ctx, const void* kin, void* kout, uint64_t n, KeyDesc kd,
                            uint64_t min_ord, cudaStream_t st, bool* done, uint32_t* distinct);

// Which partition levels aggregate the slot atomics of lanes that share a
// bucket (measured on GB300: it pays where the lanes of a warp row often
// share buckets without the whole row doing so, and costs up to 2.5x where
// they rarely do).  The feature record gives level 1 for inputs of runs
// broken by displaced keys (few descents; wholly ordered rows take the plain
// path's one-atomic case).  The histogram adds a level when two random keys
// of one bucket of the level before fall in the same bucket with probability
// kGroupCollide or more (frequent keys).
// kRunsLikely: neighbouring keys tend to share a bucket (few descents, or
// few ascents: reversed runs), so the levels without aggregation check warp
// rows for one shared bucket; without it (keys in random order: about n / 2
// descents) those checks are skipped.
constexpr uint32_t kGroupLevel1 = 1;
constexpr uint32_t kRunsLikely = 2;
constexpr double kGroupCollide = 0.25;
inline bool runs_likely(unsigned long long descents, unsigned long long n) {
    return descents < n / 4 || descents > n - n / 4;
}
inline uint32_t group_slots(const ahs_features_t& f) {
    return (f.descents < f.n / 4 ? kGroupLevel1 : 0u) | (runs_likely(f.descents, f.n) ? kRunsLikely : 0u);
}

}  // namespace ahs
