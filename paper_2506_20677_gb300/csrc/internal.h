// Internal (non-ABI) declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ahs.h"

namespace ahs {

// Device-resident feature record, written by the feature kernels and copied to
// the host in one piece.  Self-resetting block counters live here too.
constexpr uint32_t kSkipOrdered = 1, kSkipReversed = 2, kSkipStrictReversed = 4;

struct DevFeatures {
    unsigned long long min_ord;   // order-preserving image of the smallest key
    unsigned long long max_ord;
    unsigned long long descents;
    unsigned long long ascents;
    unsigned long long n;
    unsigned long long span;
    uint32_t shift;
    uint32_t nbins;
    double entropy;
    double entropy_norm;
    uint32_t k1_done;             // last-block counters (return to 0 after each use)
    uint32_t k3_done;
    uint32_t rh_done;             // radix digit-histogram kernel
    uint32_t k2_wrapped;          // a packed K2 counter wrapped: rerun K2 in the split layout
    unsigned long long pad[5];
};
static_assert(sizeof(DevFeatures) == 128, "DevFeatures layout");

constexpr uint32_t kMaxBins = 1u << 16;             // histogram bins, Section III-A reading
constexpr uint32_t kHistSmemBytes = 21846u * 8u;    // shared memory of the histogram kernel
constexpr uint32_t kHistThreads = 1024;
constexpr uint32_t kEntropyBlocks = kMaxBins / 256;

// Key type descriptors.
struct KeyDesc {
    uint32_t bytes;      // 4 or 8
    uint64_t flip;       // sign bit for signed types
};
inline KeyDesc key_desc(ahs_key_type t) {
    switch (t) {
    case AHS_U32: return {4, 0};
    case AHS_I32: return {4, 0x80000000ull};
    case AHS_U64: return {8, 0};
    default: return {8, 0x8000000000000000ull};
    }
}

// ------------------------------------------------------------------ features
struct FeatureScratch {
    DevFeatures* rec;                 // persistent, zero-initialised
    unsigned long long* k1_partials;  // 3 per K1 block
    uint32_t* slabs;                  // hist_blocks x kMaxBins
    unsigned long long* hist;         // kMaxBins exact counts (u64)
    double* ent_partials;             // kEntropyBlocks
    // Optional pinned host mirrors that K3 fills (null: device copies only).
    DevFeatures* host_rec = nullptr;
    unsigned long long* host_hist = nullptr;   // nbins counts
    // K2 and K3 skip an input K1 found presorted (no histogram; entropy NaN):
    // kSkipOrdered: no descents; kSkipReversed: no ascents (keys only);
    // kSkipStrictReversed: strictly decreasing (with a payload).
    uint32_t skip_sorted = 0;
};
uint32_t k1_blocks(uint64_t n, int sms);
size_t features_scratch_bytes(int sms);
cudaError_t launch_features(const void* keys, uint64_t n, KeyDesc kd, const FeatureScratch& s,
                            int sms, cudaStream_t st);
// After launch_features, when the record says a packed histogram counter
// wrapped (DevFeatures::k2_wrapped): K2 again in the exact split layout, then
// K3.  The record's K1 results stay.
cudaError_t launch_features_split_retry(const void* keys, uint64_t n, KeyDesc kd,
                                        const FeatureScratch& s, int sms, cudaStream_t st);

// ------------------------------------------------------------------ counting
// Keys-only counting sort (Listing 2) from the exact histogram of the feature
// pass (requires hist_shift == 0).  prefix: kMaxBins + 1 u64 of scratch.
cudaError_t launch_counting_fill(void* out, uint64_t n, KeyDesc kd, const DevFeatures* rec,
                                 const unsigned long long* hist, unsigned long long* prefix,
                                 uint64_t min_ord, uint32_t nbins, int sms, cudaStream_t st);

// The same fill over a sparse set of values: run j (j < status[1]) holds
// the value min + vals[j] at positions [prefix[j], prefix[j + 1]); nothing is
// written when status[0] != 0.  The run count and flag are read on the
// device, so the launch can be queued behind the kernels that produce them.
cudaError_t launch_sparse_fill(void* out, uint64_t n, KeyDesc kd, const unsigned long long* prefix,
                               const void* vals, const uint32_t* status, uint64_t min_ord, int sms,
                               cudaStream_t st);

// dst[n - 1 - i] = src[i] for elements of 4 or 8 bytes; dst == src allowed.
cudaError_t launch_reverse(void* dst, const void* src, uint64_t n, uint32_t elem_bytes, int sms,
                           cudaStream_t st);

// Copy `words` 32-bit words (keys or payload) from src to dst.
cudaError_t launch_copy32(void* dst, const void* src, uint64_t words, int sms, cudaStream_t st);
// Many copies of 32-bit words in one launch.  `items` must be readable by the
// device (device memory, or pinned host memory, which the kernel reads in
// place) until the launch completes; items of up to kCopyItemWords words
// keep the CTAs balanced.
struct CopyItem {
    void* dst;
    const void* src;
    uint64_t words;
};
constexpr uint64_t kCopyItemWords = 1ull << 16;
cudaError_t launch_copy_list(const CopyItem* items, uint32_t count, uint64_t words, int sms,
                             cudaStream_t st);
// Zero `words` 32-bit words.
cudaError_t launch_zero32(void* dst, uint64_t words, int sms, cudaStream_t st);
// Move `bytes` between pinned host memory (mapped into the device's address
// space) and device memory with a kernel, not a copy engine: a sort's small
// uploads and read-backs then never queue behind bulk copies the caller runs
// on the copy engines at the same time.
cudaError_t launch_transfer(void* dst, const void* src, size_t bytes, cudaStream_t st);

// --------------------------------------------------------------------- radix
constexpr uint32_t kMaxRadixPasses = 8;
struct RadixPlan {
    uint32_t passes;
    uint32_t radix;                       // digit alphabet of every pass: 16, 256, 512, 1024 or 2048
    uint32_t shift[kMaxRadixPasses];      // low bit of each pass's digit
    uint32_t bits[kMaxRadixPasses];       // digit width of each pass (<= log2 radix)
};
// Passes and digit widths for digits of at most max_bits bits (1..11).
RadixPlan radix_plan(uint64_t span, uint32_t max_bits = 8);
size_t radix_scratch_bytes(uint64_t n, uint32_t key_bytes, bool has_vals, const RadixPlan& plan);
struct RadixScratch {
    void* keys_tmp;                   // n keys
    uint32_t* vals_tmp;               // n payload words (or null)
    unsigned long long* digit_hist;   // kMaxRadixPasses x 2048 (u64), then the digit bases (u32)
    uint32_t* status;                 // passes x tiles x radix look-back words
    uint32_t* tile_counters;          // kMaxRadixPasses
    uint64_t tiles;
};
RadixScratch radix_carve(void* base, uint64_t n, uint32_t key_bytes, bool has_vals,
                         const RadixPlan& plan);
// Stable LSD radix sort over ord(x) - min (onesweep passes with decoupled look-back).
// stall_tile: a tile that withholds its look-back publication (test hook), or ~0u.
cudaError_t launch_radix_sort(const void* keys_in, void* keys_out, const uint32_t* vals_in,
                              uint32_t* vals_out, uint64_t n, KeyDesc kd, uint64_t min_ord,
                              const RadixPlan& plan, const RadixScratch& rs, DevFeatures* rec,
                              uint32_t* err, int sms, cudaStream_t st, uint32_t stall_tile = ~0u);

// ------------------------------------------------------- one-block sort (SMALL)
uint64_t blocksort_capacity(uint32_t key_bytes, bool has_vals);
cudaError_t launch_blocksort_single(const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                    uint32_t* vals_out, uint64_t n, KeyDesc kd, cudaStream_t st);

// ------------------------------------------------------ general: sample sort
size_t samplesort_scratch_bytes(uint64_t n, uint32_t key_bytes, bool has_vals);

}  // namespace ahs
