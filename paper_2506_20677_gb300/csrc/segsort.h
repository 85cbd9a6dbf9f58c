// Segmented partition machinery shared by the single-array general path and
// the batched forms: stable multi-way partitions of many segments at once,
// by sample splitters (sample sort) or by an 8-bit digit of key - segment min
// (segmented LSD radix), and the shared-memory sort of small segments.
#pragma once

#include <vector>

#include "ctx.h"
#include "samplesort.h"

namespace ahs {

// A segment of the key buffer: keys [begin, begin + size) relative to the
// base pointers the caller passes; min_ord (digit mode) is the order-
// preserving image of the segment's smallest key.
struct SegRange {
    unsigned long long begin;
    uint32_t size;
    unsigned long long min_ord;
};

// Device scratch for total keys n_total in at most nseg initial segments.
size_t segsort_scratch_bytes(uint64_t n_total, uint64_t nseg, uint32_t key_bytes, bool vals);

// Sample sort of every segment in `segs` (each sorted on its own), keys
// read from kin and written to kout at the same positions; `extra` are
// segments already known to fit one CTA, sorted from kin in the same final
// launch.  Synchronises `st` once per partition level.
ahs_status run_segmented_general(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                                 uint32_t* vout, uint64_t n_total, const std::vector<SegRange>& segs,
                                 const std::vector<SegRange>& extra, KeyDesc kd, void* scratch,
                                 cudaStream_t st, uint32_t* levels_out, uint32_t* buckets_out);

// A keys-only segment whose 256-bucket coarse histogram (counts of the
// feature histogram's bin >> 8, bins of (ord(x) - min_ord) >> shift) is known.
struct HistRange {
    SegRange r;
    uint32_t shift;              // the segment's histogram shift
    bool group;                  // few descents: slot atomics aggregated per warp
    bool runs;                   // few descents or few ascents: warp rows checked for one bucket
    const uint32_t* coarse;      // 256 counts (host memory)
};

// Keys only: one partition pass of every segment by the high byte of its
// histogram bin, kin -> kout, with bucket offsets from the coarse histograms
// (planned on the host before the launch, no counting pass), then the
// shared-memory sorts of the buckets in place; buckets larger than a CTA
// (heavy bins) are sorted in place by the sampled levels.  `extra` are
// segments of at most one CTA's keys, sorted from kin in the same launches.
ahs_status run_batched_general_hist(ahs_ctx* ctx, const void* kin, void* kout, uint64_t n_total,
                                    const std::vector<HistRange>& segs,
                                    const std::vector<SegRange>& extra, KeyDesc kd, void* scratch,
                                    cudaStream_t st, uint32_t* levels_out, uint32_t* buckets_out);

// Stable LSD radix of every segment (digits of key - segment min, 8 bits a
// pass, `passes` passes), kin -> kout, no host synchronisation.
ahs_status run_segmented_radix(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                               uint32_t* vout, uint64_t n_total, const std::vector<SegRange>& segs,
                               uint32_t passes, KeyDesc kd, void* scratch, cudaStream_t st);

// Sort small segments (each <= kBucketCap keys) and copy already-ordered
// segments (any size) from kin into kout with one CTA each, one launch per
// size class.  Synchronises `st`.
ahs_status run_small_segments(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                              uint32_t* vout, const std::vector<SegRange>& sort_segs,
                              const std::vector<SegRange>& copy_segs, KeyDesc kd, cudaStream_t st);

}  // namespace ahs
