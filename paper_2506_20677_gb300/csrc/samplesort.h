// Types shared by the general path (sample sort) and the bucket sorts.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace ahs {

// Largest bucket one CTA sorts in shared memory, and the size classes of the
// bucket kernels (threads x keys: 128x8, 256x8, 192x16, 256x16, 256x18,
// 384x16, 512x16).  Classes at most 1.5x apart keep a bucket's CTA at least
// two thirds full; the 4,608 class catches histogram bins of just over
// 4,096 keys (2^28 keys in 2^16 bins).
constexpr uint32_t kBucketCap = 8192;
// Coarse histogram of a segment: counts of the feature histogram's bin >> 8.
constexpr uint32_t kCoarseBuckets = 256;
constexpr int kBucketClasses = 7;
constexpr uint32_t kBucketClassCap[kBucketClasses] = {1024, 2048, 3072, 4096, 4608, 6144, 8192};

// A bucket that leaves the partition levels: its keys sit in buffer `where`
// (0: temporary, 1: the output, 2: the input) at [begin, begin + size).  When
// the partition fixed the bucket's range (bits != kBoundsUnknown), every key
// has lo <= ord(x) < lo + 2^bits and the sort digits start from lo.
constexpr uint8_t kBoundsUnknown = 0xff;
struct FinalBucket {
    unsigned long long begin;
    unsigned long long lo;
    uint32_t size;
    uint8_t where;
    uint8_t sort;      // 0: all keys equal (or one key), copy only
    uint8_t bits;
    uint8_t pad;
};
static_assert(sizeof(FinalBucket) == 24, "FinalBucket layout");

inline FinalBucket final_bucket(unsigned long long begin, uint32_t size, uint8_t where, bool sort) {
    return FinalBucket{begin, 0ull, size, where, (uint8_t)sort, kBoundsUnknown, 0};
}
inline FinalBucket final_bucket_bounded(unsigned long long begin, uint32_t size, uint8_t where,
                                        unsigned long long lo, uint32_t bits) {
    return FinalBucket{begin, lo, size, where, 1, (uint8_t)bits, 0};
}

// Class caps are multiples of 512 keys: the class of a size is a lookup on
// (size - 1) / 512 (sizes past the last cap take the last class).
struct BucketClassTable {
    uint8_t c[kBucketCap / 512];
    constexpr BucketClassTable() : c{} {
        for (uint32_t i = 0; i < kBucketCap / 512; ++i) {
            uint8_t k = kBucketClasses - 1;
            for (int j = kBucketClasses - 1; j >= 0; --j)
                if ((i + 1) * 512 <= kBucketClassCap[j]) k = (uint8_t)j;
            c[i] = k;
        }
    }
};
static_assert([] {
    for (uint32_t cap : kBucketClassCap)
        if (cap % 512) return false;
    return true;
}(), "bucket class caps are multiples of 512");
inline uint32_t bucket_class(uint32_t size) {
    static constexpr BucketClassTable t{};
    const uint32_t i = size ? (size - 1) / 512 : 0;
    return i < kBucketCap / 512 ? t.c[i] : kBucketClasses - 1;
}
cudaError_t launch_bucket_finish(const FinalBucket* d_lists[kBucketClasses],
                                 const uint32_t counts[kBucketClasses],
                                 const uint64_t keys[kBucketClasses], const void* buf0, const void* buf1,
                                 const void* buf2, void* out, const uint32_t* vbuf0,
                                 const uint32_t* vbuf1, const uint32_t* vbuf2, uint32_t* vout,
                                 KeyDesc kd, cudaStream_t st);

}  // namespace ahs
