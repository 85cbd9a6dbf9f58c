// General path: splitter-based sample sort with shared-memory bucket sorts.
//
// The paper's general case is quicksort with a median-of-three pivot
// (Listing 4): partition around a pivot into (<, =, >) and recurse.  Here each
// level partitions every open segment around up to 255 splitters at once,
// chosen as quantiles of a sorted random sample of 8,192 keys (the median-of-
// three generalised to many pivots; Leischner, Osipov & Sanders 2010 for the
// GPU sample-sort scheme).  Keys equal to a splitter form their own
// "equality" bucket, the analogue of the (= pivot) part of a three-way
// partition, so duplicate-heavy segments always shrink.  A partition level is
//   sample -> count (per tile, per bucket) -> segmented column scan -> stable scatter
// and a bucket that fits one CTA (<= 8,192 keys) is sorted in shared memory.
// Every step is stable, so a payload comes out in the unique stable order.
//
// The same partition kernels, with the bucket of a key taken as an 8-bit digit
// of (key - segment min) instead of its splitter interval, give a segmented
// LSD radix sort for the batched form (many arrays sorted in one launch per
// pass).
#include <algorithm>
#include <cstring>
#include <vector>

#include "blocksort.cuh"
#include "common.cuh"
#include "ctx.h"
#include "hostpar.h"
#include "internal.h"
#include "rank.cuh"
#include "samplesort.h"
#include "segsort.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kThreads = 512;
constexpr int kIpt = 16;
constexpr uint32_t kTile = kThreads * kIpt;     // keys per partition tile
constexpr uint32_t kMaxSplit = 255;             // distinct splitters per segment
constexpr uint32_t kSlots = 256;                // per segment: tree[1..255] then sorted[0..255]
constexpr uint32_t kCols = 512;                 // 2 * 255 + 1 buckets, padded
constexpr uint32_t kOversample = 32;
constexpr uint32_t kSamples = (kMaxSplit + 1) * kOversample;   // 8,192
constexpr uint32_t kChunkTiles = 32;
constexpr uint32_t kMaxLevels = 16;
constexpr uint32_t kCopyChunk = 4096;           // keys one CTA copies of an unsorted bucket
constexpr int kSplit = 0;                       // bucket = splitter interval / equality
constexpr int kDigit = 1;                       // bucket = 8-bit digit of key - segment min
constexpr int kTable = 3;                       // bucket = table[(key - min) >> shift] (histogram bin)
constexpr int kHistCopies = 4;
static_assert(kThreads % 32 == 0 && kThreads >= 32, "whole warps");
static_assert((uint32_t)kThreads * kIpt >= kSamples, "one CTA must hold the whole splitter sample");
static_assert(kCols % kThreads == 0 || kThreads % kCols == 0, "bucket columns divide the block");
static_assert(kCols < 1024 && kThreads * kIpt <= (1u << 22), "scatter packs (slot << 10) | bucket");

struct SegDesc {
    unsigned long long begin;
    uint32_t size;
    uint32_t first_chunk;
    uint32_t nchunks;
    uint32_t first_tile;   // index of the segment's first tile in the pass's tile order
    unsigned long long min_ord;
    uint32_t dshift;       // digit passes: 0 = the pass's shift, else this segment's shift + 1
    uint32_t pad;
};
struct TileDesc {
    unsigned long long begin;
    uint32_t size;
    uint32_t seg;
};
struct ChunkDesc {
    uint32_t first_tile;
    uint32_t ntiles;
    uint32_t seg;
    uint32_t pad;
};
static_assert(sizeof(SegDesc) == 40 && sizeof(TileDesc) == 16 && sizeof(ChunkDesc) == 16, "layout");

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // SplitMix64 output function (Steele, Lea & Flood 2014).
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Splitter bucket of ord value o: descend the implicit binary tree of the 255
// (padded) splitters without branches -- after 8 levels j - 256 is the number
// of splitters below o -- then test equality with that splitter.
// 2j for sorted[j-1] < o < sorted[j], 2j+1 for o == sorted[j].
template <typename K>
__device__ __forceinline__ uint32_t classify_split(const K* tree, const K* sorted, uint32_t m, K o) {
    uint32_t j = 1;
#pragma unroll
    for (int l = 0; l < 8; ++l) j = 2 * j + (o > tree[j] ? 1u : 0u);
    const uint32_t idx = j - 256;
    return (idx < m && sorted[idx] == o) ? 2 * idx + 1 : 2 * idx;
}

template <typename K, int MODE>
struct Classifier {
    const K* tree;
    const K* sorted;
    uint32_t m;
    K mn;
    uint32_t shift;
    const uint8_t* table;   // kTable: bucket of each histogram bin
    __device__ __forceinline__ uint32_t operator()(K o) const {
        if constexpr (MODE == kSplit) {
            return classify_split(tree, sorted, m, o);
        } else if constexpr (MODE == kTable) {
            // m = the table's size: a key outside the histogram's range (an
            // input changed since its features were taken) reads no further.
            const K bin = (K)(o - mn) >> shift;
            return __ldg(table + (bin < (K)m ? (uint32_t)bin : m - 1));
        } else {
            return (uint32_t)((K)(o - mn) >> shift) & 0xffu;
        }
    }
};

// Splitters a segment of `size` keys takes: enough for buckets of about half
// a CTA's capacity, at most 255 (the tree's size).
__host__ __device__ __forceinline__ uint32_t split_count(uint64_t size) {
    const uint64_t want = (size + kBucketCap / 2 - 1) / (kBucketCap / 2);
    return (uint32_t)(want <= 2 ? 1 : (want - 1 > kMaxSplit ? kMaxSplit : want - 1));
}

// One CTA per segment: draw 32 keys per wanted splitter at hashed positions,
// sort them in shared memory, keep the distinct values among the quantiles,
// pad with the largest value and lay them out as an implicit search tree.
template <typename K>
__global__ void __launch_bounds__(kThreads)
ss_sample(const K* __restrict__ src, const SegDesc* __restrict__ segs, uint32_t level, K flip,
          K* __restrict__ splitters, uint32_t* __restrict__ nsplit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = BlockSortSmem<K, false, kThreads, kIpt>;
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    __shared__ K s_sorted[kSlots];
    const SegDesc sg = segs[blockIdx.x];
    const unsigned long long salt =
        ((unsigned long long)level << 48) ^ ((unsigned long long)blockIdx.x << 20);
    const uint32_t m = split_count(sg.size);
    const uint32_t nsamp = (m + 1) * kOversample;
    for (uint32_t i = threadIdx.x; i < nsamp; i += kThreads) {
        const unsigned long long h = mix64((salt + i + 1) * 0x9E3779B97F4A7C15ull);
        const unsigned long long pos = __umul64hi(h, (unsigned long long)sg.size);
        S.keys[i] = src[sg.begin + pos];
    }
    __syncthreads();
    block_sort<K, false, kThreads, kIpt>(S.keys, S.keys, nullptr, nullptr, nsamp, flip, S);
    __syncthreads();
    uint32_t keep = 0;
    K cand = 0;
    if (threadIdx.x < m) {
        cand = S.keys[(threadIdx.x + 1) * kOversample - 1] ^ flip;
        keep = (threadIdx.x == 0 || cand != (K)(S.keys[threadIdx.x * kOversample - 1] ^ flip)) ? 1u : 0u;
    }
    uint32_t total;
    const uint32_t at = block_exclusive_scan<kThreads>(keep, S.scan, &total);
    if (keep) s_sorted[at] = cand;
    __syncthreads();
    for (uint32_t i = total + threadIdx.x; i < kSlots; i += kThreads) s_sorted[i] = ~K(0);
    __syncthreads();
    K* out = splitters + (size_t)blockIdx.x * 2 * kSlots;
    if (threadIdx.x < kSlots) {
        const uint32_t j = threadIdx.x;
        out[kSlots + j] = s_sorted[j];
        if (j >= 1) {
            const uint32_t d = 31 - __clz(j);              // depth of node j
            const uint32_t p = j - (1u << d);              // position within its level
            out[j] = s_sorted[((2 * p + 1) << (7 - d)) - 1];
        } else {
            out[0] = 0;
        }
    }
    if (threadIdx.x == 0) nsplit[blockIdx.x] = total;
}

// Per tile: bucket histogram (4 copies spread the atomics of skewed inputs),
// written as one row of the tiles x buckets matrix, or (TOTALS) added into the
// segment's bucket totals.
template <typename K, int MODE, bool TOTALS>
__global__ void __launch_bounds__(kThreads)
ss_count(const K* __restrict__ src, const TileDesc* __restrict__ tiles,
         const SegDesc* __restrict__ segs, const K* __restrict__ splitters,
         const uint32_t* __restrict__ nsplit, K flip, uint32_t shift, uint32_t* __restrict__ counts) {
    __shared__ K s_sp[2 * kSlots];
    __shared__ uint32_t hist[kHistCopies][kCols];
    const TileDesc t = tiles[blockIdx.x];
    Classifier<K, MODE> cls{};
    if constexpr (MODE == kSplit) {
        const K* g = splitters + (size_t)t.seg * 2 * kSlots;
        for (uint32_t i = threadIdx.x; i < 2 * kSlots; i += kThreads) s_sp[i] = g[i];
        cls.tree = s_sp;
        cls.sorted = s_sp + kSlots;
        cls.m = nsplit[t.seg];
    } else {
        cls.mn = (K)segs[t.seg].min_ord;
        cls.shift = shift;
    }
    for (uint32_t i = threadIdx.x; i < kHistCopies * kCols; i += kThreads) (&hist[0][0])[i] = 0;
    __syncthreads();
    uint32_t* mine = hist[(threadIdx.x >> 5) % kHistCopies];
    const K* p = src + t.begin;
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < t.size; i += kThreads) {
        const uint32_t b = cls((K)(p[i] ^ flip));
        if (AHS_DCHECK(b < kCols, "count bucket", b)) atomicAdd(&mine[b], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kCols; i += kThreads) {
        const uint32_t c = hist[0][i] + hist[1][i] + hist[2][i] + hist[3][i];
        if constexpr (TOTALS) {
            if (c) atomicAdd(&counts[(size_t)t.seg * kCols + i], c);
        } else {
            counts[(size_t)blockIdx.x * kCols + i] = c;
        }
    }
}

// Per segment: exclusive scan of the bucket totals; the bases seed the
// scatter's per-bucket cursors.
__global__ void __launch_bounds__(kCols)
ss_scan_totals(const uint32_t* __restrict__ seg_tot, uint32_t* __restrict__ seg_base,
               uint32_t* __restrict__ cursor) {
    __shared__ uint32_t scratch[kCols / 32 + 1];
    const size_t at = (size_t)blockIdx.x * kCols + threadIdx.x;
    uint32_t total;
    const uint32_t base = block_exclusive_scan<kCols>(seg_tot[at], scratch, &total);
    seg_base[at] = base;
    cursor[at] = base;
}

// Segmented column scan of the tiles x buckets count matrix, in three steps:
// (a) per chunk of <= 32 tiles, column sums; (b) per segment, exclusive scan of
// the chunk sums down each column and of the column totals across buckets;
// (c) per chunk, running sums down the tiles (counts become offsets relative
// to the segment's first key).
__global__ void __launch_bounds__(kCols)
ss_scan_a(const uint32_t* __restrict__ counts, const ChunkDesc* __restrict__ chunks,
          uint32_t* __restrict__ chunk_sum) {
    const ChunkDesc c = chunks[blockIdx.x];
    const uint32_t j = threadIdx.x;
    uint32_t s = 0;
    for (uint32_t t = 0; t < c.ntiles; ++t) s += counts[(size_t)(c.first_tile + t) * kCols + j];
    chunk_sum[(size_t)blockIdx.x * kCols + j] = s;
}

__global__ void __launch_bounds__(kCols)
ss_scan_b(uint32_t* __restrict__ chunk_sum, const SegDesc* __restrict__ segs,
          uint32_t* __restrict__ seg_tot, uint32_t* __restrict__ seg_base) {
    __shared__ uint32_t scratch[kCols / 32 + 1];
    const SegDesc sg = segs[blockIdx.x];
    const uint32_t j = threadIdx.x;
    uint32_t run = 0;
    for (uint32_t c = 0; c < sg.nchunks; ++c) {
        uint32_t* p = chunk_sum + (size_t)(sg.first_chunk + c) * kCols + j;
        const uint32_t v = *p;
        *p = run;
        run += v;
    }
    uint32_t total;
    const uint32_t base = block_exclusive_scan<kCols>(run, scratch, &total);
    if (seg_tot) {
        seg_tot[(size_t)blockIdx.x * kCols + j] = run;
        seg_base[(size_t)blockIdx.x * kCols + j] = base;
    }
    for (uint32_t c = 0; c < sg.nchunks; ++c) chunk_sum[(size_t)(sg.first_chunk + c) * kCols + j] += base;
}

__global__ void __launch_bounds__(kCols)
ss_scan_c(uint32_t* __restrict__ counts, const ChunkDesc* __restrict__ chunks,
          const uint32_t* __restrict__ chunk_sum) {
    const ChunkDesc c = chunks[blockIdx.x];
    const uint32_t j = threadIdx.x;
    uint32_t run = chunk_sum[(size_t)blockIdx.x * kCols + j];
    for (uint32_t t = 0; t < c.ntiles; ++t) {
        uint32_t* p = counts + (size_t)(c.first_tile + t) * kCols + j;
        const uint32_t v = *p;
        *p = run;
        run += v;
    }
}

template <typename K, bool VALS>
struct ScatterSmem {
    K sp[2 * kSlots];
    uint32_t warp_hist[kThreads / 32][kCols];
    uint32_t warp_mask[kRankScatter == kRankAtomicOr ? kThreads / 32 : 1][kCols];
    uint32_t tile_count[kCols];
    uint32_t tile_start[kCols];
    uint32_t gbase[kCols];
    uint32_t scan[kThreads / 32 + 1];
    uint16_t bid[kTile];
    K keys[kTile];
    uint32_t vals[VALS ? kTile : 1];
};

// Per tile: classify, rank stably by bucket, stage in bucket order, write
// each bucket's run to its offset.
template <typename K, bool VALS, int MODE>
__global__ void __launch_bounds__(kThreads)
ss_scatter(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
           uint32_t* __restrict__ vdst, const TileDesc* __restrict__ tiles,
           const SegDesc* __restrict__ segs, const K* __restrict__ splitters,
           const uint32_t* __restrict__ nsplit, K flip, uint32_t shift,
           const uint32_t* __restrict__ offs) {
    constexpr int W = kThreads / 32;
    constexpr int WARP_ITEMS = 32 * kIpt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<K, VALS>& S = *reinterpret_cast<ScatterSmem<K, VALS>*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const TileDesc t = tiles[blockIdx.x];
    const SegDesc sg = segs[t.seg];
    Classifier<K, MODE> cls{};
    if constexpr (MODE == kSplit) {
        const K* g = splitters + (size_t)t.seg * 2 * kSlots;
        for (uint32_t i = tid; i < 2 * kSlots; i += kThreads) S.sp[i] = g[i];
        cls.tree = S.sp;
        cls.sorted = S.sp + kSlots;
        cls.m = nsplit[t.seg];
    } else {
        cls.mn = (K)sg.min_ord;
        cls.shift = shift;
    }
    for (uint32_t i = tid; i < W * kCols; i += kThreads) (&S.warp_hist[0][0])[i] = 0;
    if constexpr (kRankScatter == kRankAtomicOr)
        for (uint32_t i = tid; i < W * kCols; i += kThreads) (&S.warp_mask[0][0])[i] = 0;
    __syncthreads();

    K key[kIpt];
    uint32_t b[kIpt];
    const K* p = src + t.begin;
    const uint32_t wbase = warp * WARP_ITEMS;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        const uint32_t q = wbase + 32 * i + lane;
        if (q < t.size) {
            key[i] = p[q];
            b[i] = cls((K)(key[i] ^ flip));
        } else {
            key[i] = 0;
            b[i] = kCols;
        }
    }
    uint32_t dr[kIpt];
    warp_rank<kIpt, kCols, kRankScatter>(b, dr, S.warp_hist[warp],
                                      S.warp_mask[kRankScatter == kRankAtomicOr ? warp : 0]);
    __syncthreads();
    for (uint32_t j = tid; j < kCols; j += kThreads) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t c = S.warp_hist[w][j];
            S.warp_hist[w][j] = run;
            run += c;
        }
        S.tile_count[j] = run;
    }
    __syncthreads();
    scan_digit_counts<kThreads, kCols>(S.tile_count, S.tile_start, S.scan);
    for (uint32_t j = tid; j < kCols; j += kThreads)
        S.gbase[j] = (uint32_t)(offs[(size_t)blockIdx.x * kCols + j]) - S.tile_start[j];
    __syncthreads();
    constexpr int SH = RankPack<kCols>::kShift;
    const uint32_t* vp = VALS ? vsrc + t.begin : nullptr;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        const uint32_t bk = dr[i] & RankPack<kCols>::kMask;
        if (bk < kCols) {
            const uint32_t lp = S.tile_start[bk] + S.warp_hist[warp][bk] + (dr[i] >> SH);
            if (!AHS_DCHECK(lp < t.size, "scatter stage", lp)) continue;
            S.keys[lp] = key[i];
            S.bid[lp] = (uint16_t)bk;
            if constexpr (VALS) S.vals[lp] = vp[wbase + 32 * i + lane];
        }
    }
    __syncthreads();
    K* out = dst + sg.begin;
    uint32_t* vout = VALS ? vdst + sg.begin : nullptr;
    for (uint32_t j = tid; j < t.size; j += kThreads) {
        const uint32_t gp = S.gbase[S.bid[j]] + j;
        if (gp >= sg.size) continue;   // cannot happen with consistent offsets; never write outside
        out[gp] = S.keys[j];
        if constexpr (VALS) vout[gp] = S.vals[j];
    }
}

// ------------------------------------------------------------ keys-only scatter
//
// Without a payload the order of equal-bucket keys inside a bucket is free (the
// bucket is sorted afterwards), so the scatter need not be stable.  Each CTA is
// persistent and walks the tile list with a stride of the grid; tile k+2G is
// fetched into shared memory by the bulk-async copy engine while tiles k and
// k+G are processed.  A key's slot in its tile's bucket run is one returning
// shared-memory atomic; the tile's run of each bucket is placed by one global
// atomic on the bucket's cursor (no cross-tile prefix is needed); the tile is
// staged in bucket order and written out in coalesced runs.
constexpr int kFastThreads = 512;
constexpr uint32_t kSegCache = 256;   // segments of a pass that derives its tiles
static_assert(kFastThreads == (int)kCols, "one bucket column per thread");
// Words per segment in the cursor array of a pass: 2 m + 1 <= kCols buckets
// with equality buckets, 256 for the digit and range classifiers.
template <int MODE>
constexpr uint32_t cursor_stride() { return MODE == kSplit ? kCols : 256u; }

template <typename K>
struct FastCfg {
    static constexpr int kIpt = sizeof(K) == 4 ? 16 : 8;
    static constexpr uint32_t kTileKeys = kFastThreads * kIpt;   // 32 KiB of keys
    static constexpr uint32_t kVec = 16 / sizeof(K);               // keys per 16 bytes
};

template <typename K>
struct FastSmem {
    static constexpr uint32_t TILE = FastCfg<K>::kTileKeys;
    K buf[2][TILE + FastCfg<K>::kVec];
    K sp[2][2 * kSlots];   // splitters of the tile in buf[s] (sample-sort levels)
    uint16_t bid[TILE];
    uint32_t hist[kCols];
    uint32_t tile_start[kCols];
    K* gptr[kCols];           // where the tile's run of each bucket goes, less its staged start
    uint32_t scan[kFastThreads / 32 + 1];
    SegDesc seg[kSegCache];   // the pass's segments, when it has no tile list
    TileDesc tile[2];         // the tile in buf[s]
    uint64_t bar[2];
};

static_assert(2 * (sizeof(FastSmem<uint32_t>) + 1024) <= 228 * 1024 &&
                  2 * (sizeof(FastSmem<uint64_t>) + 1024) <= 228 * 1024,
              "two partition CTAs per SM");

// Tile k of a pass without a tile list: segment q owns tiles
// [segs[q].first_tile, segs[q+1].first_tile), each of `tile_keys` keys but
// its last.
__device__ __forceinline__ TileDesc tile_of(const SegDesc* segs, uint32_t nsegs, uint32_t k,
                                            uint32_t tile_keys) {
    uint32_t lo = 0, hi = nsegs;   // last q with first_tile <= k
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (segs[mid].first_tile <= k) lo = mid;
        else hi = mid;
    }
    const uint32_t off = (k - segs[lo].first_tile) * tile_keys;
    const uint32_t size = segs[lo].size;
    return {segs[lo].begin + off, size - off < tile_keys ? size - off : tile_keys, lo};
}

// How the slots of a tile's keys are taken (one shared atomic per key at
// most):
//  kSlotsPlain  one atomic per key (keys in random order);
//  kSlotsRuns   a warp whose whole group of 32 V consecutive keys shares a
//               bucket takes its slots with one atomic, else a warp row of
//               32 keys that shares one, else one atomic per key (runs of
//               presorted input; the checks cost about six instructions a
//               key where no run ever forms);
//  kSlotsGroup  every set of lanes with one bucket takes its slots by one
//               atomic of its lowest lane (rows whose lanes often share
//               buckets without the whole row doing so; the match costs more
//               the more distinct buckets a row holds).
constexpr int kSlotsPlain = 0;
constexpr int kSlotsRuns = 1;
constexpr int kSlotsGroup = 2;

// dsel (nullable): one byte per (segment, bucket) cursor; a bucket whose byte
// is set is written to dst2 instead of dst (at the same offsets), so that
// buckets final after this pass can land in the output while the others go
// to the temporary buffer of the next pass.
template <typename K, int MODE, int SLOTS = kSlotsRuns>
__global__ void __launch_bounds__(kFastThreads, 2)
ss_scatter_keys(const K* __restrict__ src, K* __restrict__ dst, const TileDesc* __restrict__ tiles,
                const SegDesc* __restrict__ segs, uint32_t nsegs, uint32_t ntiles,
                const K* __restrict__ splitters,
                const uint32_t* __restrict__ nsplit, K flip, uint32_t shift,
                uint32_t* __restrict__ cursor, uint32_t* __restrict__ err,
                K* __restrict__ dst2 = nullptr, const uint8_t* __restrict__ dsel = nullptr,
                const uint8_t* __restrict__ table = nullptr) {
    constexpr int IPT = FastCfg<K>::kIpt;
    constexpr uint32_t TILE = FastCfg<K>::kTileKeys;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    FastSmem<K>& S = *reinterpret_cast<FastSmem<K>*>(smem_raw);
    const uint32_t tid = threadIdx.x;
    const uint32_t G = gridDim.x;

    constexpr uint32_t kSpBytes = 2 * kSlots * (uint32_t)sizeof(K);
    auto issue = [&](int s, uint32_t k) {   // thread 0
        if (k >= ntiles) { cp_async_commit(); return; }   // keep one group per issue
        const TileDesc t = tiles ? tiles[k] : tile_of(S.seg, nsegs, k, TILE);
        S.tile[s] = t;
        constexpr bool kTree = MODE == kSplit;
        issue_run(S.buf[s], src + t.begin, t.size, &S.bar[s], kTree ? kSpBytes : 0u);
        if constexpr (kTree)
            bulk_load(S.sp[s], splitters + (size_t)t.seg * 2 * kSlots, kSpBytes, &S.bar[s]);
    };
    if (!tiles) {   // nsegs <= kSegCache (the host checks)
        for (uint32_t q = tid; q < nsegs; q += kFastThreads) S.seg[q] = segs[q];
        __syncthreads();
    }
    if (tid == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        mbar_init_fence();
        issue(0, blockIdx.x);
        issue(1, blockIdx.x + G);
    }
    for (uint32_t j = tid; j < kCols; j += kFastThreads) S.hist[j] = 0;
    __syncthreads();

    Classifier<K, MODE> cls{};
    cls.table = table;
    if constexpr (MODE == kTable) cls.m = nsplit ? *nsplit : 1u;   // table size
    uint32_t parity = 0;   // bit s: phase of buffer s's barrier
    for (uint32_t it = 0;; ++it) {
        const uint32_t k = blockIdx.x + it * G;
        if (k >= ntiles) break;
        const int s = it & 1;
        if (!mbar_wait(&S.bar[s], (parity >> s) & 1u)) report_error(err, kDevCopyTimeout);
        parity ^= 1u << s;
        if (tid == 0) cp_async_wait_prior();   // head and tail keys of this tile
        __syncthreads();   // also publishes S.tile[s], written when the tile was issued
        const TileDesc t = S.tile[s];
        const SegDesc sg = tiles ? segs[t.seg] : S.seg[t.seg];
        const TileSplit<K> sp(src + t.begin, t.size);
        K* buf = S.buf[s];
        if constexpr (MODE == kSplit) {
            cls.tree = S.sp[s];
            cls.sorted = S.sp[s] + kSlots;
            cls.m = nsplit[t.seg];
        } else {
            cls.mn = (K)sg.min_ord;
            cls.shift = sg.dshift ? sg.dshift - 1 : shift;
        }

        // Bucket of each key and its slot in the tile's run of that bucket
        // (SLOTS says how the slots are taken).
        // br = (slot << 10) | bucket; bucket kCols marks a lane past the tile.
        // Each thread reads its keys as 16-byte vectors of V consecutive keys
        // (key i is element i % V of the thread's vector i / V; the order of
        // keys inside a tile is free without a payload).
        constexpr int V = FastCfg<K>::kVec;
        const uint32_t lane = lane_id();
        K key[IPT];
        uint32_t br[IPT];
        const bool vec_ok = sp.pad == 0;   // the tile starts on a 16-byte boundary
#pragma unroll
        for (int g = 0; g < IPT / V; ++g) {
            const uint32_t p0 = (uint32_t)g * (kFastThreads * V) + tid * V;
            if (vec_ok && p0 + V <= t.size) {
                const Vec16<K> x = *reinterpret_cast<const Vec16<K>*>(&buf[p0]);
#pragma unroll
                for (int e = 0; e < V; ++e) key[g * V + e] = x.e[e];
            } else {
#pragma unroll
                for (int e = 0; e < V; ++e) key[g * V + e] = p0 + e < t.size ? buf[sp.pad + p0 + e] : K(0);
            }
        }
        uint32_t bk[IPT];
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const uint32_t p = (uint32_t)(i / V) * (kFastThreads * V) + tid * V + (uint32_t)(i % V);
            bk[i] = p < t.size ? cls((K)(key[i] ^ flip)) : kCols;
        }
#pragma unroll
        for (int g = 0; g < IPT / V; ++g) {
            if constexpr (SLOTS == kSlotsRuns) {
                // The warp's whole group of 32 V consecutive keys in one bucket
                // (runs of presorted input) takes its slots with one atomic.
                const uint32_t b = bk[g * V];
                bool lane_one = b < kCols;
#pragma unroll
                for (int e = 1; e < V; ++e) lane_one = lane_one && bk[g * V + e] == b;
                const uint32_t bw = __shfl_sync(AHS_FULL_MASK, b, 0);
                if (__all_sync(AHS_FULL_MASK, lane_one && b == bw)) {
                    uint32_t base = 0;
                    if (lane == 0) base = atomicAdd(&S.hist[b], 32u * V);
                    base = __shfl_sync(AHS_FULL_MASK, base, 0) + V * lane;
#pragma unroll
                    for (int e = 0; e < V; ++e) br[g * V + e] = ((base + e) << 10) | b;
                    continue;
                }
            }
#pragma unroll
            for (int e = 0; e < V; ++e) {
                const int i = g * V + e;
                const uint32_t b = bk[i];
                uint32_t r = 0;
                if constexpr (SLOTS == kSlotsGroup) {
                    const uint32_t m = __match_any_sync(AHS_FULL_MASK, b);
                    const uint32_t leader = __ffs(m) - 1;
                    uint32_t base = 0;
                    if (lane == leader && b < kCols) base = atomicAdd(&S.hist[b], (uint32_t)__popc(m));
                    r = __shfl_sync(AHS_FULL_MASK, base, leader) + __popc(m & lanemask_lt());
                } else if constexpr (SLOTS == kSlotsPlain) {
                    r = b < kCols ? atomicAdd(&S.hist[b], 1u) : 0u;
                } else {
                    const uint32_t b0 = __shfl_sync(AHS_FULL_MASK, b, 0);
                    if (__all_sync(AHS_FULL_MASK, b == b0 && b < kCols)) {
                        uint32_t base = 0;
                        if (lane == 0) base = atomicAdd(&S.hist[b], 32u);
                        r = __shfl_sync(AHS_FULL_MASK, base, 0) + lane;
                    } else {
                        r = b < kCols ? atomicAdd(&S.hist[b], 1u) : 0u;
                    }
                }
                br[i] = (r << 10) | b;
            }
        }
        __syncthreads();

        // Reserve each bucket's run in the segment (thread j, bucket j);
        // tile-local run starts.  The reservation's result is first needed
        // after the staging, so the atomic's round trip to L2 overlaps the
        // scan and the staging stores.
        const uint32_t j = tid;   // kFastThreads == kCols
        uint32_t base;
        {
            const uint32_t c = S.hist[j];
            S.hist[j] = 0;
            // c == 0 for every column past the classifier's buckets.
            base = c ? atomicAdd(&cursor[(size_t)t.seg * cursor_stride<MODE>() + j], c) : 0u;
            uint32_t total;
            S.tile_start[j] = block_exclusive_scan<kFastThreads>(c, S.scan, &total);
        }
        __syncthreads();

        // Stage in bucket order (the tile's keys are all in registers now).
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const uint32_t b = br[i] & 1023u;
            if (b < kCols) {
                const uint32_t lp = S.tile_start[b] + (br[i] >> 10);
                if (AHS_DCHECK(lp < t.size, "fast scatter stage", lp)) {
                    buf[lp] = key[i];
                    // A digit is cheaper to recompute than to stage.
                    if constexpr (MODE != kDigit) S.bid[lp] = (uint16_t)b;
                }
            }
        }
        // Where bucket j's run goes.  A run that would leave its segment (a
        // histogram that does not describe these keys) is reported and not
        // written.  Only the reservation stays in a register across the
        // staging; the run's start and size are read back.
        {
            const uint32_t ex = S.tile_start[j];
            const uint32_t c = (j + 1 < kCols ? S.tile_start[j + 1] : t.size) - ex;
            const SegDesc& sq = tiles ? segs[t.seg] : S.seg[t.seg];
            const size_t cj = (size_t)t.seg * cursor_stride<MODE>() + j;
            K* d = (dsel != nullptr && c && dsel[cj]) ? dst2 : dst;
            const bool inside = (unsigned long long)base + c <= sq.size;
            if (!inside) report_error(err, kDevBadState);
            S.gptr[j] = inside ? d + sq.begin + ((long long)base - (long long)ex) : nullptr;
        }
        __syncthreads();

        // Write the staged tile: consecutive lanes write consecutive staged
        // keys, so a warp's store covers one contiguous run.  (Four
        // consecutive keys a thread, stored as vectors, measured slower on
        // GB300: each store instruction then spans keys four apart.)
#pragma unroll 4
        for (uint32_t j = tid; j < t.size; j += kFastThreads) {
            const K x = buf[j];
            uint32_t b;
            if constexpr (MODE == kDigit) b = cls((K)(x ^ flip));
            else b = S.bid[j];
            K* const o = S.gptr[b];
            if (o != nullptr) o[j] = x;
        }
        __syncthreads();
        if (tid == 0) {
            fence_proxy_async_smem();
            issue(s, k + 2 * G);
        }
    }
}

// Per tile of the list: min and max of ord(x), folded into the tile's
// segment slot (mm[2 s] = min, mm[2 s + 1] = max; the host seeds them).
template <typename K>
__global__ void __launch_bounds__(kThreads)
seg_tile_minmax(const K* __restrict__ src, const TileDesc* __restrict__ tiles, K flip,
                unsigned long long* __restrict__ mm) {
    __shared__ unsigned long long s_mn[kThreads / 32], s_mx[kThreads / 32];
    const TileDesc t = tiles[blockIdx.x];
    K mn = ~K(0), mx = 0;
    for (uint32_t i = threadIdx.x; i < t.size; i += kThreads) {
        const K o = src[t.begin + i] ^ flip;
        mn = o < mn ? o : mn;
        mx = o > mx ? o : mx;
    }
    unsigned long long a = warp_min((unsigned long long)mn), b = warp_max((unsigned long long)mx);
    const uint32_t warp = threadIdx.x >> 5;
    if (lane_id() == 0) { s_mn[warp] = a; s_mx[warp] = b; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kThreads / 32; ++w) {
            a = s_mn[w] < a ? s_mn[w] : a;
            b = s_mx[w] > b ? s_mx[w] : b;
        }
        atomicMin(&mm[2 * t.seg], a);
        atomicMax(&mm[2 * t.seg + 1], b);
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename F>
cudaError_t set_smem(F fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Host-built work lists and the per-level device metadata, which lives in the
// context's auxiliary buffer sized for this level.
struct Level {
    std::vector<SegDesc> segs;
    std::vector<TileDesc> tiles;
    std::vector<ChunkDesc> chunks;
    SegDesc* d_segs = nullptr;
    TileDesc* d_tiles = nullptr;
    ChunkDesc* d_chunks = nullptr;
    uint32_t* counts = nullptr;
    uint32_t* chunk_sum = nullptr;
    uint32_t* seg_tot = nullptr;
    uint32_t* seg_base = nullptr;
    uint32_t* cursor = nullptr;
    void* splitters = nullptr;
    uint32_t* nsplit = nullptr;
};

void build_lists(const std::vector<SegRange>& open, Level& L, uint32_t tile_keys = kTile) {
    L.segs.clear();
    L.tiles.clear();
    L.chunks.clear();
    for (uint32_t s = 0; s < open.size(); ++s) {
        SegDesc sd{};
        sd.begin = open[s].begin;
        sd.size = open[s].size;
        sd.min_ord = open[s].min_ord;
        sd.first_chunk = (uint32_t)L.chunks.size();
        const uint32_t nt = (uint32_t)ceil_div(sd.size, tile_keys);
        const uint32_t t0 = (uint32_t)L.tiles.size();
        sd.first_tile = t0;
        for (uint32_t t = 0; t < nt; ++t) {
            const uint32_t off = t * tile_keys;
            L.tiles.push_back({sd.begin + off, std::min(tile_keys, sd.size - off), s});
        }
        for (uint32_t t = 0; t < nt; t += kChunkTiles)
            L.chunks.push_back({t0 + t, std::min(kChunkTiles, nt - t), s, 0});
        sd.nchunks = (uint32_t)L.chunks.size() - sd.first_chunk;
        L.segs.push_back(sd);
    }
}

// Carve the level's metadata in ctx->aux and upload the lists (synchronises
// the stream so the pinned staging can be reused).
ahs_status upload_level(ahs_ctx* ctx, Level& L, uint32_t key_bytes, bool split, cudaStream_t st) {
    const size_t ns = L.segs.size(), nt = L.tiles.size(), nc = L.chunks.size();
    const size_t b_segs = a256(ns * sizeof(SegDesc)), b_tiles = a256(nt * sizeof(TileDesc)),
                 b_chunks = a256(nc * sizeof(ChunkDesc));
    const size_t b_counts = a256(nt * kCols * 4), b_csum = a256(nc * kCols * 4),
                 b_seg = a256(ns * kCols * 4), b_spl = split ? a256(ns * 2 * kSlots * key_bytes) : 0,
                 b_ns = a256(ns * 4);
    ahs_status rc = ensure_aux(ctx, b_segs + b_tiles + b_chunks + b_counts + b_csum + 3 * b_seg +
                                        b_spl + b_ns);
    if (rc == AHS_OK) rc = ensure_stage(ctx, b_segs + b_tiles + b_chunks);
    if (rc != AHS_OK) return rc;
    char* p = static_cast<char*>(ctx->aux);
    L.d_segs = reinterpret_cast<SegDesc*>(p); p += b_segs;
    L.d_tiles = reinterpret_cast<TileDesc*>(p); p += b_tiles;
    L.d_chunks = reinterpret_cast<ChunkDesc*>(p); p += b_chunks;
    L.counts = reinterpret_cast<uint32_t*>(p); p += b_counts;
    L.chunk_sum = reinterpret_cast<uint32_t*>(p); p += b_csum;
    L.seg_tot = reinterpret_cast<uint32_t*>(p); p += b_seg;
    L.seg_base = reinterpret_cast<uint32_t*>(p); p += b_seg;
    L.cursor = reinterpret_cast<uint32_t*>(p); p += b_seg;
    L.splitters = split ? p : nullptr; p += b_spl;
    L.nsplit = reinterpret_cast<uint32_t*>(p);
    char* hs = static_cast<char*>(ctx->h_stage);
    std::memcpy(hs, L.segs.data(), ns * sizeof(SegDesc));
    std::memcpy(hs + b_segs, L.tiles.data(), nt * sizeof(TileDesc));
    std::memcpy(hs + b_segs + b_tiles, L.chunks.data(), nc * sizeof(ChunkDesc));
    cudaError_t e = launch_transfer(L.d_segs, hs, b_segs + b_tiles + b_chunks, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(ctx, e);
}

// One partition of every segment of the level, src -> dst: stable with a
// payload (count matrix, segmented column scan, ranked scatter), unstable
// without (bucket totals, cursors, persistent scatter) -- FAST, keys only.
template <typename K, bool VALS, int MODE>
cudaError_t partition(const Level& L, const K* src, K* dst, const uint32_t* vsrc, uint32_t* vdst,
                      K flip, uint32_t level, uint32_t shift, bool totals, cudaStream_t st,
                      bool fast = false, int sms = kDefaultSms, uint32_t* err = nullptr) {
    const uint32_t ns = (uint32_t)L.segs.size(), nt = (uint32_t)L.tiles.size(),
                   nc = (uint32_t)L.chunks.size();
    uint64_t keys = 0;
    for (const SegDesc& sd : L.segs) keys += sd.size;
    K* spl = static_cast<K*>(L.splitters);
    if constexpr (MODE == kSplit) {
        TraceScope ts("sample_splitters", ns, st);
        ss_sample<K><<<ns, kThreads, sizeof(BlockSortSmem<K, false, kThreads, kIpt>), st>>>(
            src, L.d_segs, level, flip, spl, L.nsplit);
    }
    if (!VALS && fast) {
        cudaError_t e = launch_zero32(L.seg_tot, (uint64_t)ns * kCols, sms, st);
        if (e != cudaSuccess) return e;
        {
            TraceScope ts(MODE == kSplit ? "sample_count" : "segradix_count", keys, st);
            ss_count<K, MODE, true><<<nt, kThreads, 0, st>>>(src, L.d_tiles, L.d_segs, spl,
                                                             L.nsplit, flip, shift, L.seg_tot);
        }
        {
            TraceScope ts(MODE == kSplit ? "sample_scan" : "segradix_scan", ns, st);
            ss_scan_totals<<<ns, kCols, 0, st>>>(L.seg_tot, L.seg_base, L.cursor);
        }
        {
            const uint32_t grid = (uint32_t)std::min<uint64_t>(nt, 2ull * (uint64_t)sms);
            TraceScope ts(MODE == kSplit ? "sample_scatter" : "segradix_scatter", keys, st);
            ss_scatter_keys<K, MODE><<<grid, kFastThreads, sizeof(FastSmem<K>), st>>>(
                src, dst, L.d_tiles, L.d_segs, ns, nt, spl, L.nsplit, flip, shift, L.cursor, err);
        }
        return cudaGetLastError();
    }
    {
        TraceScope ts(MODE == kSplit ? "sample_count" : "segradix_count", keys, st);
        ss_count<K, MODE, false><<<nt, kThreads, 0, st>>>(src, L.d_tiles, L.d_segs, spl, L.nsplit,
                                                          flip, shift, L.counts);
    }
    {
        TraceScope ts(MODE == kSplit ? "sample_scan" : "segradix_scan", nt, st);
        ss_scan_a<<<nc, kCols, 0, st>>>(L.counts, L.d_chunks, L.chunk_sum);
        ss_scan_b<<<ns, kCols, 0, st>>>(L.chunk_sum, L.d_segs, totals ? L.seg_tot : nullptr,
                                        L.seg_base);
        ss_scan_c<<<nc, kCols, 0, st>>>(L.counts, L.d_chunks, L.chunk_sum);
    }
    {
        TraceScope ts(MODE == kSplit ? "sample_scatter" : "segradix_scatter", keys, st);
        ss_scatter<K, VALS, MODE><<<nt, kThreads, sizeof(ScatterSmem<K, VALS>), st>>>(
            src, dst, vsrc, vdst, L.d_tiles, L.d_segs, spl, L.nsplit, flip, shift, L.counts);
    }
    return cudaGetLastError();
}

template <typename K, bool VALS>
cudaError_t set_attrs() {
    cudaError_t e = set_smem(ss_sample<K>, sizeof(BlockSortSmem<K, false, kThreads, kIpt>));
    if (e == cudaSuccess) e = set_smem(ss_scatter<K, VALS, kSplit>, sizeof(ScatterSmem<K, VALS>));
    if (e == cudaSuccess) e = set_smem(ss_scatter<K, VALS, kDigit>, sizeof(ScatterSmem<K, VALS>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kSplit>, sizeof(FastSmem<K>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kDigit, kSlotsPlain>, sizeof(FastSmem<K>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kDigit, kSlotsRuns>, sizeof(FastSmem<K>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kDigit, kSlotsGroup>, sizeof(FastSmem<K>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kTable, kSlotsPlain>, sizeof(FastSmem<K>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kTable, kSlotsRuns>, sizeof(FastSmem<K>));
    if (e == cudaSuccess) e = set_smem(ss_scatter_keys<K, kTable, kSlotsGroup>, sizeof(FastSmem<K>));
    return e;
}

// ss_scatter_keys with its slot mode chosen at run time.
template <typename K, int MODE, typename... A>
cudaError_t launch_scatter_keys(int slots, uint32_t grid, size_t smem, cudaStream_t st, A... args) {
    if (slots == kSlotsGroup)
        ss_scatter_keys<K, MODE, kSlotsGroup><<<grid, kFastThreads, smem, st>>>(args...);
    else if (slots == kSlotsPlain)
        ss_scatter_keys<K, MODE, kSlotsPlain><<<grid, kFastThreads, smem, st>>>(args...);
    else
        ss_scatter_keys<K, MODE, kSlotsRuns><<<grid, kFastThreads, smem, st>>>(args...);
    return cudaGetLastError();
}

// Final buckets written straight into the pinned staging, one region of
// `cap` entries per size class of the bucket kernels; unsorted (copy) buckets
// larger than kCopyChunk are split so that many CTAs share them.
struct ClassLists {
    FinalBucket* region[kBucketClasses];
    size_t cap = 0;
    uint32_t count[kBucketClasses] = {};
    uint64_t keys[kBucketClasses] = {};
    uint32_t sorted = 0;
    bool overflow = false;
    void put(int k, const FinalBucket& f) {
        if (count[k] >= cap) { overflow = true; return; }
        region[k][count[k]++] = f;
        keys[k] += f.size;
    }
    void add(const FinalBucket& f) {
        if (!f.sort && f.size > kCopyChunk) {
            for (uint32_t o = 0; o < f.size; o += kCopyChunk)
                put(0, final_bucket(f.begin + o, std::min(kCopyChunk, f.size - o), f.where, false));
            return;
        }
        put(f.sort ? (int)bucket_class(f.size) : 0, f);
        sorted += f.sort;
    }
};


// Final buckets sorted into the size classes as they are found (a large
// copy, the equality bucket of a heavy key, is split so that many CTAs share
// it), so the upload is one copy per class.
struct FinalSet {
    std::vector<FinalBucket> cls[kBucketClasses];
    uint64_t keys[kBucketClasses] = {};
    uint32_t sorted = 0;
    void reserve(size_t n) {
        cls[0].reserve(n / 4 + 64);
        for (int k = 1; k < kBucketClasses; ++k) cls[k].reserve(n / 2 + 16);
    }
    void add(const FinalBucket& f) {
        if (!f.sort && f.size > kCopyChunk) {
            for (uint32_t o = 0; o < f.size; o += kCopyChunk)
                cls[0].push_back(final_bucket(f.begin + o, std::min(kCopyChunk, f.size - o), f.where, false));
            keys[0] += f.size;
            return;
        }
        const int k = f.sort ? (int)bucket_class(f.size) : 0;
        cls[k].push_back(f);
        keys[k] += f.size;
        sorted += f.sort;
    }
};

// Upload a final-bucket set to the auxiliary buffer and run the bucket sorts
// (one launch per size class); synchronises before returning so the pinned
// staging can be reused.
ahs_status finish_buckets_sets(ahs_ctx* ctx, const FinalSet* sets, size_t nsets, const void* ktmp,
                               const void* kout, const void* kin, const uint32_t* vtmp, uint32_t* vout,
                               const uint32_t* vin, KeyDesc kd, cudaStream_t st, uint32_t* sorted) {
    // Class k's list is the concatenation of every set's class-k entries.
    size_t nf = 0, at[kBucketClasses];
    uint32_t counts[kBucketClasses];
    uint64_t keys[kBucketClasses];
    uint32_t nsorted = 0;
    for (int k = 0; k < kBucketClasses; ++k) {
        at[k] = nf;
        size_t c = 0;
        uint64_t kk = 0;
        for (size_t i = 0; i < nsets; ++i) {
            c += sets[i].cls[k].size();
            kk += sets[i].keys[k];
        }
        counts[k] = (uint32_t)c;
        keys[k] = kk;
        nf += c;
    }
    for (size_t i = 0; i < nsets; ++i) nsorted += sets[i].sorted;
    if (sorted) *sorted = nsorted;
    if (nf == 0) return AHS_OK;
    ahs_status rc = ensure_aux(ctx, nf * sizeof(FinalBucket));
    if (rc == AHS_OK) rc = ensure_stage(ctx, nf * sizeof(FinalBucket));
    if (rc != AHS_OK) return rc;
    FinalBucket* hf = static_cast<FinalBucket*>(ctx->h_stage);
    FinalBucket* df = static_cast<FinalBucket*>(ctx->aux);
    const FinalBucket* lists[kBucketClasses];
    // (set, class) pieces copied into the pinned staging in parallel.
    std::vector<std::pair<size_t, int>> piece;
    std::vector<size_t> dst;
    for (int k = 0; k < kBucketClasses; ++k) {
        size_t o = at[k];
        for (size_t i = 0; i < nsets; ++i) {
            if (!sets[i].cls[k].empty()) {
                piece.push_back({i, k});
                dst.push_back(o);
            }
            o += sets[i].cls[k].size();
        }
        lists[k] = df + at[k];
    }
    parallel_chunks(piece.size(), chunks_for(nf, 1u << 16), [&](size_t, size_t lo, size_t hi) {
        for (size_t q = lo; q < hi; ++q) {
            const std::vector<FinalBucket>& v = sets[piece[q].first].cls[piece[q].second];
            std::memcpy(hf + dst[q], v.data(), v.size() * sizeof(FinalBucket));
        }
    });
    cudaError_t e = launch_transfer(df, hf, nf * sizeof(FinalBucket), st);
    if (e == cudaSuccess)
        e = launch_bucket_finish(lists, counts, keys, ktmp, kout, kin, const_cast<void*>(kout),
                                 vtmp, vout, vin, vout, kd, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(ctx, e);
}

ahs_status finish_buckets(ahs_ctx* ctx, const FinalSet& fs, const void* ktmp, const void* kout,
                          const void* kin, const uint32_t* vtmp, uint32_t* vout, const uint32_t* vin,
                          KeyDesc kd, cudaStream_t st, uint32_t* sorted) {
    return finish_buckets_sets(ctx, &fs, 1, ktmp, kout, kin, vtmp, vout, vin, kd, st, sorted);
}

// Partition levels by sampled splitters until every bucket fits a CTA, then
// the bucket sorts.
template <typename K, bool VALS>
ahs_status general_t(ahs_ctx* ctx, const K* kin, K* kout, const uint32_t* vin, uint32_t* vout,
                     uint64_t n_total, const std::vector<SegRange>& segs,
                     const std::vector<SegRange>& extra, K flip, void* scratch, cudaStream_t st,
                     uint32_t* levels_out, uint32_t* buckets_out) {
    char* p = static_cast<char*>(scratch);
    K* ktmp = reinterpret_cast<K*>(p);
    uint32_t* vtmp = VALS ? reinterpret_cast<uint32_t*>(p + a256(n_total * sizeof(K))) : nullptr;
    cudaError_t e = set_attrs<K, VALS>();
    if (e != cudaSuccess) return cuda_status(ctx, e);

    // Final buckets in several sets: one for the segments that need no
    // level, then one per planning thread per level.
    std::vector<FinalSet> finals(1);
    finals[0].reserve(extra.size() + segs.size() + 64);
    for (const SegRange& x : extra)
        finals[0].add(final_bucket(x.begin, x.size, 2, x.size > 1));
    std::vector<SegRange> open;
    for (const SegRange& x : segs) {
        if (x.size <= kBucketCap) finals[0].add(final_bucket(x.begin, x.size, 2, x.size > 1));
        else open.push_back(x);
    }
    Level L;
    uint32_t level = 0;
    while (!open.empty()) {
        if (level >= kMaxLevels) return AHS_ERR_UNIMPLEMENTED;
        ++level;
        // Level 1 reads the input; odd levels write the temporary buffer, even
        // levels the output, so a level never overwrites its own source.
        const K* src = level == 1 ? kin : (level % 2 == 0 ? ktmp : kout);
        const uint32_t* vsrc = level == 1 ? vin : (level % 2 == 0 ? vtmp : vout);
        K* dst = (level % 2 == 1) ? ktmp : kout;
        uint32_t* vdst = (level % 2 == 1) ? vtmp : vout;
        const uint8_t where = (level % 2 == 1) ? 0 : 1;
        build_lists(open, L, VALS ? kTile : FastCfg<K>::kTileKeys);
        ahs_status rc = upload_level(ctx, L, sizeof(K), true, st);
        if (rc != AHS_OK) return rc;
        e = partition<K, VALS, kSplit>(L, src, dst, vsrc, vdst, flip, level, 0, true, st, !VALS,
                                       ctx->sms, ctx->d_err);
        const size_t ns = L.segs.size(), bread = ns * kCols * 4;
        if (e == cudaSuccess) rc = ensure_stage(ctx, 2 * bread);
        if (rc != AHS_OK) return rc;
        char* hs = static_cast<char*>(ctx->h_stage);
        if (e == cudaSuccess) e = launch_transfer(hs, L.seg_tot, bread, st);
        if (e == cudaSuccess) e = launch_transfer(hs + bread, L.seg_base, bread, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(ctx, e);
        const uint32_t* tot = reinterpret_cast<const uint32_t*>(hs);
        const uint32_t* base = reinterpret_cast<const uint32_t*>(hs + bread);
        // Each segment's buckets: final (sorted or copied) or open at the
        // next level -- planned by segment in parallel.
        const size_t nch = chunks_for(ns, 256);
        const size_t f0 = finals.size();
        finals.resize(f0 + nch);
        std::vector<std::vector<SegRange>> next_of(nch);
        parallel_chunks(ns, nch, [&](size_t c, size_t lo, size_t hi) {
            FinalSet& fs = finals[f0 + c];
            uint64_t keys = 0;
            for (size_t q = lo; q < hi; ++q) keys += L.segs[q].size;
            fs.reserve(keys / (kBucketCap / 2) + 64);
            for (size_t q = lo; q < hi; ++q) {
                const uint32_t cols = 2 * split_count(L.segs[q].size) + 1;   // buckets in use
                for (uint32_t j = 0; j < cols; ++j) {
                    const uint32_t sz = tot[q * kCols + j];
                    if (sz == 0) continue;
                    const unsigned long long b0 = L.segs[q].begin + base[q * kCols + j];
                    const bool equal = (j & 1u) != 0;
                    if (equal || sz == 1) {
                        if (where == 0) fs.add(final_bucket(b0, sz, where, false));   // copy to output
                    } else if (sz <= kBucketCap) {
                        fs.add(final_bucket(b0, sz, where, true));
                    } else {
                        next_of[c].push_back({b0, sz, 0});
                    }
                }
            }
        });
        std::vector<SegRange> next;
        for (auto& v : next_of) next.insert(next.end(), v.begin(), v.end());
        open.swap(next);
    }
    *levels_out = level;
    return finish_buckets_sets(ctx, finals.data(), finals.size(), ktmp, kout, kin, vtmp, vout, vin,
                               KeyDesc{(uint32_t)sizeof(K), (uint64_t)flip}, st, buckets_out);
}

template <typename K, bool VALS>
ahs_status radix_segs_t(ahs_ctx* ctx, const K* kin, K* kout, const uint32_t* vin, uint32_t* vout,
                        uint64_t n_total, const std::vector<SegRange>& segs, uint32_t passes,
                        K flip, void* scratch, cudaStream_t st) {
    if (segs.empty() || passes == 0) return AHS_OK;
    char* p = static_cast<char*>(scratch);
    K* ktmp = reinterpret_cast<K*>(p);
    uint32_t* vtmp = VALS ? reinterpret_cast<uint32_t*>(p + a256(n_total * sizeof(K))) : nullptr;
    cudaError_t e = set_attrs<K, VALS>();
    if (e != cudaSuccess) return cuda_status(ctx, e);
    Level L;
    build_lists(segs, L);
    ahs_status rc = upload_level(ctx, L, sizeof(K), false, st);
    if (rc != AHS_OK) return rc;
    // The last pass writes kout: odd pass counts start kin -> kout.
    const K* src = kin;
    const uint32_t* vsrc = vin;
    for (uint32_t q = 0; q < passes; ++q) {
        const bool to_out = ((passes - 1 - q) % 2) == 0;
        K* dst = to_out ? kout : ktmp;
        uint32_t* vdst = to_out ? vout : vtmp;
        e = partition<K, VALS, kDigit>(L, src, dst, vsrc, vdst, flip, 0, 8 * q, false, st);
        if (e != cudaSuccess) return cuda_status(ctx, e);
        src = dst;
        vsrc = vdst;
    }
    return AHS_OK;
}

// ------------------------------------------------- keys-only histogram-guided partitions
//
// The feature pass leaves the exact histogram of the top 16 bits of
// u = ord(x) - min (bin = u >> s, s = bitlen(span) - 16), so partition passes
// whose bucket boundaries are bin boundaries know their bucket sizes without a
// counting pass:
//   RADIX (most significant digit first): pass 1 by the high byte of the bin,
//     pass 2 by its low byte -- every bin's keys then sit at their final
//     position, and a bin holds keys that differ only in their low s bits.
//   GENERAL (sample sort with splitters from the histogram): level 1 splits at
//     boundaries of 256-bin blocks when no block holds more than twice its
//     share of the keys (classified by bit extraction), else at runs of bins
//     of about n / 256 keys each (classified by a bin -> bucket table); level
//     2 cuts each run into buckets spanning at most 16 bits of u.
//   Level 1 writes the runs that level 2 does not split straight to the
//   output.  (Measured on GB300 for Zipf keys: the table classifier is bound
//   by the latency of its lookups -- the 64 KB table does not stay in the L1
//   that shared memory leaves -- so a level 1 by runs costs more than the
//   level-2 traffic it saves; the radix strategy keeps bit extraction.)
// Buckets that fit a CTA are sorted in shared memory; larger ones (bins heavier
// than a CTA, with no finer information in the histogram) are checked for a
// single value and otherwise sample-sorted.  All lists of a sort are built on
// the host up front and uploaded in one copy, and the passes and bucket sorts
// are launched back to back.

// Upload segments, tiles and host-computed cursors of one pass into ctx->aux.
ahs_status upload_msd(ahs_ctx* ctx, Level& L, const std::vector<uint32_t>& cursor, cudaStream_t st,
                      const void* splitters = nullptr, size_t splitter_bytes = 0) {
    const size_t ns = L.segs.size(), nt = L.tiles.size();
    const size_t b_segs = a256(ns * sizeof(SegDesc)), b_tiles = a256(nt * sizeof(TileDesc)),
                 b_cur = a256(cursor.size() * 4), b_spl = a256(splitter_bytes);
    const size_t total = b_segs + b_tiles + b_cur + b_spl;
    ahs_status rc = ensure_aux(ctx, total);
    if (rc == AHS_OK) rc = ensure_stage(ctx, total);
    if (rc != AHS_OK) return rc;
    char* p = static_cast<char*>(ctx->aux);
    L.d_segs = reinterpret_cast<SegDesc*>(p);
    L.d_tiles = reinterpret_cast<TileDesc*>(p + b_segs);
    L.cursor = reinterpret_cast<uint32_t*>(p + b_segs + b_tiles);
    L.splitters = splitter_bytes ? p + b_segs + b_tiles + b_cur : nullptr;
    char* hs = static_cast<char*>(ctx->h_stage);
    std::memcpy(hs, L.segs.data(), ns * sizeof(SegDesc));
    std::memcpy(hs + b_segs, L.tiles.data(), nt * sizeof(TileDesc));
    if (!cursor.empty()) std::memcpy(hs + b_segs + b_tiles, cursor.data(), cursor.size() * 4);
    if (splitter_bytes) std::memcpy(hs + b_segs + b_tiles + b_cur, splitters, splitter_bytes);
    cudaError_t e = launch_transfer(p, hs, total, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(ctx, e);
}

// Host: greedy grouping of bins [b0, b1) into at most 256 runs of about
// `target` keys and at most `max_bins` bins (a bin heavier than the target
// is a run of its own).  Returns the first bin of every run after the first.
std::vector<uint32_t> group_bins(const HistView& hist, uint32_t b0,
                                 uint32_t b1, unsigned long long target,
                                 uint32_t max_bins = 0xffffffffu) {
    std::vector<uint32_t> starts;
    unsigned long long acc = 0;
    uint32_t first = b0;
    for (uint32_t b = b0; b < b1; ++b) {
        if (b > first && (acc + hist[b] > target || b - first >= max_bins) &&
            starts.size() < kSlots - 1) {
            starts.push_back(b);
            acc = 0;
            first = b;
        }
        acc += hist[b];
    }
    return starts;
}

// Runs of the output larger than one CTA sorts, each the keys of one or a few
// histogram bins: a min / max pass drops those holding a single value, the
// rest are sorted in place by the sample sort.
template <typename K>
ahs_status finish_large(ahs_ctx* ctx, const std::vector<SegRange>& large, K* kout, uint64_t n,
                        K flip, void* scratch, cudaStream_t st, uint32_t* levels_out,
                        uint32_t* buckets_out) {
    if (large.empty()) return AHS_OK;
    K* ktmp = static_cast<K*>(scratch);
    Level L;
    std::vector<SegRange> multi;
    build_lists(large, L, kTile);
    ahs_status rc = upload_msd(ctx, L, {}, st);
    if (rc != AHS_OK) return rc;
    const size_t ns = large.size();
    // The temporary buffer is free here: it holds the min / max slots.
    unsigned long long* d_mm = reinterpret_cast<unsigned long long*>(ktmp);
    std::vector<unsigned long long> seed(2 * ns);
    for (size_t q = 0; q < ns; ++q) { seed[2 * q] = ~0ull; seed[2 * q + 1] = 0ull; }
    rc = ensure_stage(ctx, 2 * ns * 8);
    if (rc != AHS_OK) return rc;
    std::memcpy(ctx->h_stage, seed.data(), 2 * ns * 8);
    cudaError_t e = launch_transfer(d_mm, ctx->h_stage, 2 * ns * 8, st);
    if (e == cudaSuccess) {
        uint64_t lk = 0;
        for (const SegRange& x : large) lk += x.size;
        TraceScope ts("msd_bin_minmax", lk, st);
        seg_tile_minmax<K><<<(uint32_t)L.tiles.size(), kThreads, 0, st>>>(kout, L.d_tiles, flip, d_mm);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = launch_transfer(ctx->h_stage, d_mm, 2 * ns * 8, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    const unsigned long long* mm = static_cast<const unsigned long long*>(ctx->h_stage);
    for (size_t q = 0; q < ns; ++q)
        if (mm[2 * q] != mm[2 * q + 1]) multi.push_back({large[q].begin, large[q].size, mm[2 * q]});
    if (multi.empty()) return AHS_OK;
    uint32_t lv = 0, bk = 0;
    rc = general_t<K, false>(ctx, kout, kout, nullptr, nullptr, n, multi, {}, flip, scratch, st, &lv, &bk);
    *levels_out += lv;
    *buckets_out += bk;
    return rc;
}


// Arrays appended at 256-byte offsets into a window of the pinned staging
// buffer, later copied in one piece to the same offsets of ctx->aux.
struct Blob {
    char* base;      // pinned host window
    size_t cap;
    size_t used = 0;
    size_t add(const void* p, size_t bytes) {
        const size_t off = used;
        used += a256(bytes ? bytes : 1);
        if (used > cap) return ~size_t(0);   // caller checks overflow()
        if (bytes) std::memcpy(base + off, p, bytes);
        return off;
    }
    bool overflow() const { return used > cap; }
};


template <typename K>
ahs_status keys_hist_t(ahs_ctx* ctx, const K* kin, K* kout, uint64_t n, K flip, K mn,
                       const HistView& hist, uint32_t shift, bool msd,
                       uint32_t group, void* scratch, cudaStream_t st, uint32_t* levels_out,
                       uint32_t* buckets_out) {
    K* ktmp = static_cast<K*>(scratch);
    cudaError_t e = set_attrs<K, false>();
    if (e != cudaSuccess) return cuda_status(ctx, e);
    constexpr uint32_t TK = FastCfg<K>::kTileKeys;
    const uint32_t nbins = (uint32_t)hist.size();
    const bool inplace = static_cast<const void*>(kin) == static_cast<const void*>(kout);
    std::vector<unsigned long long> binpos(nbins + 1, 0);
    for (uint32_t i = 0; i < nbins; ++i) binpos[i + 1] = binpos[i] + hist[i];
    if (binpos[nbins] != n) return AHS_ERR_CUDA;   // the histogram must describe these keys
    // Keys of bins [b0, b1) lie in [bin_lo(b0), bin_lo(b0) + 2^range_bits(b0, b1)).
    auto bin_lo = [&](uint32_t b) { return (unsigned long long)(K)(mn + ((K)b << shift)); };
    auto range_bits = [&](uint32_t b0, uint32_t b1) {
        return bitlen64((((unsigned long long)(b1 - b0)) << shift) - 1);
    };

    // Staging and device windows for the three uploads (level 1, level 2,
    // final buckets), sized by upper bounds so that no upload has to wait for
    // an earlier one: the host prepares level 2 while level 1 runs, and the
    // bucket lists while level 2 runs.
    const size_t capA = a256(sizeof(SegDesc)) + a256(kCols * 4) + a256(kMaxBins) + 256 + a256(kCols);
    const size_t capB = 2 * (a256(256 * sizeof(SegDesc)) + a256(256 * kCols * 4) + a256(kMaxBins) + 256);
    const size_t class_cap = nbins + n / kCopyChunk + 8;   // entries of one class region
    const size_t class_bytes = a256(class_cap * sizeof(FinalBucket));
    const size_t capC = kBucketClasses * class_bytes;
    ahs_status rc = ensure_aux(ctx, capA + capB + capC);
    if (rc == AHS_OK) rc = ensure_stage(ctx, capA + capB + capC);
    if (rc != AHS_OK) return rc;
    char* aux = static_cast<char*>(ctx->aux);
    char* stage = static_cast<char*>(ctx->h_stage);

    // One partition pass: segments (min_ord carries the first bin), the bin
    // starts of each segment's buckets after the first, and its classifier.
    struct Pass {
        std::vector<SegRange> segs;
        std::vector<std::vector<uint32_t>> starts;
        bool digit = false;
        int slots = kSlotsRuns;   // how the kernel takes the keys' slots
        uint32_t dshift = 0;
        const K* src = nullptr;
        K* dst = nullptr;
        K* dst2 = nullptr;              // buckets whose dsel byte is set go here
        std::vector<uint8_t> dsel;      // per (segment, bucket) cursor; empty: all to dst
        std::vector<uint32_t> ends;     // last bin + 1 of each segment
    };
    // Lists of `P` into the blob, then its launch (after the blob's copy).
    struct Placed {
        size_t o_segs, o_cur, o_tbl, o_tbn, o_dsel;
        uint32_t ns, nt;
        uint64_t keys;
    };
    auto place = [&](const Pass& P, Blob& blob) -> Placed {
        // Segments with their first tile; the kernel derives the tiles.
        std::vector<SegDesc> segs(P.segs.size());
        uint32_t nt = 0;
        for (size_t q = 0; q < P.segs.size(); ++q) {
            SegDesc& sd = segs[q];
            sd.begin = P.segs[q].begin;
            sd.size = P.segs[q].size;
            sd.min_ord = P.segs[q].min_ord;
            sd.first_tile = nt;
            nt += (uint32_t)ceil_div(sd.size, TK);
        }
        constexpr uint32_t CS = cursor_stride<kDigit>();
        static_assert(CS == cursor_stride<kTable>(), "one cursor layout for both classifiers");
        std::vector<uint32_t> cur(P.segs.size() * CS, 0);
        // Table classifier: the bucket of every bin the pass's segments cover
        // (segments are disjoint runs of bins, so one table serves them all).
        std::vector<uint8_t> tbl;
        if (!P.digit) tbl.assign(nbins, 0);
        Placed pl{};
        for (size_t q = 0; q < P.segs.size(); ++q) {
            const uint32_t first = (uint32_t)P.segs[q].min_ord;   // first bin of the segment
            for (size_t j = 0; j < P.starts[q].size(); ++j) {
                const uint32_t b = P.starts[q][j];
                cur[q * CS + j + 1] = (uint32_t)(binpos[b] - binpos[first]);
            }
            if (!P.digit) {
                uint32_t bucket = 0;
                for (uint32_t b = first, j = 0; b < P.ends[q]; ++b) {
                    while (j < P.starts[q].size() && P.starts[q][j] <= b) { ++j; ++bucket; }
                    tbl[b] = (uint8_t)bucket;
                }
            }
            pl.keys += P.segs[q].size;
        }
        // The digit classifier takes the ord value of the segment's first bin,
        // the table classifier the bin origin (the input's smallest key).
        for (SegDesc& sd : segs)
            sd.min_ord = P.digit ? (unsigned long long)(K)(mn + ((K)sd.min_ord << shift))
                                 : (unsigned long long)mn;
        pl.o_segs = blob.add(segs.data(), segs.size() * sizeof(SegDesc));
        pl.o_cur = blob.add(cur.data(), cur.size() * 4);
        pl.o_tbl = P.digit ? 0 : blob.add(tbl.data(), tbl.size());
        const uint32_t tbl_n = nbins;
        pl.o_tbn = P.digit ? 0 : blob.add(&tbl_n, sizeof(tbl_n));
        pl.o_dsel = P.dsel.empty() ? 0 : blob.add(P.dsel.data(), P.dsel.size());
        pl.ns = (uint32_t)segs.size();
        pl.nt = nt;
        return pl;
    };
    auto upload = [&](const Blob& blob, size_t window) -> cudaError_t {
        return launch_transfer(aux + window, stage + window, blob.used, st);
    };
    auto launch = [&](const Pass& P, const Placed& pl, size_t window) -> cudaError_t {
        if (pl.ns > kSegCache) return cudaErrorInvalidValue;   // level-1 runs are at most 256
        const uint32_t grid = (uint32_t)std::min<uint64_t>(pl.nt, 2ull * (uint64_t)ctx->sms);
        const char* w = aux + window;
        const SegDesc* d_segs = reinterpret_cast<const SegDesc*>(w + pl.o_segs);
        uint32_t* d_cur = reinterpret_cast<uint32_t*>(aux + window + pl.o_cur);
        TraceScope ts(msd ? "msd_scatter" : "sample_scatter", pl.keys, st);
        const uint8_t* tbl = P.digit ? nullptr : reinterpret_cast<const uint8_t*>(w + pl.o_tbl);
        const uint32_t* tbn = P.digit ? nullptr : reinterpret_cast<const uint32_t*>(w + pl.o_tbn);
        const uint8_t* dsel = P.dsel.empty() ? nullptr : reinterpret_cast<const uint8_t*>(w + pl.o_dsel);
        const TileDesc* no_tiles = nullptr;
        const K* no_splitters = nullptr;
        if (P.digit)
            return launch_scatter_keys<K, kDigit>(P.slots, grid, sizeof(FastSmem<K>), st, P.src, P.dst,
                                                  no_tiles, d_segs, pl.ns, pl.nt, no_splitters,
                                                  (const uint32_t*)nullptr, flip, P.dshift, d_cur,
                                                  ctx->d_err, P.dst2, dsel, (const uint8_t*)nullptr);
        return launch_scatter_keys<K, kTable>(P.slots, grid, sizeof(FastSmem<K>), st, P.src, P.dst,
                                              no_tiles, d_segs, pl.ns, pl.nt, no_splitters, tbn, flip,
                                              shift, d_cur, ctx->d_err, P.dst2, dsel, tbl);
    };

    // A level-1 run of bins [b0, b1) is split by level 2 when it holds more
    // than a CTA's keys in more than one bin.
    auto splits_further = [&](uint32_t b0, uint32_t b1) {
        return binpos[b1] - binpos[b0] > kBucketCap && b1 - b0 > 1;
    };

    const int runs_slots = (group & kRunsLikely) ? kSlotsRuns : kSlotsPlain;
    // Level 1: input -> temporary (runs that level 2 splits) or output.
    const unsigned long long share = std::max<unsigned long long>((n + 255) / 256, 1);
    bool blocks = nbins > 256;
    for (uint32_t c = 0; !msd && blocks && c * 256 < nbins; ++c)
        blocks = binpos[std::min(nbins, (c + 1) * 256)] - binpos[c * 256] <= 2 * share;
    std::vector<uint32_t> s1;
    if (blocks) {
        for (uint32_t b = 256; b < nbins; b += 256) s1.push_back(b);
    } else {
        s1 = group_bins(hist, 0, nbins, share);
    }
    {
        Pass P1;
        P1.segs.push_back({0ull, (uint32_t)n, 0ull});
        P1.starts.push_back(s1);
        P1.ends.push_back(nbins);
        P1.digit = blocks;
        P1.dshift = shift + 8;
        // Probability that two random keys share a level-1 bucket.
        double d1 = 0.0;
        for (size_t g = 0; g <= s1.size(); ++g) {
            const uint32_t b0 = g == 0 ? 0u : s1[g - 1], b1 = g == s1.size() ? nbins : s1[g];
            const double share = (double)(binpos[b1] - binpos[b0]) / (double)n;
            d1 += share * share;
        }
        P1.slots = (group & kGroupLevel1) != 0 || d1 >= kGroupCollide ? kSlotsGroup : runs_slots;
        P1.src = kin;
        P1.dst = ktmp;
        // Runs that no later pass splits (at most a CTA's keys, or one bin)
        // are written straight to the output -- unless the output is the
        // input, which other tiles of this pass are still reading.
        if (!inplace) {
            P1.dst2 = kout;
            P1.dsel.assign(cursor_stride<kDigit>(), 0);
            for (size_t g = 0; g <= s1.size(); ++g) {
                const uint32_t b0 = g == 0 ? 0u : s1[g - 1], b1 = g == s1.size() ? nbins : s1[g];
                P1.dsel[g] = !splits_further(b0, b1);
            }
        }
        Blob A{stage, capA};
        const Placed pl = place(P1, A);
        if (A.overflow()) return AHS_ERR_CUDA;
        e = upload(A, 0);
        if (e == cudaSuccess) e = launch(P1, pl, 0);
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    *levels_out = 1;

    // Level 2: every multi-bin run above a CTA's capacity, temporary -> output;
    // runs that fit a CTA (and single heavy bins) leave here.  Only what the
    // launch needs is planned before it; the final buckets are listed while
    // the pass runs.
    std::vector<SegRange> large;
    Pass Pd, Pr;
    Pd.digit = true;
    {
        // Probability that two random keys of one level-1 bucket share a bin.
        double d2 = 0.0;
        for (size_t g = 0; g <= s1.size(); ++g) {
            const uint32_t b0 = g == 0 ? 0u : s1[g - 1], b1 = g == s1.size() ? nbins : s1[g];
            const unsigned long long cg = binpos[b1] - binpos[b0];
            if (cg == 0) continue;
            double sq = 0.0;
            for (uint32_t b = b0; b < b1; ++b) sq += (double)hist[b] * (double)hist[b];
            d2 += sq / (double)cg;
        }
        d2 /= (double)n;
        Pd.slots = Pr.slots = d2 >= kGroupCollide ? kSlotsGroup : runs_slots;
    }
    Pd.dshift = shift;
    Pd.src = Pr.src = ktmp;
    Pd.dst = Pr.dst = kout;
    const uint32_t span_bins = msd || shift >= 16 ? 1u : 1u << (16 - shift);
    // Per level-1 run: -1 if it is final, else (pass, index) of its level-2 segment.
    std::vector<int32_t> split2(s1.size() + 1, -1);
    for (size_t g = 0; g <= s1.size(); ++g) {
        const uint32_t b0 = g == 0 ? 0u : s1[g - 1], b1 = g == s1.size() ? nbins : s1[g];
        const unsigned long long sz = binpos[b1] - binpos[b0];
        if (!splits_further(b0, b1)) continue;
        std::vector<uint32_t> st2 = group_bins(hist, b0, b1, kBucketCap / 2,
                                               std::max<uint32_t>(span_bins, (b1 - b0 + 255) / 256));
        bool single = (b1 - b0 <= 256) && st2.size() == b1 - b0 - 1;
        for (size_t j = 0; single && j < st2.size(); ++j) single = st2[j] == b0 + 1 + j;
        Pass& P = single ? Pd : Pr;
        split2[g] = (int32_t)((single ? 0u : 1u << 30) | (uint32_t)P.segs.size());
        P.segs.push_back({binpos[b0], (uint32_t)sz, (unsigned long long)b0});
        P.starts.push_back(std::move(st2));
        P.ends.push_back(b1);
    }
    {
        Blob B{stage + capA, capB};
        Placed pd{}, pr{};
        if (!Pd.segs.empty()) pd = place(Pd, B);
        if (!Pr.segs.empty()) pr = place(Pr, B);
        if (B.overflow()) return AHS_ERR_CUDA;
        if (B.used) {
            e = upload(B, capA);
            if (e == cudaSuccess && !Pd.segs.empty()) e = launch(Pd, pd, capA);
            if (e == cudaSuccess && !Pr.segs.empty()) e = launch(Pr, pr, capA);
            if (e != cudaSuccess) return cuda_status(ctx, e);
            *levels_out = 2;
        }
    }
    // Final buckets, into the class regions of the third window: level-1 runs
    // that are final and the sub-buckets of the level-2 segments, all in the
    // output by now and sorted there in place.
    ClassLists cl;
    cl.cap = class_cap;
    for (int k = 0; k < kBucketClasses; ++k)
        cl.region[k] = reinterpret_cast<FinalBucket*>(stage + capA + capB + k * class_bytes);
    for (size_t g = 0; g <= s1.size(); ++g) {
        const uint32_t b0 = g == 0 ? 0u : s1[g - 1], b1 = g == s1.size() ? nbins : s1[g];
        const unsigned long long sz = binpos[b1] - binpos[b0];
        if (sz == 0) continue;
        if (split2[g] < 0) {
            // Out of place, level 1 wrote the run to the output (sorted there
            // in place); in place, it is in the temporary buffer.
            const uint8_t where = inplace ? 0 : 1;
            if (sz <= kBucketCap && sz > 1)
                cl.add(final_bucket_bounded(binpos[b0], (uint32_t)sz, where, bin_lo(b0), range_bits(b0, b1)));
            else if (inplace)
                cl.add(final_bucket(binpos[b0], (uint32_t)sz, 0, false));   // copy out
            if (sz > kBucketCap) large.push_back({binpos[b0], (uint32_t)sz, 0ull});
            continue;
        }
        const Pass& P = (split2[g] >> 30) ? Pr : Pd;
        const std::vector<uint32_t>& st2 = P.starts[split2[g] & ((1 << 30) - 1)];
        uint32_t lo_b = b0;
        for (size_t j = 0; j <= st2.size(); ++j) {
            const uint32_t hi_b = j == st2.size() ? b1 : st2[j];
            const unsigned long long ssz = binpos[hi_b] - binpos[lo_b];
            if (ssz >= 2) {
                if (ssz <= kBucketCap)
                    cl.add(final_bucket_bounded(binpos[lo_b], (uint32_t)ssz, 1, bin_lo(lo_b),
                                                range_bits(lo_b, hi_b)));
                else
                    large.push_back({binpos[lo_b], (uint32_t)ssz, 0ull});
            }
            lo_b = hi_b;
        }
    }
    if (cl.overflow) return AHS_ERR_CUDA;
    {
        const FinalBucket* lists[kBucketClasses];
        for (int k = 0; k < kBucketClasses && e == cudaSuccess; ++k) {
            const size_t off = capA + capB + k * class_bytes;
            lists[k] = reinterpret_cast<const FinalBucket*>(aux + off);
            if (cl.count[k])
                e = launch_transfer(aux + off, stage + off, cl.count[k] * sizeof(FinalBucket), st);
        }
        if (e == cudaSuccess)
            e = launch_bucket_finish(lists, cl.count, cl.keys, ktmp, kout, kin, kout, nullptr, nullptr,
                                     nullptr, nullptr, KeyDesc{(uint32_t)sizeof(K), (uint64_t)flip}, st);
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    *buckets_out = cl.sorted;
    if (large.empty()) return AHS_OK;
    // The pinned staging still feeds the copies above: wait before reusing it.
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    return finish_large<K>(ctx, large, kout, n, flip, scratch, st, levels_out, buckets_out);
}

// The batched general class, keys only, with coarse histograms: see
// run_batched_general_hist.  The pass's lists are planned and launched
// first; the final buckets are listed while it runs.  Consecutive digit
// buckets are merged into sort units of up to kUnitKeys keys (a small
// segment would otherwise leave 256 buckets of a few keys each).
constexpr uint32_t kUnitKeys = 4096;

template <typename K>
ahs_status batched_hist_t(ahs_ctx* ctx, const K* kin, K* kout, uint64_t n_total,
                          const std::vector<HistRange>& segs, const std::vector<SegRange>& extra,
                          K flip, void* scratch, cudaStream_t st, uint32_t* levels_out,
                          uint32_t* buckets_out) {
    cudaError_t e = set_attrs<K, false>();
    if (e != cudaSuccess) return cuda_status(ctx, e);
    constexpr uint32_t TK = FastCfg<K>::kTileKeys;
    constexpr uint32_t CS = cursor_stride<kDigit>();
    // One launch per slot mode: segments whose warps often share a bucket
    // (few descents) take the aggregated slot atomics, reversed runs the
    // run checks, keys in random order one atomic per key.
    constexpr int kVariants = 3;
    constexpr int kSlotsOf[kVariants] = {kSlotsPlain, kSlotsGroup, kSlotsRuns};
    auto variant = [](const HistRange& h) { return h.group ? 1 : (h.runs ? 2 : 0); };
    size_t n_seg[kVariants] = {0, 0, 0}, n_til[kVariants] = {0, 0, 0};
    for (const HistRange& h : segs) {
        const int v = variant(h);
        ++n_seg[v];
        n_til[v] += ceil_div(h.r.size, TK);
    }
    size_t b_seg[kVariants], b_til[kVariants], b_cur[kVariants], at[kVariants][3], total = 0;
    for (int v = 0; v < kVariants; ++v) {
        b_seg[v] = a256(n_seg[v] * sizeof(SegDesc));
        b_til[v] = a256(n_til[v] * sizeof(TileDesc));
        b_cur[v] = a256(n_seg[v] * CS * 4);
        at[v][0] = total;
        at[v][1] = total + b_seg[v];
        at[v][2] = total + b_seg[v] + b_til[v];
        total += b_seg[v] + b_til[v] + b_cur[v];
    }
    ahs_status rc = ensure_aux(ctx, total);
    if (rc == AHS_OK) rc = ensure_stage(ctx, total);
    if (rc != AHS_OK) return rc;
    char* aux = static_cast<char*>(ctx->aux);
    char* hs = static_cast<char*>(ctx->h_stage);
    // Each segment's launch, index and first tile (a running count), then
    // the lists filled by segment in parallel.
    const size_t ns = segs.size();
    std::vector<uint32_t> q_of(ns), t_of(ns);
    {
        size_t q_seg[kVariants] = {0, 0, 0}, q_til[kVariants] = {0, 0, 0};
        for (size_t i = 0; i < ns; ++i) {
            const int v = variant(segs[i]);
            q_of[i] = (uint32_t)q_seg[v]++;
            t_of[i] = (uint32_t)q_til[v];
            q_til[v] += ceil_div(segs[i].r.size, TK);
        }
    }
    std::vector<uint8_t> bad(chunks_for(ns, 512), 0);
    parallel_chunks(ns, bad.size(), [&](size_t c, size_t lo, size_t hi) {
        for (size_t i = lo; i < hi; ++i) {
            const HistRange& h = segs[i];
            const int v = variant(h);
            SegDesc d{};
            d.begin = h.r.begin;
            d.size = h.r.size;
            d.min_ord = h.r.min_ord;
            d.dshift = h.shift + 8 + 1;   // digit = bin >> 8 (a bin has <= 16 bits)
            d.first_tile = t_of[i];
            const uint32_t q = q_of[i];
            TileDesc* td = reinterpret_cast<TileDesc*>(hs + at[v][1]) + t_of[i];
            for (uint32_t o = 0, k = 0; o < d.size; o += TK, ++k)
                td[k] = {d.begin + o, std::min(TK, d.size - o), q};
            reinterpret_cast<SegDesc*>(hs + at[v][0])[q] = d;
            // Cursors: each digit bucket's first position in the segment.
            uint32_t* cur = reinterpret_cast<uint32_t*>(hs + at[v][2]) + (size_t)q * CS;
            uint32_t pos = 0;
            for (uint32_t j = 0; j < kCoarseBuckets; ++j) {
                cur[j] = pos;
                pos += h.coarse[j];
            }
            if (pos != h.r.size) bad[c] = 1;   // the histogram must describe the segment
        }
    });
    for (uint8_t b : bad)
        if (b) return AHS_ERR_CUDA;
    e = launch_transfer(aux, hs, total, st);
    for (int v = 0; v < kVariants && e == cudaSuccess; ++v) {
        if (!n_seg[v]) continue;
        const uint32_t nt = (uint32_t)n_til[v];
        const uint32_t grid = (uint32_t)std::min<uint64_t>(nt, 2ull * (uint64_t)ctx->sms);
        uint64_t keys = 0;
        for (const HistRange& h : segs) keys += variant(h) == v ? h.r.size : 0;
        TraceScope ts("batch_digit_scatter", keys, st);
        const SegDesc* ds = reinterpret_cast<const SegDesc*>(aux + at[v][0]);
        const TileDesc* dt = reinterpret_cast<const TileDesc*>(aux + at[v][1]);
        uint32_t* dc = reinterpret_cast<uint32_t*>(aux + at[v][2]);
        e = launch_scatter_keys<K, kDigit>(kSlotsOf[v], grid, sizeof(FastSmem<K>), st, kin, kout, dt, ds,
                                           (uint32_t)n_seg[v], nt, nullptr, nullptr, flip, 0u, dc,
                                           ctx->d_err);
    }
    if (e != cudaSuccess) return cuda_status(ctx, e);
    // While the pass runs: the sort units (runs of consecutive digit buckets
    // of at most kUnitKeys keys; a single bucket up to a CTA's capacity) and
    // the buckets heavier than a CTA.
    const size_t nch = chunks_for(ns, 512);
    std::vector<FinalSet> finals(nch + 1);
    std::vector<std::vector<SegRange>> large_of(nch);
    for (const SegRange& x : extra) finals[nch].add(final_bucket(x.begin, x.size, 2, x.size > 1));
    parallel_chunks(ns, nch, [&](size_t c, size_t lo, size_t hi) {
        FinalSet& fs = finals[c];
        uint64_t keys = 0;
        for (size_t i = lo; i < hi; ++i) keys += segs[i].r.size;
        fs.reserve(keys / (kUnitKeys / 2) + 64);
        for (size_t i = lo; i < hi; ++i) {
            const HistRange& h = segs[i];
            const uint32_t sh = h.shift + 8;
            uint32_t pos = 0, j0 = 0, usz = 0;
            auto close = [&](uint32_t j1) {   // unit = digit buckets [j0, j1)
                if (usz >= 2) {
                    const unsigned long long lo_ord =
                        (unsigned long long)(K)(h.r.min_ord + ((unsigned long long)j0 << sh));
                    fs.add(final_bucket_bounded(h.r.begin + pos - usz, usz, 1, lo_ord,
                                                bitlen64((((unsigned long long)(j1 - j0)) << sh) - 1)));
                }
                j0 = j1;
                usz = 0;
            };
            for (uint32_t j = 0; j < kCoarseBuckets; ++j) {
                const uint32_t sz = h.coarse[j];
                if (sz > kBucketCap) {
                    close(j);
                    large_of[c].push_back({h.r.begin + pos, sz, 0ull});
                    pos += sz;
                    j0 = j + 1;
                    continue;
                }
                if (usz && usz + sz > kUnitKeys) close(j);
                usz += sz;
                pos += sz;
            }
            close(kCoarseBuckets);
        }
    });
    std::vector<SegRange> large;
    for (auto& v : large_of) large.insert(large.end(), v.begin(), v.end());
    // The pass's lists came from the staging buffer: wait before reusing it.
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    *levels_out = 1;
    rc = finish_buckets_sets(ctx, finals.data(), finals.size(), scratch, kout, kin, nullptr, nullptr,
                             nullptr, KeyDesc{(uint32_t)sizeof(K), (uint64_t)flip}, st, buckets_out);
    if (rc != AHS_OK || large.empty()) return rc;
    uint32_t lv = 0, bk = 0;
    rc = general_t<K, false>(ctx, kout, kout, nullptr, nullptr, n_total, large, {}, flip, scratch, st,
                             &lv, &bk);
    *levels_out += lv;
    *buckets_out += bk;
    return rc;
}

}  // namespace

size_t samplesort_scratch_bytes(uint64_t n, uint32_t key_bytes, bool has_vals) {
    return segsort_scratch_bytes(n, 1, key_bytes, has_vals);
}

size_t segsort_scratch_bytes(uint64_t n_total, uint64_t, uint32_t key_bytes, bool vals) {
    return a256(n_total * key_bytes) + (vals ? a256(n_total * 4) : 0) + 256;
}

ahs_status run_segmented_general(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                                 uint32_t* vout, uint64_t n_total, const std::vector<SegRange>& segs,
                                 const std::vector<SegRange>& extra, KeyDesc kd, void* scratch,
                                 cudaStream_t st, uint32_t* levels_out, uint32_t* buckets_out) {
    *levels_out = 0;
    *buckets_out = 0;
    const bool v = vin != nullptr;
    if (kd.bytes == 4) {
        const uint32_t f = (uint32_t)kd.flip;
        return v ? general_t<uint32_t, true>(ctx, (const uint32_t*)kin, (uint32_t*)kout, vin, vout, n_total, segs, extra, f, scratch, st, levels_out, buckets_out)
                 : general_t<uint32_t, false>(ctx, (const uint32_t*)kin, (uint32_t*)kout, nullptr, nullptr, n_total, segs, extra, f, scratch, st, levels_out, buckets_out);
    }
    return v ? general_t<uint64_t, true>(ctx, (const uint64_t*)kin, (uint64_t*)kout, vin, vout, n_total, segs, extra, kd.flip, scratch, st, levels_out, buckets_out)
             : general_t<uint64_t, false>(ctx, (const uint64_t*)kin, (uint64_t*)kout, nullptr, nullptr, n_total, segs, extra, kd.flip, scratch, st, levels_out, buckets_out);
}

ahs_status run_batched_general_hist(ahs_ctx* ctx, const void* kin, void* kout, uint64_t n_total,
                                    const std::vector<HistRange>& segs,
                                    const std::vector<SegRange>& extra, KeyDesc kd, void* scratch,
                                    cudaStream_t st, uint32_t* levels_out, uint32_t* buckets_out) {
    *levels_out = 0;
    *buckets_out = 0;
    if (kd.bytes == 4)
        return batched_hist_t<uint32_t>(ctx, (const uint32_t*)kin, (uint32_t*)kout, n_total, segs, extra,
                                        (uint32_t)kd.flip, scratch, st, levels_out, buckets_out);
    return batched_hist_t<uint64_t>(ctx, (const uint64_t*)kin, (uint64_t*)kout, n_total, segs, extra,
                                    kd.flip, scratch, st, levels_out, buckets_out);
}

ahs_status run_segmented_radix(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                               uint32_t* vout, uint64_t n_total, const std::vector<SegRange>& segs,
                               uint32_t passes, KeyDesc kd, void* scratch, cudaStream_t st) {
    const bool v = vin != nullptr;
    if (kd.bytes == 4) {
        const uint32_t f = (uint32_t)kd.flip;
        return v ? radix_segs_t<uint32_t, true>(ctx, (const uint32_t*)kin, (uint32_t*)kout, vin, vout, n_total, segs, passes, f, scratch, st)
                 : radix_segs_t<uint32_t, false>(ctx, (const uint32_t*)kin, (uint32_t*)kout, nullptr, nullptr, n_total, segs, passes, f, scratch, st);
    }
    return v ? radix_segs_t<uint64_t, true>(ctx, (const uint64_t*)kin, (uint64_t*)kout, vin, vout, n_total, segs, passes, kd.flip, scratch, st)
             : radix_segs_t<uint64_t, false>(ctx, (const uint64_t*)kin, (uint64_t*)kout, nullptr, nullptr, n_total, segs, passes, kd.flip, scratch, st);
}

ahs_status run_small_segments(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                              uint32_t* vout, const std::vector<SegRange>& sort_segs,
                              const std::vector<SegRange>& copy_segs, KeyDesc kd, cudaStream_t st) {
    FinalSet finals;
    finals.reserve(sort_segs.size() + copy_segs.size());
    for (const SegRange& x : sort_segs) finals.add(final_bucket(x.begin, x.size, 2, x.size > 1));
    for (const SegRange& x : copy_segs) finals.add(final_bucket(x.begin, x.size, 2, false));
    // No temporary buffer is involved: every bucket reads kin and writes kout.
    return finish_buckets(ctx, finals, kout, kout, kin, vout, vout, vin, kd, st, nullptr);
}

ahs_status run_msd_radix(ahs_ctx* ctx, const void* kin, void* kout, uint64_t n, KeyDesc kd,
                         uint64_t min_ord, const HistView& hist,
                         uint32_t shift, uint32_t group, void* scratch, cudaStream_t st,
                         uint32_t* levels_out, uint32_t* buckets_out) {
    *levels_out = 0;
    *buckets_out = 0;
    if (n > 0xffffffffull || hist.empty() || hist.size() > kMaxBins) return AHS_ERR_INVALID_ARG;
    if (kd.bytes == 4)
        return keys_hist_t<uint32_t>(ctx, (const uint32_t*)kin, (uint32_t*)kout, n, (uint32_t)kd.flip,
                                     (uint32_t)min_ord, hist, shift, true, group, scratch, st,
                                     levels_out, buckets_out);
    return keys_hist_t<uint64_t>(ctx, (const uint64_t*)kin, (uint64_t*)kout, n, kd.flip, min_ord,
                                 hist, shift, true, group, scratch, st, levels_out, buckets_out);
}

ahs_status run_samplesort(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                          uint32_t* vout, uint64_t n, KeyDesc kd, void* scratch, cudaStream_t st,
                          uint32_t* levels_out, uint32_t* buckets_out,
                          const HistView* hist, uint64_t min_ord,
                          uint32_t shift, uint32_t group) {
    *levels_out = 0;
    *buckets_out = 0;
    if (n <= kBucketCap) {
        *buckets_out = 1;
        return cuda_status(ctx, launch_blocksort_single(kin, kout, vin, vout, n, kd, st));
    }
    if (!vin && hist && hist->size() > 256 && n <= 0xffffffffull) {
        if (kd.bytes == 4)
            return keys_hist_t<uint32_t>(ctx, (const uint32_t*)kin, (uint32_t*)kout, n,
                                         (uint32_t)kd.flip, (uint32_t)min_ord, *hist, shift, false,
                                         group, scratch, st, levels_out, buckets_out);
        return keys_hist_t<uint64_t>(ctx, (const uint64_t*)kin, (uint64_t*)kout, n, kd.flip,
                                     min_ord, *hist, shift, false, group, scratch, st, levels_out,
                                     buckets_out);
    }
    std::vector<SegRange> segs{{0ull, (uint32_t)n, 0ull}};
    return run_segmented_general(ctx, kin, kout, vin, vout, n, segs, {}, kd, scratch, st,
                                 levels_out, buckets_out);
}

}  // namespace ahs
