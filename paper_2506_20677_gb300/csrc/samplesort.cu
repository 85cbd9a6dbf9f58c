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
#include <algorithm>
#include <cstring>
#include <vector>

#include "blocksort.cuh"
#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "samplesort.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kThreads = 512;
constexpr int kIpt = 16;
constexpr uint32_t kTile = kThreads * kIpt;     // keys per partition tile
constexpr uint32_t kMaxSplit = 255;             // distinct splitters per segment
constexpr uint32_t kCols = 512;                 // 2 * 255 + 1 buckets, padded
constexpr uint32_t kOversample = 32;
constexpr uint32_t kSamples = (kMaxSplit + 1) * kOversample;   // 8,192
constexpr uint32_t kChunkTiles = 32;
constexpr uint32_t kMaxLevels = 16;

struct SegDesc {
    unsigned long long begin;
    uint32_t size;
    uint32_t first_chunk;
    uint32_t nchunks;
    uint32_t pad[3];
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
static_assert(sizeof(SegDesc) == 32 && sizeof(TileDesc) == 16 && sizeof(ChunkDesc) == 16, "layout");

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
    // SplitMix64 output function (Steele, Lea & Flood 2014).
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Bucket of ord value o among m distinct ascending splitters sp:
// 2j for sp[j-1] < o < sp[j], 2j+1 for o == sp[j].
template <typename K>
__device__ __forceinline__ uint32_t classify(const K* sp, uint32_t m, K o) {
    uint32_t lo = 0, len = m;
    while (len > 0) {
        const uint32_t half = len >> 1;
        if (sp[lo + half] < o) {
            lo += half + 1;
            len -= half + 1;
        } else {
            len = half;
        }
    }
    return (lo < m && sp[lo] == o) ? 2 * lo + 1 : 2 * lo;
}

// One CTA per segment: draw kSamples keys at hashed positions, sort them in
// shared memory, keep the distinct values among the 255 quantiles.
template <typename K>
__global__ void __launch_bounds__(kThreads)
ss_sample(const K* __restrict__ src, const SegDesc* __restrict__ segs, uint32_t level, K flip,
          K* __restrict__ splitters, uint32_t* __restrict__ nsplit) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    using Smem = BlockSortSmem<K, false, kThreads, kIpt>;
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);
    const SegDesc sg = segs[blockIdx.x];
    const unsigned long long salt =
        ((unsigned long long)level << 48) ^ ((unsigned long long)blockIdx.x << 20);
    for (uint32_t i = threadIdx.x; i < kSamples; i += kThreads) {
        const unsigned long long h = mix64((salt + i + 1) * 0x9E3779B97F4A7C15ull);
        const unsigned long long pos = __umul64hi(h, (unsigned long long)sg.size);
        S.keys[i] = src[sg.begin + pos];
    }
    __syncthreads();
    block_sort<K, false, kThreads, kIpt>(S.keys, S.keys, nullptr, nullptr, kSamples, flip, S);
    __syncthreads();
    uint32_t keep = 0;
    K cand = 0;
    if (threadIdx.x < kMaxSplit) {
        cand = S.keys[(threadIdx.x + 1) * kOversample - 1] ^ flip;
        keep = (threadIdx.x == 0 || cand != (K)(S.keys[threadIdx.x * kOversample - 1] ^ flip)) ? 1u : 0u;
    }
    uint32_t total;
    const uint32_t at = block_exclusive_scan<kThreads>(keep, S.scan, &total);
    if (keep) splitters[(size_t)blockIdx.x * (kMaxSplit + 1) + at] = cand;
    if (threadIdx.x == 0) nsplit[blockIdx.x] = total;
}

// Per tile: bucket histogram.
template <typename K>
__global__ void __launch_bounds__(kThreads)
ss_count(const K* __restrict__ src, const TileDesc* __restrict__ tiles, const K* __restrict__ splitters,
         const uint32_t* __restrict__ nsplit, K flip, uint32_t* __restrict__ counts) {
    __shared__ K sp[kMaxSplit + 1];
    __shared__ uint32_t hist[kCols];
    const TileDesc t = tiles[blockIdx.x];
    const uint32_t m = nsplit[t.seg];
    for (uint32_t i = threadIdx.x; i < m; i += kThreads) sp[i] = splitters[(size_t)t.seg * (kMaxSplit + 1) + i];
    for (uint32_t i = threadIdx.x; i < kCols; i += kThreads) hist[i] = 0;
    __syncthreads();
    const K* p = src + t.begin;
#pragma unroll 4
    for (uint32_t i = threadIdx.x; i < t.size; i += kThreads) {
        const uint32_t b = classify(sp, m, (K)(p[i] ^ flip));
        if (AHS_DCHECK(b < kCols, "count bucket", b)) atomicAdd(&hist[b], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kCols; i += kThreads)
        counts[(size_t)blockIdx.x * kCols + i] = hist[i];
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
    seg_tot[(size_t)blockIdx.x * kCols + j] = run;
    seg_base[(size_t)blockIdx.x * kCols + j] = base;
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
    K sp[kMaxSplit + 1];
    uint32_t warp_hist[kThreads / 32][kCols];
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
template <typename K, bool VALS>
__global__ void __launch_bounds__(kThreads)
ss_scatter(const K* __restrict__ src, K* __restrict__ dst, const uint32_t* __restrict__ vsrc,
           uint32_t* __restrict__ vdst, const TileDesc* __restrict__ tiles,
           const SegDesc* __restrict__ segs, const K* __restrict__ splitters,
           const uint32_t* __restrict__ nsplit, K flip, const uint32_t* __restrict__ offs) {
    constexpr int W = kThreads / 32;
    constexpr int WARP_ITEMS = 32 * kIpt;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    ScatterSmem<K, VALS>& S = *reinterpret_cast<ScatterSmem<K, VALS>*>(smem_raw);
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const TileDesc t = tiles[blockIdx.x];
    const uint32_t m = nsplit[t.seg];
    for (uint32_t i = tid; i < m; i += kThreads) S.sp[i] = splitters[(size_t)t.seg * (kMaxSplit + 1) + i];
    for (uint32_t i = tid; i < W * kCols; i += kThreads) (&S.warp_hist[0][0])[i] = 0;
    __syncthreads();

    K key[kIpt];
    uint32_t b[kIpt], rank[kIpt];
    const K* p = src + t.begin;
    const uint32_t wbase = warp * WARP_ITEMS;
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        const uint32_t q = wbase + 32 * i + lane;
        if (q < t.size) {
            key[i] = p[q];
            b[i] = classify(S.sp, m, (K)(key[i] ^ flip));
        } else {
            key[i] = 0;
            b[i] = kCols;
        }
    }
    uint32_t* wh = S.warp_hist[warp];
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        const uint32_t peers = __match_any_sync(AHS_FULL_MASK, b[i]);
        const uint32_t leader = __ffs(peers) - 1;
        uint32_t old = 0;
        if (lane == leader && b[i] < kCols) old = atomicAdd(&wh[b[i]], __popc(peers));
        old = __shfl_sync(AHS_FULL_MASK, old, leader);
        rank[i] = old + __popc(peers & lt);
    }
    __syncthreads();
    {
        const uint32_t j = tid;   // kThreads == kCols
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
#pragma unroll
    for (int i = 0; i < kIpt; ++i) {
        if (b[i] < kCols) {
            const uint32_t lp = S.tile_start[b[i]] + S.warp_hist[warp][b[i]] + rank[i];
            if (!AHS_DCHECK(lp < t.size, "scatter stage", lp)) continue;
            S.keys[lp] = key[i];
            S.bid[lp] = (uint16_t)b[i];
        }
    }
    if constexpr (VALS) {
        const uint32_t* vp = vsrc + t.begin;
#pragma unroll
        for (int i = 0; i < kIpt; ++i) {
            if (b[i] < kCols) {
                const uint32_t lp = S.tile_start[b[i]] + S.warp_hist[warp][b[i]] + rank[i];
                if (AHS_DCHECK(lp < t.size, "scatter vstage", lp)) S.vals[lp] = vp[wbase + 32 * i + lane];
            }
        }
    }
    __syncthreads();
    const SegDesc sg = segs[t.seg];
    K* out = dst + sg.begin;
    uint32_t* vout = VALS ? vdst + sg.begin : nullptr;
    for (uint32_t j = tid; j < t.size; j += kThreads) {
        const uint32_t gp = S.gbase[S.bid[j]] + j;
        if (gp >= sg.size) continue;   // cannot happen with consistent offsets; never write outside
        out[gp] = S.keys[j];
        if constexpr (VALS) vout[gp] = S.vals[j];
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carve {
    void* ktmp;
    uint32_t* vtmp;
    uint32_t* counts;
    uint32_t* chunk_sum;
    uint32_t* seg_tot;
    uint32_t* seg_base;
    void* splitters;
    uint32_t* nsplit;
    SegDesc* segs;
    TileDesc* tiles;
    ChunkDesc* chunks;
};

struct Bounds {
    uint64_t segs, tiles, chunks;
};

Bounds bounds_for(uint64_t n) {
    Bounds b;
    b.segs = n / (kBucketCap + 1) + 2;
    b.tiles = 2 * (n / kTile) + b.segs + 2;
    b.chunks = b.tiles / kChunkTiles + b.segs + 2;
    return b;
}

size_t carve_bytes(uint64_t n, uint32_t kb, bool vals) {
    const Bounds b = bounds_for(n);
    return a256(n * kb) + (vals ? a256(n * 4) : 0) + a256(b.tiles * kCols * 4) +
           a256(b.chunks * kCols * 4) + 2 * a256(b.segs * kCols * 4) +
           a256(b.segs * (kMaxSplit + 1) * kb) + a256(b.segs * 4) + a256(b.segs * sizeof(SegDesc)) +
           a256(b.tiles * sizeof(TileDesc)) + a256(b.chunks * sizeof(ChunkDesc)) + 256;
}

Carve carve(void* base, uint64_t n, uint32_t kb, bool vals) {
    const Bounds b = bounds_for(n);
    Carve c{};
    char* p = static_cast<char*>(base);
    auto take = [&](size_t bytes) { char* r = p; p += a256(bytes); return r; };
    c.ktmp = take(n * kb);
    c.vtmp = vals ? reinterpret_cast<uint32_t*>(take(n * 4)) : nullptr;
    c.counts = reinterpret_cast<uint32_t*>(take(b.tiles * kCols * 4));
    c.chunk_sum = reinterpret_cast<uint32_t*>(take(b.chunks * kCols * 4));
    c.seg_tot = reinterpret_cast<uint32_t*>(take(b.segs * kCols * 4));
    c.seg_base = reinterpret_cast<uint32_t*>(take(b.segs * kCols * 4));
    c.splitters = take(b.segs * (kMaxSplit + 1) * kb);
    c.nsplit = reinterpret_cast<uint32_t*>(take(b.segs * 4));
    c.segs = reinterpret_cast<SegDesc*>(take(b.segs * sizeof(SegDesc)));
    c.tiles = reinterpret_cast<TileDesc*>(take(b.tiles * sizeof(TileDesc)));
    c.chunks = reinterpret_cast<ChunkDesc*>(take(b.chunks * sizeof(ChunkDesc)));
    return c;
}

template <typename F>
cudaError_t set_smem(F fn, size_t bytes) {
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

struct OpenSeg {
    unsigned long long begin;
    uint32_t size;
};

template <typename K, bool VALS>
ahs_status samplesort_t(ahs_ctx* ctx, const K* kin, K* kout, const uint32_t* vin, uint32_t* vout,
                        uint64_t n, K flip, void* scratch, cudaStream_t st, uint32_t* levels_out,
                        uint32_t* buckets_out) {
    const Carve c = carve(scratch, n, sizeof(K), VALS);
    K* ktmp = static_cast<K*>(c.ktmp);
    cudaError_t e;
    e = set_smem(ss_sample<K>, sizeof(BlockSortSmem<K, false, kThreads, kIpt>));
    if (e == cudaSuccess) e = set_smem(ss_scatter<K, VALS>, sizeof(ScatterSmem<K, VALS>));
    if (e != cudaSuccess) return cuda_status(ctx, e);

    std::vector<OpenSeg> open{{0ull, (uint32_t)n}};
    std::vector<FinalBucket> finals;
    std::vector<SegDesc> hsegs;
    std::vector<TileDesc> htiles;
    std::vector<ChunkDesc> hchunks;
    uint32_t level = 0;
    while (!open.empty()) {
        if (level >= kMaxLevels) return AHS_ERR_UNIMPLEMENTED;
        ++level;
        // Level 1 reads the input; odd levels write the temporary buffer, even
        // levels the output, so a level never overwrites its own source.
        const K* src = level == 1 ? kin : (level % 2 == 0 ? ktmp : kout);
        const uint32_t* vsrc = level == 1 ? vin : (level % 2 == 0 ? c.vtmp : vout);
        K* dst = (level % 2 == 1) ? ktmp : kout;
        uint32_t* vdst = (level % 2 == 1) ? c.vtmp : vout;
        const uint8_t where = (level % 2 == 1) ? 0 : 1;

        hsegs.clear();
        htiles.clear();
        hchunks.clear();
        for (uint32_t s = 0; s < open.size(); ++s) {
            SegDesc sd{};
            sd.begin = open[s].begin;
            sd.size = open[s].size;
            sd.first_chunk = (uint32_t)hchunks.size();
            const uint32_t nt = (uint32_t)ceil_div(sd.size, kTile);
            const uint32_t t0 = (uint32_t)htiles.size();
            for (uint32_t t = 0; t < nt; ++t) {
                const uint32_t off = t * kTile;
                htiles.push_back({sd.begin + off, std::min(kTile, sd.size - off), s});
            }
            for (uint32_t t = 0; t < nt; t += kChunkTiles)
                hchunks.push_back({t0 + t, std::min(kChunkTiles, nt - t), s, 0});
            sd.nchunks = (uint32_t)hchunks.size() - sd.first_chunk;
            hsegs.push_back(sd);
        }
        const size_t bseg = hsegs.size() * sizeof(SegDesc), btile = htiles.size() * sizeof(TileDesc),
                     bchunk = hchunks.size() * sizeof(ChunkDesc);
        const size_t bread = hsegs.size() * kCols * 4;
        ahs_status rc = ensure_stage(ctx, std::max(bseg + btile + bchunk, 2 * bread));
        if (rc != AHS_OK) return rc;
        char* hs = static_cast<char*>(ctx->h_stage);
        std::memcpy(hs, hsegs.data(), bseg);
        std::memcpy(hs + bseg, htiles.data(), btile);
        std::memcpy(hs + bseg + btile, hchunks.data(), bchunk);
        e = cudaMemcpyAsync(c.segs, hs, bseg, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(c.tiles, hs + bseg, btile, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c.chunks, hs + bseg + btile, bchunk, cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) return cuda_status(ctx, e);

        K* spl = static_cast<K*>(c.splitters);
        const uint32_t ns = (uint32_t)hsegs.size(), nt = (uint32_t)htiles.size(),
                       nc = (uint32_t)hchunks.size();
        uint64_t level_keys = 0;
        for (const SegDesc& sd : hsegs) level_keys += sd.size;
        {
            TraceScope ts("sample_splitters", ns, st);
            ss_sample<K><<<ns, kThreads, sizeof(BlockSortSmem<K, false, kThreads, kIpt>), st>>>(
                src, c.segs, level, flip, spl, c.nsplit);
        }
        {
            TraceScope ts("sample_count", level_keys, st);
            ss_count<K><<<nt, kThreads, 0, st>>>(src, c.tiles, spl, c.nsplit, flip, c.counts);
        }
        {
            TraceScope ts("sample_scan", nt, st);
            ss_scan_a<<<nc, kCols, 0, st>>>(c.counts, c.chunks, c.chunk_sum);
            ss_scan_b<<<ns, kCols, 0, st>>>(c.chunk_sum, c.segs, c.seg_tot, c.seg_base);
            ss_scan_c<<<nc, kCols, 0, st>>>(c.counts, c.chunks, c.chunk_sum);
        }
        {
            TraceScope ts("sample_scatter", level_keys, st);
            ss_scatter<K, VALS><<<nt, kThreads, sizeof(ScatterSmem<K, VALS>), st>>>(
                src, dst, vsrc, vdst, c.tiles, c.segs, spl, c.nsplit, flip, c.counts);
        }
        e = cudaGetLastError();
        // The stage buffer is reused for the readback: wait for the uploads.
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs, c.seg_tot, bread, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(hs + bread, c.seg_base, bread, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(ctx, e);

        const uint32_t* tot = reinterpret_cast<const uint32_t*>(hs);
        const uint32_t* base = reinterpret_cast<const uint32_t*>(hs + bread);
        std::vector<OpenSeg> next;
        for (uint32_t s = 0; s < ns; ++s) {
            for (uint32_t j = 0; j < kCols; ++j) {
                const uint32_t sz = tot[(size_t)s * kCols + j];
                if (sz == 0) continue;
                const unsigned long long b0 = hsegs[s].begin + base[(size_t)s * kCols + j];
                const bool equal = (j & 1u) != 0;
                if (equal || sz == 1) {
                    if (where == 0) finals.push_back({b0, sz, where, 0, 0});   // copy to output
                } else if (sz <= kBucketCap) {
                    finals.push_back({b0, sz, where, 1, 0});
                } else {
                    next.push_back({b0, sz});
                }
            }
        }
        open.swap(next);
    }

    // Bucket sorts, one launch per size class.
    std::vector<FinalBucket> cls[3];
    uint32_t sorted_buckets = 0;
    for (const FinalBucket& f : finals) {
        cls[f.sort ? bucket_class(f.size) : 0].push_back(f);
        sorted_buckets += f.sort;
    }
    const size_t nf = finals.size();
    if (nf) {
        ahs_status rc = ensure_aux(ctx, nf * sizeof(FinalBucket));
        if (rc == AHS_OK) rc = ensure_stage(ctx, nf * sizeof(FinalBucket));
        if (rc != AHS_OK) return rc;
        FinalBucket* hf = static_cast<FinalBucket*>(ctx->h_stage);
        FinalBucket* df = static_cast<FinalBucket*>(ctx->aux);
        const FinalBucket* lists[3];
        uint32_t counts[3];
        uint64_t keys[3];
        size_t at = 0;
        for (int k = 0; k < 3; ++k) {
            std::memcpy(hf + at, cls[k].data(), cls[k].size() * sizeof(FinalBucket));
            lists[k] = df + at;
            counts[k] = (uint32_t)cls[k].size();
            keys[k] = 0;
            for (const FinalBucket& f : cls[k]) keys[k] += f.size;
            at += cls[k].size();
        }
        e = cudaMemcpyAsync(df, hf, nf * sizeof(FinalBucket), cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = launch_bucket_finish(lists, counts, keys, ktmp, kout, kout, c.vtmp, vout, vout,
                                     KeyDesc{(uint32_t)sizeof(K), (uint64_t)flip}, st);
        // The pinned stage holds the list until the copy has been consumed.
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    *levels_out = level;
    *buckets_out = sorted_buckets;
    return AHS_OK;
}

}  // namespace

size_t samplesort_scratch_bytes(uint64_t n, uint32_t key_bytes, bool has_vals) {
    return carve_bytes(n, key_bytes, has_vals);
}

ahs_status run_samplesort(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin,
                          uint32_t* vout, uint64_t n, KeyDesc kd, void* scratch, cudaStream_t st,
                          uint32_t* levels_out, uint32_t* buckets_out) {
    *levels_out = 0;
    *buckets_out = 0;
    if (n <= kBucketCap) {
        *buckets_out = 1;
        return cuda_status(ctx, launch_blocksort_single(kin, kout, vin, vout, n, kd, st));
    }
    const bool v = vin != nullptr;
    if (kd.bytes == 4) {
        const uint32_t f = (uint32_t)kd.flip;
        return v ? samplesort_t<uint32_t, true>(ctx, (const uint32_t*)kin, (uint32_t*)kout, vin, vout, n, f, scratch, st, levels_out, buckets_out)
                 : samplesort_t<uint32_t, false>(ctx, (const uint32_t*)kin, (uint32_t*)kout, nullptr, nullptr, n, f, scratch, st, levels_out, buckets_out);
    }
    return v ? samplesort_t<uint64_t, true>(ctx, (const uint64_t*)kin, (uint64_t*)kout, vin, vout, n, kd.flip, scratch, st, levels_out, buckets_out)
             : samplesort_t<uint64_t, false>(ctx, (const uint64_t*)kin, (uint64_t*)kout, nullptr, nullptr, n, kd.flip, scratch, st, levels_out, buckets_out);
}

}  // namespace ahs
