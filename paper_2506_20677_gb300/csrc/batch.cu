// Batched form: many independent arrays (segments of one buffer) sorted with
// one launch sequence per strategy class instead of one call per array.
//
//   1. segmented features: per segment n, min, max, descents (one pass over
//      all keys, chunked), then the entropy of its <= 2^16-bin histogram (one
//      CTA per segment below 65,536 keys with 16-bit counters; a cluster of two
//      CTAs per larger segment, each counting half of the bins);
//   2. the host selects a strategy per segment (same selector as ahs_sort);
//   3. per class: IDENTITY / SMALL -> one-CTA kernels; COUNTING -> one CTA per
//      segment (histogram, prefix, fill); RADIX -> segmented LSD passes;
//      GENERAL -> segmented sample sort.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "samplesort.h"
#include "segsort.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr uint32_t kChunkKeys = 16384;
constexpr int kMmThreads = 256;
constexpr int kHistT = 1024;
constexpr uint32_t kSmallHistMax = 65535;       // 16-bit counters cannot overflow below this
constexpr uint32_t kSegHistSmem = 32768u * 4u;  // 65,536 u16 counters / 32,768 u32 counters

struct SegChunk {
    unsigned long long begin;   // absolute (relative to the batch base)
    uint32_t len;
    uint32_t seg;
    unsigned long long seg_end;
};

struct SegFeat {
    unsigned long long min_ord;
    unsigned long long max_ord;
    unsigned long long descents;
    double ent[2];
    unsigned long long pad;
};
static_assert(sizeof(SegFeat) == 48, "SegFeat layout");

struct HistSeg {
    unsigned long long begin;
    uint32_t size;
    uint32_t seg;
    uint32_t slot;   // row of the coarse histogram (bin >> 8 counts), or kNoCoarse
    uint32_t pad;
};
constexpr uint32_t kNoCoarse = 0xffffffffu;
constexpr uint32_t kCoarse = 256;   // coarse buckets: the bin's high byte

// Adds this CTA's counts of bins [lo, lo + len) (u32 counters, or u16 pairs
// when PACKED) to the segment's coarse histogram row, one warp per bucket.
template <bool PACKED>
__device__ __forceinline__ void flush_coarse(const uint32_t* cnt, uint32_t lo, uint32_t len,
                                             uint32_t* row) {
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    const uint32_t c0 = lo >> 8, c1 = (lo + len + 255) >> 8;
    for (uint32_t c = c0 + warp; c < c1; c += kHistT / 32) {
        uint32_t sum = 0;
        for (uint32_t b = (c << 8) + lane; b < (c << 8) + 256; b += 32) {
            if (b < lo || b >= lo + len) continue;
            const uint32_t i = b - lo;
            sum += PACKED ? (cnt[i >> 1] >> (16 * (i & 1))) & 0xffffu : cnt[i];
        }
        sum = warp_sum(sum);
        if (lane == 0 && sum) atomicAdd(&row[c], sum);
    }
}

__global__ void seg_init(SegFeat* f, uint32_t nseg) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nseg) {
        f[i].min_ord = ~0ull;
        f[i].max_ord = 0;
        f[i].descents = 0;
        f[i].ent[0] = 0.0;
        f[i].ent[1] = 0.0;
    }
}

// Per chunk: min / max of ord(x) and descents, merged into the segment record.
template <typename K>
__global__ void __launch_bounds__(kMmThreads)
seg_minmax(const K* __restrict__ keys, const SegChunk* __restrict__ chunks, K flip,
           SegFeat* __restrict__ feat) {
    const SegChunk c = chunks[blockIdx.x];
    K mn = ~K(0), mx = 0;
    uint32_t desc = 0;
    const uint32_t lane = lane_id();
    // Warp-contiguous rows: the successor of a lane's key is the next lane's,
    // and lane 31 loads its own (usually a cache hit).
    for (uint32_t r = threadIdx.x - lane; r < c.len; r += kMmThreads) {
        const uint32_t i = r + lane;
        const bool ok = i < c.len;
        const unsigned long long e = c.begin + i;
        const K o = ok ? (K)(keys[e] ^ flip) : K(0);
        const K nx = __shfl_down_sync(AHS_FULL_MASK, o, 1);
        const bool has_next = ok && e + 1 < c.seg_end;
        const K succ = (lane == 31 || i + 1 >= c.len) && has_next ? (K)(keys[e + 1] ^ flip) : nx;
        if (ok) {
            mn = o < mn ? o : mn;
            mx = o > mx ? o : mx;
            if (has_next) desc += (o > succ) ? 1u : 0u;
        }
    }
    __shared__ unsigned long long s[3][kMmThreads / 32];
    unsigned long long a = warp_min((unsigned long long)mn), b = warp_max((unsigned long long)mx),
                       d = warp_sum((unsigned long long)desc);
    if (lane_id() == 0) { s[0][threadIdx.x >> 5] = a; s[1][threadIdx.x >> 5] = b; s[2][threadIdx.x >> 5] = d; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kMmThreads / 32; ++w) {
            a = s[0][w] < a ? s[0][w] : a;
            b = s[1][w] > b ? s[1][w] : b;
            d += s[2][w];
        }
        atomicMin(&feat[c.seg].min_ord, a);
        atomicMax(&feat[c.seg].max_ord, b);
        if (d) atomicAdd(&feat[c.seg].descents, d);
    }
}

// Calls f(key) for keys[0..n): each thread keeps kSegUnroll strided loads in
// flight, so one CTA alone can stream a segment at a useful rate.
constexpr int kSegUnroll = 8;
template <int T, typename K, typename F>
__device__ __forceinline__ void for_each_key(const K* __restrict__ keys, uint32_t n, F&& f) {
    constexpr uint32_t kStep = (uint32_t)T * kSegUnroll;
    uint32_t base = 0;
    for (; base + kStep <= n; base += kStep) {
        K x[kSegUnroll];
#pragma unroll
        for (int u = 0; u < kSegUnroll; ++u) x[u] = __ldg(keys + base + u * T + threadIdx.x);
#pragma unroll
        for (int u = 0; u < kSegUnroll; ++u) f(x[u]);
    }
    for (uint32_t i = base + threadIdx.x; i < n; i += T) f(keys[i]);
}

__device__ __forceinline__ void seg_bins(unsigned long long mn, unsigned long long mx, uint32_t* s,
                                         uint32_t* nb) {
    const unsigned long long span = mx - mn;
    const uint32_t bl = bitlen64(span);
    *s = bl > 16 ? bl - 16 : 0;
    *nb = (uint32_t)((span >> *s) + 1);
}

__device__ __forceinline__ double block_sum_1024(double v, double* red) {
    v = warp_sum(v);
    if (lane_id() == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < kHistT / 32; ++w) t += red[w];
    return t;
}

// Entropy terms in fp64 cost far more than the counting on this GPU (its
// fp64 rate is a small fraction of the fp32 rate), so every distinct bin
// count is evaluated once: cc[c] collects how many bins (or keys) have count
// c for c < kCcMax, and only rarer, larger counts are evaluated per bin.
constexpr uint32_t kCcMax = 4096;

__device__ __forceinline__ double plogp(uint32_t c, double inv) {
    const double p = (double)c * inv;
    return -p * log2(p);
}

// Sum over c of weight(c) * plogp(c) for the collected counts (all threads).
__device__ __forceinline__ double cc_sum(const uint32_t* cc, double inv, bool per_key) {
    double t = 0.0;
    for (uint32_t c = threadIdx.x + 1; c < kCcMax; c += kHistT) {
        const uint32_t w = cc[c];
        if (w) t += (double)(per_key ? w / c : w) * plogp(c, inv);
    }
    return t;
}

// One CTA per segment of at most 65,535 keys: 16-bit counters, two per word.
template <typename K>
__global__ void __launch_bounds__(kHistT, 1)
seg_hist_small(const K* __restrict__ keys, const HistSeg* __restrict__ segs, K flip,
               SegFeat* __restrict__ feat, uint32_t* __restrict__ coarse) {
    extern __shared__ __align__(16) uint32_t cnt[];
    __shared__ double red[kHistT / 32];
    __shared__ uint32_t cc[kCcMax];
    __shared__ uint32_t cs[kCoarse];
    const HistSeg g = segs[blockIdx.x];
    const K mn = (K)feat[g.seg].min_ord;
    uint32_t s, nb;
    seg_bins(feat[g.seg].min_ord, feat[g.seg].max_ord, &s, &nb);
    const uint32_t words = (nb + 1) / 2;
    const double inv = 1.0 / (double)g.size;
    double term = 0.0;
    const K* p = keys + g.begin;
    for (uint32_t i = threadIdx.x; i < kCcMax; i += kHistT) cc[i] = 0;
    for (uint32_t i = threadIdx.x; i < kCoarse; i += kHistT) cs[i] = 0;
    const bool by_key = (uint64_t)g.size * 4 < nb;
    const bool want_coarse = g.slot != kNoCoarse;
    if (by_key) {
        // Far fewer keys than bins: touch only the keys' own counters (zero
        // them, count), then every key adds one to cc[count of its bin]; a
        // bin of count c is seen c times.
        for_each_key<kHistT>(p, g.size, [&](K x) {
            cnt[(uint32_t)((K)((K)(x ^ flip) - mn) >> s) >> 1] = 0;
        });
        __syncthreads();
        for_each_key<kHistT>(p, g.size, [&](K x) {
            const uint32_t bin = (uint32_t)((K)((K)(x ^ flip) - mn) >> s);
            atomicAdd(&cnt[bin >> 1], 1u << (16 * (bin & 1)));
        });
        __syncthreads();
        for_each_key<kHistT>(p, g.size, [&](K x) {
            const uint32_t bin = (uint32_t)((K)((K)(x ^ flip) - mn) >> s);
            const uint32_t c = (cnt[bin >> 1] >> (16 * (bin & 1))) & 0xffffu;
            if (c < kCcMax) atomicAdd(&cc[c], 1u);
            else term += plogp(c, inv) / (double)c;
            if (want_coarse) atomicAdd(&cs[bin >> 8], 1u);
        });
        __syncthreads();
        if (want_coarse)
            for (uint32_t i = threadIdx.x; i < kCoarse; i += kHistT)
                if (cs[i]) coarse[(size_t)g.slot * kCoarse + i] = cs[i];
    } else {
        for (uint32_t i = threadIdx.x; i < words; i += kHistT) cnt[i] = 0;
        __syncthreads();
        for_each_key<kHistT>(p, g.size, [&](K x) {
            const uint32_t bin = (uint32_t)((K)((K)(x ^ flip) - mn) >> s);
            atomicAdd(&cnt[bin >> 1], 1u << (16 * (bin & 1)));
        });
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < words; i += kHistT) {
            const uint32_t w = cnt[i];
            const uint32_t c0 = w & 0xffffu, c1 = w >> 16;
            if (c0) { if (c0 < kCcMax) atomicAdd(&cc[c0], 1u); else term += plogp(c0, inv); }
            if (c1) { if (c1 < kCcMax) atomicAdd(&cc[c1], 1u); else term += plogp(c1, inv); }
        }
        if (want_coarse) flush_coarse<true>(cnt, 0, nb, coarse + (size_t)g.slot * kCoarse);
    }
    __syncthreads();
    term += cc_sum(cc, inv, by_key);
    const double t = block_sum_1024(term, red);
    if (threadIdx.x == 0) feat[g.seg].ent[0] = t;
}

// A cluster of two CTAs per larger segment: both read it (the second read is
// served by L2) and each counts half of the bins in 32-bit counters.
template <typename K>
__global__ void __launch_bounds__(kHistT, 1)
seg_hist_large(const K* __restrict__ keys, const HistSeg* __restrict__ segs, K flip,
               SegFeat* __restrict__ feat, uint32_t* __restrict__ coarse) {
    extern __shared__ __align__(16) uint32_t cnt[];
    __shared__ double red[kHistT / 32];
    __shared__ uint32_t cc[kCcMax];
    const uint32_t h = blockIdx.x & 1u;
    const HistSeg g = segs[blockIdx.x >> 1];
    const K mn = (K)feat[g.seg].min_ord;
    uint32_t s, nb;
    seg_bins(feat[g.seg].min_ord, feat[g.seg].max_ord, &s, &nb);
    const uint32_t half = (nb + 1) >> 1;
    const uint32_t lo = h * half;
    const uint32_t len = h ? nb - half : half;
    for (uint32_t i = threadIdx.x; i < len; i += kHistT) cnt[i] = 0;
    for (uint32_t i = threadIdx.x; i < kCcMax; i += kHistT) cc[i] = 0;
    __syncthreads();
    for_each_key<kHistT>(keys + g.begin, g.size, [&](K x) {
        const uint32_t b = (uint32_t)((K)((K)(x ^ flip) - mn) >> s) - lo;
        if (b < len) atomicAdd(&cnt[b], 1u);
    });
    __syncthreads();
    double term = 0.0;
    const double inv = 1.0 / (double)g.size;
    for (uint32_t i = threadIdx.x; i < len; i += kHistT) {
        const uint32_t c = cnt[i];
        if (c) { if (c < kCcMax) atomicAdd(&cc[c], 1u); else term += plogp(c, inv); }
    }
    if (g.slot != kNoCoarse) flush_coarse<false>(cnt, lo, len, coarse + (size_t)g.slot * kCoarse);
    __syncthreads();
    term += cc_sum(cc, inv, false);
    const double t = block_sum_1024(term, red);
    if (threadIdx.x == 0) feat[g.seg].ent[h] = t;
}

// Counting sort of one segment per CTA (keys only, k <= kCountMaxBins):
// histogram of key - min in shared memory, exclusive prefix, then the output
// filled value by value (the keys are not re-read for placement).
constexpr uint32_t kCountMaxBins = 32768;
struct CountSeg {
    unsigned long long begin;
    uint32_t size;
    uint32_t nb;
    unsigned long long min_ord;
};

template <typename K>
__global__ void __launch_bounds__(kHistT, 1)
seg_counting(const K* __restrict__ keys, K* __restrict__ out, const CountSeg* __restrict__ segs,
             K flip) {
    extern __shared__ __align__(16) uint32_t cnt[];   // nb counts, then reused as prefix
    __shared__ uint32_t scratch[kHistT / 32 + 1];
    __shared__ uint32_t s_lo, s_hi;
    const CountSeg g = segs[blockIdx.x];
    const K mn = (K)g.min_ord;
    for (uint32_t i = threadIdx.x; i <= g.nb; i += kHistT) cnt[i] = 0;
    __syncthreads();
    for_each_key<kHistT>(keys + g.begin, g.size, [&](K x) {
        atomicAdd(&cnt[(uint32_t)((K)(x ^ flip) - mn)], 1u);
    });
    __syncthreads();
    // Exclusive prefix over nb bins (each thread a contiguous run of bins).
    const uint32_t per = (g.nb + kHistT - 1) / kHistT;
    const uint32_t j0 = threadIdx.x * per;
    uint32_t loc = 0;
    for (uint32_t j = j0; j < j0 + per && j < g.nb; ++j) loc += cnt[j];
    uint32_t total;
    uint32_t run = block_exclusive_scan<kHistT>(loc, scratch, &total);
    for (uint32_t j = j0; j < j0 + per && j < g.nb; ++j) {
        const uint32_t c = cnt[j];
        cnt[j] = run;
        run += c;
    }
    if (threadIdx.x == 0) cnt[g.nb] = g.size;
    __syncthreads();
    // Fill: position q holds value min + j for the j with prefix[j] <= q < prefix[j+1].
    K* o = out + g.begin;
    for (uint32_t base = 0; base < g.size; base += kHistT) {
        const uint32_t q = base + threadIdx.x;
        if (q < g.size) {
            uint32_t lo = 0, hi = g.nb - 1;
            while (lo < hi) {
                const uint32_t mid = (lo + hi + 1) >> 1;
                if (cnt[mid] <= q) lo = mid;
                else hi = mid - 1;
            }
            o[q] = (K)(mn + (K)lo) ^ flip;
        }
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

template <typename K>
ahs_status batch_t(ahs_ctx* ctx, const K* kin, K* kout, const uint32_t* vin, uint32_t* vout,
                   const uint64_t* offs, uint32_t n_seg, KeyDesc kd, cudaStream_t st,
                   ahs_batch_info_t* info) {
    using clock = std::chrono::steady_clock;
    const K flip = (K)kd.flip;
    const uint64_t base = offs[0];
    const uint64_t N = offs[n_seg] - base;
    kin += base;
    kout += base;
    if (vin) {
        vin += base;
        vout += base;
    }
    const bool payload = vin != nullptr;

    // ---- 1. segmented features -------------------------------------------
    std::vector<SegChunk> chunks;
    std::vector<HistSeg> hsmall, hlarge;
    ahs_thresholds_t th;
    const bool model = ctx->cfg.select_mode == AHS_SEL_MODEL;
    if (ctx->cfg.select_mode == AHS_SEL_CUSTOM) th = ctx->custom;
    else profile_thresholds(model ? AHS_SEL_GB300 : ctx->cfg.select_mode, &th);
    // Keys-only segments the general class may take keep a coarse histogram
    // (256 counts of the bin's high byte): its first partition level is then
    // planned on the host with exact bucket sizes.
    std::vector<uint32_t> slot_of(n_seg, kNoCoarse);
    uint32_t n_slots = 0;
    for (uint32_t s = 0; s < n_seg; ++s) {
        const uint64_t b = offs[s] - base, n = offs[s + 1] - offs[s];
        for (uint64_t o = 0; o < n; o += kChunkKeys)
            chunks.push_back({b + o, (uint32_t)std::min<uint64_t>(kChunkKeys, n - o), s, b + n});
        // Entropy is only needed where the selector reads it.
        const bool need_h = n > th.n_t || model;
        if (need_h && n > 1) {
            const uint32_t slot = (!payload && n > kBucketCap) ? n_slots++ : kNoCoarse;
            slot_of[s] = slot;
            (n <= kSmallHistMax ? hsmall : hlarge).push_back({b, (uint32_t)n, s, slot, 0});
        }
    }
    const size_t b_feat = a256((size_t)n_seg * sizeof(SegFeat));
    const size_t b_coarse = a256((size_t)n_slots * kCoarseBuckets * 4);
    const size_t b_chunks = a256(chunks.size() * sizeof(SegChunk));
    const size_t b_hs = a256(hsmall.size() * sizeof(HistSeg)), b_hl = a256(hlarge.size() * sizeof(HistSeg));
    ahs_status rc = ensure_aux(ctx, b_feat + b_coarse + b_chunks + b_hs + b_hl);
    if (rc == AHS_OK) rc = ensure_stage(ctx, std::max(b_chunks + b_hs + b_hl, b_feat));
    if (rc != AHS_OK) return rc;
    char* a = static_cast<char*>(ctx->aux);
    SegFeat* d_feat = reinterpret_cast<SegFeat*>(a);
    uint32_t* d_coarse = reinterpret_cast<uint32_t*>(a + b_feat);
    SegChunk* d_chunks = reinterpret_cast<SegChunk*>(a + b_feat + b_coarse);
    HistSeg* d_hs = reinterpret_cast<HistSeg*>(a + b_feat + b_coarse + b_chunks);
    HistSeg* d_hl = reinterpret_cast<HistSeg*>(a + b_feat + b_coarse + b_chunks + b_hs);
    char* hsb = static_cast<char*>(ctx->h_stage);
    std::memcpy(hsb, chunks.data(), chunks.size() * sizeof(SegChunk));
    std::memcpy(hsb + b_chunks, hsmall.data(), hsmall.size() * sizeof(HistSeg));
    std::memcpy(hsb + b_chunks + b_hs, hlarge.data(), hlarge.size() * sizeof(HistSeg));
    cudaError_t e = launch_transfer(d_chunks, hsb, b_chunks + b_hs + b_hl, st);
    const auto t0 = clock::now();
    uint64_t keys_small = 0, keys_large = 0;
    for (const HistSeg& h : hsmall) keys_small += h.size;
    for (const HistSeg& h : hlarge) keys_large += h.size;
    if (e == cudaSuccess && n_slots) e = launch_zero32(d_coarse, (uint64_t)n_slots * kCoarseBuckets, ctx->sms, st);
    if (e == cudaSuccess) {
        {
            TraceScope ts("batch_minmax", N, st);
            seg_init<<<(n_seg + 255) / 256, 256, 0, st>>>(d_feat, n_seg);
            if (!chunks.empty())
                seg_minmax<K><<<(uint32_t)chunks.size(), kMmThreads, 0, st>>>(kin, d_chunks, flip, d_feat);
        }
        e = cudaFuncSetAttribute(seg_hist_small<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSegHistSmem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(seg_hist_large<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSegHistSmem);
        if (e == cudaSuccess && !hsmall.empty()) {
            TraceScope ts("batch_hist_small", keys_small, st);
            seg_hist_small<K><<<(uint32_t)hsmall.size(), kHistT, kSegHistSmem, st>>>(kin, d_hs, flip, d_feat,
                                                                                 d_coarse);
        }
        if (e == cudaSuccess && !hlarge.empty()) {
            TraceScope ts("batch_hist_large", keys_large, st);
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(2 * (uint32_t)hlarge.size());
            cfg.blockDim = dim3(kHistT);
            cfg.dynamicSmemBytes = kSegHistSmem;
            cfg.stream = st;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = 2;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            e = cudaLaunchKernelEx(&cfg, seg_hist_large<K>, kin, (const HistSeg*)d_hl, flip, d_feat,
                                   d_coarse);
        }
    }
    // The records come back to the staging buffer, the coarse histograms to a
    // pinned buffer of their own (read in place while the classes reuse the
    // staging buffer).
    const size_t coarse_bytes = (size_t)n_slots * kCoarseBuckets * 4;
    if (coarse_bytes > ctx->h_coarse_bytes) {
        if (ctx->h_coarse) cudaFreeHost(ctx->h_coarse);
        ctx->h_coarse = nullptr;
        ctx->h_coarse_bytes = 0;
        if (e == cudaSuccess) e = cudaHostAlloc(&ctx->h_coarse, coarse_bytes + coarse_bytes / 2,
                                                cudaHostAllocDefault);
        if (e == cudaSuccess) ctx->h_coarse_bytes = coarse_bytes + coarse_bytes / 2;
        else ctx->h_coarse = nullptr;
    }
    if (e == cudaSuccess) e = launch_transfer(hsb, d_feat, (size_t)n_seg * sizeof(SegFeat), st);
    if (e == cudaSuccess && n_slots) e = launch_transfer(ctx->h_coarse, d_coarse, coarse_bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    const auto t1 = clock::now();
    const uint32_t* coarse = static_cast<const uint32_t*>(ctx->h_coarse);

    // ---- 2. selection ------------------------------------------------------
    const SegFeat* hf = reinterpret_cast<const SegFeat*>(hsb);
    std::vector<SegRange> ident, small, radix, general, gsmall;
    std::vector<HistRange> ghist;
    std::vector<CountSeg> counting;
    uint32_t radix_passes = 0;
    if (info) std::memset(info, 0, sizeof(*info));
    for (uint32_t s = 0; s < n_seg; ++s) {
        const uint64_t b = offs[s] - base, n = offs[s + 1] - offs[s];
        ahs_features_t f{};
        f.n = n;
        if (n) {
            f.min_bits = hf[s].min_ord ^ kd.flip;
            f.max_bits = hf[s].max_ord ^ kd.flip;
            f.span = hf[s].max_ord - hf[s].min_ord;
            const uint32_t bl = bitlen64(f.span);
            f.hist_shift = bl > 16 ? bl - 16 : 0;
            f.nbins = (uint32_t)((f.span >> f.hist_shift) + 1);
            f.entropy_bits = hf[s].ent[0] + hf[s].ent[1];
            f.entropy_norm = f.nbins > 1 ? f.entropy_bits / std::log2((double)f.nbins) : 0.0;
            f.descents = hf[s].descents;
        }
        ahs_strategy st_s = choose(ctx, f, kd.bytes, payload);
        // Counting here is keys-only with the whole range in one CTA's
        // shared memory; wider ranges and payloads take the radix class.
        if (st_s == AHS_COUNTING && (payload || f.span >= kCountMaxBins)) st_s = AHS_RADIX;
        // The tuned cutoff: segments this small are sorted by one CTA
        // whatever their strategy (the launch is cheaper than a class pass).
        const uint32_t cut = ctx->tuning.batch_small_cutoff();
        if (cut && n > 1 && n <= cut && n <= kBucketCap && st_s != AHS_IDENTITY) st_s = AHS_SMALL;
        const SegRange r{b, (uint32_t)n, f.min_bits ^ kd.flip};
        switch (st_s) {
        case AHS_IDENTITY: ident.push_back(r); break;
        case AHS_SMALL: small.push_back(r); break;
        case AHS_COUNTING: counting.push_back({b, (uint32_t)n, (uint32_t)(f.span + 1), r.min_ord}); break;
        case AHS_RADIX:
            if (n <= kBucketCap) {
                small.push_back(r);
            } else if (!payload) {
                // Keys only: the low-entropy segments of this class settle
                // their heavy keys in equality buckets of the sampled-splitter
                // levels at once, where digit levels would re-scatter them up
                // to four times; equal keys make the result the same.
                general.push_back(r);
            } else {
                radix.push_back(r);
                radix_passes = std::max(radix_passes, (bitlen64(f.span) + 7) / 8);
            }
            break;
        default:
            if (n <= kBucketCap) gsmall.push_back(r);
            else if (slot_of[s] != kNoCoarse)
                ghist.push_back({r, f.hist_shift, f.descents < f.n / 4, runs_likely(f.descents, f.n),
                                 coarse + (size_t)slot_of[s] * kCoarseBuckets});
            else general.push_back(r);
            break;
        }
        if (info && st_s >= 0 && st_s < 6) {
            info->seg_per_strategy[st_s] += 1;
            info->keys_per_strategy[st_s] += n;
        }
    }
    const auto t2 = clock::now();

    // ---- 3. per-class launches ----------------------------------------------
    // IDENTITY (copies) and SMALL (one-CTA sorts) share one bucket launch per size class.
    if (!small.empty() || !ident.empty()) {
        rc = run_small_segments(ctx, kin, kout, vin, vout, small, ident, kd, st);
        if (rc != AHS_OK) return rc;
    }
    if (!counting.empty()) {
        rc = ensure_aux(ctx, counting.size() * sizeof(CountSeg));
        if (rc == AHS_OK) rc = ensure_stage(ctx, counting.size() * sizeof(CountSeg));
        if (rc != AHS_OK) return rc;
        std::memcpy(ctx->h_stage, counting.data(), counting.size() * sizeof(CountSeg));
        e = launch_transfer(ctx->aux, ctx->h_stage, counting.size() * sizeof(CountSeg), st);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(seg_counting<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (kCountMaxBins + 1) * 4);
        if (e == cudaSuccess) {
            TraceScope ts("batch_counting", info ? info->keys_per_strategy[AHS_COUNTING] : 0, st);
            seg_counting<K><<<(uint32_t)counting.size(), kHistT, (kCountMaxBins + 1) * 4, st>>>(
                kin, kout, static_cast<const CountSeg*>(ctx->aux), flip);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(ctx, e);
    }
    if (!radix.empty() || !general.empty() || !gsmall.empty() || !ghist.empty()) {
        rc = ensure_workspace(ctx, features_region(ctx->sms) + segsort_scratch_bytes(N, n_seg, kd.bytes, payload));
        if (rc != AHS_OK) return rc;
        void* scratch = static_cast<char*>(ctx->ws) + features_region(ctx->sms);
        if (!radix.empty()) {
            rc = run_segmented_radix(ctx, kin, kout, vin, vout, N, radix, radix_passes, kd, scratch, st);
            if (rc != AHS_OK) return rc;
            e = cudaStreamSynchronize(st);   // the radix lists in aux must be consumed first
            if (e != cudaSuccess) return cuda_status(ctx, e);
        }
        if (!ghist.empty()) {
            // General segments with coarse histograms (and the small ones).
            uint32_t lv = 0, nb = 0;
            rc = run_batched_general_hist(ctx, kin, kout, N, ghist, gsmall, kd, scratch, st, &lv, &nb);
            if (rc != AHS_OK) return rc;
            gsmall.clear();
        }
        if (!general.empty() || !gsmall.empty()) {
            uint32_t lv = 0, nb = 0;
            rc = run_segmented_general(ctx, kin, kout, vin, vout, N, general, gsmall, kd, scratch, st,
                                       &lv, &nb);
            if (rc != AHS_OK) return rc;
        }
    }
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    const auto t3 = clock::now();
    if (info) {
        info->n_keys = N;
        info->n_seg = n_seg;
        info->ms_features = std::chrono::duration<float, std::milli>(t1 - t0).count();
        info->ms_select = std::chrono::duration<float, std::milli>(t2 - t1).count();
        info->ms_sort = std::chrono::duration<float, std::milli>(t3 - t2).count();
    }
    return check_device_error(ctx, st);
}

}  // namespace

ahs_status run_batch(ahs_ctx* ctx, const void* kin, void* kout, const uint32_t* vin, uint32_t* vout,
                     const uint64_t* offs, uint32_t n_seg, KeyDesc kd, cudaStream_t st,
                     ahs_batch_info_t* info) {
    if (kd.bytes == 4)
        return batch_t<uint32_t>(ctx, static_cast<const uint32_t*>(kin), static_cast<uint32_t*>(kout),
                                 vin, vout, offs, n_seg, kd, st, info);
    return batch_t<uint64_t>(ctx, static_cast<const uint64_t*>(kin), static_cast<uint64_t*>(kout), vin,
                             vout, offs, n_seg, kd, st, info);
}

}  // namespace ahs

extern "C" ahs_status ahs_sort_batch(ahs_ctx* ctx, const void* d_keys_in, void* d_keys_out,
                                     const uint32_t* d_vals_in, uint32_t* d_vals_out,
                                     const uint64_t* h_seg_offsets, uint32_t n_seg,
                                     ahs_key_type type, void* stream, ahs_batch_info_t* info) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!ctx || ctx->device < 0 || (n_seg && !h_seg_offsets)) return AHS_ERR_INVALID_ARG;
    if (type < AHS_U32 || type > AHS_I64) return AHS_ERR_DTYPE;
    if (n_seg == 0) return AHS_OK;
    for (uint32_t s = 0; s < n_seg; ++s) {
        if (h_seg_offsets[s + 1] < h_seg_offsets[s]) return AHS_ERR_INVALID_ARG;
        if (h_seg_offsets[s + 1] - h_seg_offsets[s] >= (1ull << 32)) return AHS_ERR_RANGE;
    }
    const uint64_t total = h_seg_offsets[n_seg] - h_seg_offsets[0];
    if (total == 0) return AHS_OK;
    if (!d_keys_in || !d_keys_out || d_keys_in == d_keys_out) return AHS_ERR_INVALID_ARG;
    if (d_vals_in && (!d_vals_out || d_vals_in == d_vals_out)) return AHS_ERR_INVALID_ARG;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return ahs::cuda_status(ctx, e);
    ahs::TracerGuard tg(&ctx->tracer);
    return ahs::run_batch(ctx, d_keys_in, d_keys_out, d_vals_in, d_vals_out, h_seg_offsets, n_seg,
                          ahs::key_desc(type), static_cast<cudaStream_t>(stream), info);
}

extern "C" ahs_status ahs_sort_batch_dev(ahs_ctx* ctx, const void* d_keys_in, void* d_keys_out,
                                         const uint32_t* d_vals_in, uint32_t* d_vals_out,
                                         const uint64_t* d_seg_offsets, uint32_t n_seg,
                                         ahs_key_type type, void* stream, ahs_batch_info_t* info) {
    if (info) std::memset(info, 0, sizeof(*info));
    if (!ctx || ctx->device < 0 || (n_seg && !d_seg_offsets)) return AHS_ERR_INVALID_ARG;
    if (type < AHS_U32 || type > AHS_I64) return AHS_ERR_DTYPE;
    if (n_seg == 0) return AHS_OK;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return ahs::cuda_status(ctx, e);
    // The offsets come to pinned host memory by kernel (behind the work
    // already on the stream), then the host-planned batch runs as usual.
    const size_t bytes = ((size_t)n_seg + 1) * sizeof(uint64_t);
    ahs_status rc = ahs::ensure_stage(ctx, bytes);
    if (rc != AHS_OK) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    e = ahs::launch_transfer(ctx->h_stage, d_seg_offsets, bytes, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return ahs::cuda_status(ctx, e);
    // The staging buffer is reused by the batch itself: keep a copy.
    std::vector<uint64_t> offs(static_cast<const uint64_t*>(ctx->h_stage),
                               static_cast<const uint64_t*>(ctx->h_stage) + n_seg + 1);
    return ahs_sort_batch(ctx, d_keys_in, d_keys_out, d_vals_in, d_vals_out, offs.data(), n_seg,
                          type, stream, info);
}

