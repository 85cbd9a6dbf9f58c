// Counting sort, keys only (Listing 2): Count[i] is the exact histogram the
// feature pass already built (bins are values when k <= 2^16), its exclusive
// prefix sum gives each value's first output position, and the output is
// written run by run.  The keys are not read again: value min + j fills
// positions [prefix[j], prefix[j+1]).  Output order for keys only is unique,
// so the stable reverse scan of Listing 2 and this fill give the same array.
#include <algorithm>

#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kScanThreads = 1024;
constexpr int kFillThreads = 256;
constexpr int kFillUnroll = 4;

// Exclusive prefix of the nbins exact counts; prefix[nbins] = n.
__global__ void __launch_bounds__(kScanThreads)
counting_prefix(const unsigned long long* __restrict__ hist, uint32_t nb,
                unsigned long long* __restrict__ prefix) {
    constexpr uint32_t kPer = kMaxBins / kScanThreads;   // 64 bins per thread
    const uint32_t j0 = threadIdx.x * kPer;
    unsigned long long loc = 0;
    for (uint32_t j = j0; j < j0 + kPer && j < nb; ++j) loc += hist[j];
    __shared__ unsigned long long scratch[kScanThreads / 32 + 1];
    unsigned long long total;
    unsigned long long run = block_exclusive_scan<kScanThreads>(loc, scratch, &total);
    for (uint32_t j = j0; j < j0 + kPer && j < nb; ++j) {
        prefix[j] = run;
        run += hist[j];
    }
    if (threadIdx.x == 0) prefix[nb] = total;
}

// Largest j in [lo, hi] with prefix[j] <= p (the bin holding output position p).
__device__ __forceinline__ uint32_t bin_of(const unsigned long long* __restrict__ prefix,
                                           uint64_t p, uint32_t lo, uint32_t hi) {
    while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// The same, for a position known to lie in bin lo or later: steps of 1, 2,
// 4, ... from lo, then a binary search in the last step (a few dependent
// loads when bins hold many keys).
__device__ __forceinline__ uint32_t bin_from(const unsigned long long* __restrict__ prefix,
                                             uint64_t p, uint32_t lo, uint32_t nb) {
    uint32_t step = 1;
    while (lo + step < nb && prefix[lo + step] <= p) {
        lo += step;
        step <<= 1;
    }
    const uint32_t hi = lo + step - 1 < nb - 1 ? lo + step - 1 : nb - 1;
    return bin_of(prefix, p, lo, hi);
}

// Dense (vals == nullptr): run j holds value mn + j.  Sparse: run j holds
// value mn + vals[j], and the run count and a failure flag come from the
// device (status[0] != 0: nothing to fill; status[1]: runs), so the fill can
// be queued before the runs are known.
template <typename K>
__global__ void __launch_bounds__(kFillThreads)
counting_fill(K* __restrict__ out, uint64_t n, uint64_t head, uint64_t nvec,
              const unsigned long long* __restrict__ prefix, uint32_t nb, K mn, K flip,
              const K* __restrict__ vals = nullptr, const uint32_t* __restrict__ status = nullptr) {
    constexpr int V = Vec16<K>::kN;
    constexpr uint64_t kChunk = (uint64_t)kFillThreads * kFillUnroll;   // vectors
    if (status) {
        if (status[0] != 0) return;
        nb = status[1];
        if (nb == 0) return;
    }
    auto value = [&](uint32_t j) { return (K)(mn + (vals ? vals[j] : (K)j)) ^ flip; };
    if (blockIdx.x == 0) {
        const uint64_t tail0 = head + nvec * V;
        if (threadIdx.x < head) out[threadIdx.x] = value(bin_of(prefix, threadIdx.x, 0, nb - 1));
        if (threadIdx.x < n - tail0) {
            const uint64_t p = tail0 + threadIdx.x;
            out[p] = value(bin_of(prefix, p, 0, nb - 1));
        }
    }
    // Each block fills a contiguous run of chunks.  Thread 0 finds the bins of
    // chunk c + 1 (from where chunk c ends) while the block writes chunk c.
    __shared__ uint32_t s_lo[2], s_hi[2];
    K* body = out + head;
    const uint64_t nchunks = ceil_div(nvec, kChunk);
    const uint64_t per = ceil_div(nchunks, (uint64_t)gridDim.x);
    const uint64_t c0 = (uint64_t)blockIdx.x * per;
    const uint64_t c1 = c0 + per < nchunks ? c0 + per : nchunks;
    auto bins = [&](uint64_t c, uint32_t from, int slot) {   // thread 0
        const uint64_t p0 = head + c * kChunk * V;
        uint64_t vend = (c + 1) * kChunk;
        vend = vend < nvec ? vend : nvec;
        const uint64_t p1 = head + vend * V - 1;
        const uint32_t lo = bin_from(prefix, p0, from, nb);
        s_lo[slot] = lo;
        s_hi[slot] = bin_from(prefix, p1, lo, nb);
    };
    if (threadIdx.x == 0 && c0 < c1) bins(c0, bin_of(prefix, head + c0 * kChunk * V, 0, nb - 1), 0);
    __syncthreads();
    for (uint64_t c = c0; c < c1; ++c) {
        const int slot = (int)((c - c0) & 1);
        const uint32_t lo = s_lo[slot], hi = s_hi[slot];
        if (threadIdx.x == 0 && c + 1 < c1) bins(c + 1, hi, slot ^ 1);
        // A chunk inside one run (most chunks when runs are long) writes
        // one value without searching.
        const K one = value(lo);
#pragma unroll
        for (int u = 0; u < kFillUnroll; ++u) {
            const uint64_t v = c * kChunk + (uint64_t)u * kFillThreads + threadIdx.x;
            if (v >= nvec) continue;
            const uint64_t p = head + v * V;
            Vec16<K> r;
            if (lo == hi) {
#pragma unroll
                for (int e = 0; e < V; ++e) r.e[e] = one;
            } else {
                uint32_t j = bin_of(prefix, p, lo, hi);
#pragma unroll
                for (int e = 0; e < V; ++e) {
                    while (AHS_DCHECK(j < nb, "fill bin", j) && prefix[j + 1] <= p + e) ++j;
                    r.e[e] = value(j);
                }
            }
            if constexpr (sizeof(K) == 4) __stcs(reinterpret_cast<uint4*>(body + v * V), r.v);
            else __stcs(reinterpret_cast<ulonglong2*>(body + v * V), r.v);
        }
        __syncthreads();   // publishes chunk c + 1's bins; slot `slot` is free again
    }
}

__global__ void __launch_bounds__(256)
copy32_vec(uint4* __restrict__ dst, const uint4* __restrict__ src, uint64_t nvec) {
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x;
    for (; i + 3 * stride < nvec; i += 4 * stride) {
        const uint4 a = __ldcs(src + i), b = __ldcs(src + i + stride);
        const uint4 c = __ldcs(src + i + 2 * stride), d = __ldcs(src + i + 3 * stride);
        __stcs(dst + i, a);
        __stcs(dst + i + stride, b);
        __stcs(dst + i + 2 * stride, c);
        __stcs(dst + i + 3 * stride, d);
    }
    for (; i < nvec; i += stride) __stcs(dst + i, __ldcs(src + i));
}

__global__ void __launch_bounds__(256)
copy32_scalar(uint32_t* __restrict__ dst, const uint32_t* __restrict__ src, uint64_t words) {
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < words; i += stride)
        dst[i] = src[i];
}

// out[n - 1 - i] = in[i].  Each thread swaps the pair (i, n - 1 - i), so
// in == out is allowed; a warp's two reads and two writes each cover
// consecutive addresses.
template <typename T>
__global__ void __launch_bounds__(256)
reverse_pairs(T* out, const T* in, uint64_t n) {
    const uint64_t half = (n + 1) / 2;
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < half; i += stride) {
        const uint64_t j = n - 1 - i;
        const T a = in[i], b = in[j];
        out[i] = b;
        out[j] = a;
    }
}

__global__ void __launch_bounds__(256)
zero32_vec(uint4* __restrict__ dst, uint64_t nvec) {
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < nvec; i += stride)
        dst[i] = make_uint4(0, 0, 0, 0);
}

uint32_t grid_for(uint64_t items, uint32_t per_block, int sms, uint32_t per_sm) {
    uint64_t b = ceil_div(items ? items : 1, per_block);
    const uint64_t cap = (uint64_t)sms * per_sm;
    return (uint32_t)(b < cap ? b : cap);
}

template <typename K>
cudaError_t fill_t(void* out_v, uint64_t n, K flip, const unsigned long long* hist,
                   unsigned long long* prefix, K mn, uint32_t nb, int sms, cudaStream_t st) {
    K* out = static_cast<K*>(out_v);
    constexpr int V = Vec16<K>::kN;
    {
        TraceScope ts("counting_prefix", 0, st);
        counting_prefix<<<1, kScanThreads, 0, st>>>(hist, nb, prefix);
    }
    const uint64_t head = head_elems<K>(out, n);
    const uint64_t nvec = (n - head) / V;
    const uint32_t g = grid_for(ceil_div(nvec, (uint64_t)kFillThreads * kFillUnroll), 1, sms, 8);
    TraceScope ts("counting_fill", n, st);
    counting_fill<K><<<g, kFillThreads, 0, st>>>(out, n, head, nvec, prefix, nb, mn, flip);
    return cudaGetLastError();
}

template <typename K>
cudaError_t sparse_fill_t(void* out_v, uint64_t n, K flip, const unsigned long long* prefix,
                          const K* vals, const uint32_t* status, K mn, int sms, cudaStream_t st) {
    K* out = static_cast<K*>(out_v);
    constexpr int V = Vec16<K>::kN;
    const uint64_t head = head_elems<K>(out, n);
    const uint64_t nvec = (n - head) / V;
    const uint32_t g = grid_for(ceil_div(nvec, (uint64_t)kFillThreads * kFillUnroll), 1, sms, 8);
    TraceScope ts("sparse_fill", n, st);
    counting_fill<K><<<g, kFillThreads, 0, st>>>(out, n, head, nvec, prefix, 0u, mn, flip, vals, status);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_sparse_fill(void* out, uint64_t n, KeyDesc kd, const unsigned long long* prefix,
                               const void* vals, const uint32_t* status, uint64_t min_ord, int sms,
                               cudaStream_t st) {
    if (kd.bytes == 4)
        return sparse_fill_t<uint32_t>(out, n, (uint32_t)kd.flip, prefix,
                                       static_cast<const uint32_t*>(vals), status, (uint32_t)min_ord,
                                       sms, st);
    return sparse_fill_t<uint64_t>(out, n, kd.flip, prefix, static_cast<const uint64_t*>(vals),
                                   status, min_ord, sms, st);
}

cudaError_t launch_counting_fill(void* out, uint64_t n, KeyDesc kd, const DevFeatures*,
                                 const unsigned long long* hist, unsigned long long* prefix,
                                 uint64_t min_ord, uint32_t nbins, int sms, cudaStream_t st) {
    if (kd.bytes == 4)
        return fill_t<uint32_t>(out, n, (uint32_t)kd.flip, hist, prefix, (uint32_t)min_ord, nbins,
                                sms, st);
    return fill_t<uint64_t>(out, n, kd.flip, hist, prefix, min_ord, nbins, sms, st);
}

cudaError_t launch_reverse(void* dst, const void* src, uint64_t n, uint32_t elem_bytes, int sms,
                           cudaStream_t st) {
    if (n == 0) return cudaSuccess;
    TraceScope ts("reverse", n, st);
    const uint32_t g = grid_for((n + 1) / 2, 1024, sms, 8);
    if (elem_bytes == 8)
        reverse_pairs<unsigned long long><<<g, 256, 0, st>>>(static_cast<unsigned long long*>(dst),
                                                             static_cast<const unsigned long long*>(src), n);
    else
        reverse_pairs<uint32_t><<<g, 256, 0, st>>>(static_cast<uint32_t*>(dst),
                                                   static_cast<const uint32_t*>(src), n);
    return cudaGetLastError();
}

cudaError_t launch_copy32(void* dst, const void* src, uint64_t words, int sms, cudaStream_t st) {
    if (words == 0 || dst == src) return cudaSuccess;
    TraceScope ts("copy", words, st);
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst), b = reinterpret_cast<uintptr_t>(src);
    if (((a ^ b) & 15u) == 0) {
        const uint64_t head = head_elems<uint32_t>(src, words);
        const uint64_t nvec = (words - head) / 4;
        const uint64_t tail = words - head - nvec * 4;
        if (head) copy32_scalar<<<1, 256, 0, st>>>((uint32_t*)dst, (const uint32_t*)src, head);
        if (nvec)
            copy32_vec<<<grid_for(nvec, 1024, sms, 8), 256, 0, st>>>(
                reinterpret_cast<uint4*>((uint32_t*)dst + head),
                reinterpret_cast<const uint4*>((const uint32_t*)src + head), nvec);
        if (tail)
            copy32_scalar<<<1, 256, 0, st>>>((uint32_t*)dst + head + nvec * 4,
                                             (const uint32_t*)src + head + nvec * 4, tail);
    } else {
        copy32_scalar<<<grid_for(words, 1024, sms, 8), 256, 0, st>>>((uint32_t*)dst,
                                                                    (const uint32_t*)src, words);
    }
    return cudaGetLastError();
}

// A list of copies (gather / scatter of many small arrays) in one launch: one
// CTA per item at a time, 16-byte vectors where both ends allow them.
__global__ void __launch_bounds__(256)
copy_list(const CopyItem* __restrict__ items, uint32_t count) {
    for (uint32_t it = blockIdx.x; it < count; it += gridDim.x) {
        const CopyItem c = items[it];
        uint32_t* d = static_cast<uint32_t*>(c.dst);
        const uint32_t* s = static_cast<const uint32_t*>(c.src);
        const uintptr_t a = reinterpret_cast<uintptr_t>(d), b = reinterpret_cast<uintptr_t>(s);
        if (((a ^ b) & 15u) == 0) {
            const uint64_t head = head_elems<uint32_t>(s, c.words);
            const uint64_t nvec = (c.words - head) / 4;
            for (uint64_t i = threadIdx.x; i < head; i += 256) d[i] = s[i];
            const uint4* sv = reinterpret_cast<const uint4*>(s + head);
            uint4* dv = reinterpret_cast<uint4*>(d + head);
            for (uint64_t i = threadIdx.x; i < nvec; i += 256) dv[i] = sv[i];
            for (uint64_t i = head + nvec * 4 + threadIdx.x; i < c.words; i += 256) d[i] = s[i];
        } else {
            for (uint64_t i = threadIdx.x; i < c.words; i += 256) d[i] = s[i];
        }
    }
}

__global__ void __launch_bounds__(256)
transfer_words(unsigned long long* __restrict__ dst, const unsigned long long* __restrict__ src,
               uint64_t words) {
    const uint64_t stride = (uint64_t)gridDim.x * 256;
    for (uint64_t i = (uint64_t)blockIdx.x * 256 + threadIdx.x; i < words; i += stride)
        dst[i] = src[i];
}

__global__ void __launch_bounds__(256)
transfer_bytes(unsigned char* __restrict__ dst, const unsigned char* __restrict__ src,
               uint64_t bytes) {
    for (uint64_t i = threadIdx.x; i < bytes; i += 256) dst[i] = src[i];
}

cudaError_t launch_transfer(void* dst, const void* src, size_t bytes, cudaStream_t st) {
    if (bytes == 0 || dst == src) return cudaSuccess;
    TraceScope ts("transfer", 0, st);
    const uintptr_t a = reinterpret_cast<uintptr_t>(dst), b = reinterpret_cast<uintptr_t>(src);
    const size_t words = bytes / 8;
    if (((a | b) & 7u) == 0 && words) {
        // Work lists are kilobytes to a few megabytes: up to 64 CTAs keep
        // enough host reads in flight.
        transfer_words<<<(uint32_t)std::min<uint64_t>(ceil_div(words, 256), 64), 256, 0, st>>>(
            static_cast<unsigned long long*>(dst), static_cast<const unsigned long long*>(src), words);
        if (bytes % 8)
            transfer_bytes<<<1, 256, 0, st>>>(static_cast<unsigned char*>(dst) + words * 8,
                                             static_cast<const unsigned char*>(src) + words * 8,
                                             bytes % 8);
    } else {
        transfer_bytes<<<1, 256, 0, st>>>(static_cast<unsigned char*>(dst),
                                         static_cast<const unsigned char*>(src), bytes);
    }
    return cudaGetLastError();
}

cudaError_t launch_copy_list(const CopyItem* items, uint32_t count, uint64_t words, int sms,
                             cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    TraceScope ts("copy_list", words, st);
    const uint32_t grid = std::min<uint32_t>(count, 8u * (uint32_t)sms);
    copy_list<<<grid, 256, 0, st>>>(items, count);
    return cudaGetLastError();
}

cudaError_t launch_zero32(void* dst, uint64_t words, int sms, cudaStream_t st) {
    if (words == 0) return cudaSuccess;
    TraceScope ts("zero", words, st);
    // Workspace regions are 256-byte aligned and sized in whole vectors.
    const uint64_t nvec = ceil_div(words, 4);
    zero32_vec<<<grid_for(nvec, 1024, sms, 8), 256, 0, st>>>(reinterpret_cast<uint4*>(dst), nvec);
    return cudaGetLastError();
}

}  // namespace ahs
