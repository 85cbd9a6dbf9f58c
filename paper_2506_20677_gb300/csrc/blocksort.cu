// One-block sorts: the SMALL strategy (a whole input that fits one CTA) and
// the segmented bucket sort of the general path (one CTA per bucket).
#include <algorithm>

#include "blocksort.cuh"
#include "internal.h"
#include "trace.h"
#include "samplesort.h"

namespace ahs {
namespace {

template <typename K, bool VALS, int T, int IPT>
__global__ void __launch_bounds__(T)
blocksort_single(const K* keys_in, K* keys_out, const uint32_t* vals_in, uint32_t* vals_out,
                 uint32_t n, K flip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    if constexpr (VALS) {
        auto& S = *reinterpret_cast<BlockSortSmem<K, VALS, T, IPT>*>(smem_raw);
        block_sort<K, VALS, T, IPT>(keys_in, keys_out, vals_in, vals_out, n, flip, S);
    } else {
        block_sort_keys<K, T, IPT>(keys_in, keys_out, n, flip, smem_raw);
    }
}

// One CTA per final bucket: sort src[begin, begin+size) into out (sorted
// buckets), or copy it (buckets whose keys are all equal need no pass).  The
// source is buffer 0 (temporary), 1 (the output itself) or 2 (the input).
// Resident CTAs per SM each keys-only uint32 bucket class is compiled for,
// as measured: 256 x 16 at five CTAs (a few spilled bytes) beat four by 4 %,
// while 256 x 18 lost 9 % at five.  Wider keys and payloads leave the
// register budget to the compiler.
template <typename K, bool VALS, int T, int IPT>
struct BucketMinBlocks {
    static constexpr int kN =
        (sizeof(K) == 4 && !VALS)
            ? (T <= 128 ? 8 : (T <= 192 ? 5 : (T <= 256 ? (IPT <= 16 ? 5 : 4) : (T <= 384 ? 3 : 2))))
            : 1;
};

template <typename K, bool VALS, int T, int IPT>
__global__ void __launch_bounds__(T, BucketMinBlocks<K, VALS, T, IPT>::kN)
bucket_finish(const FinalBucket* __restrict__ list, const K* buf0, const K* buf1, const K* buf2,
              K* out, const uint32_t* vbuf0, const uint32_t* vbuf1, const uint32_t* vbuf2,
              uint32_t* vout, K flip) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const FinalBucket b = list[blockIdx.x];
    const K* src = (b.where == 0 ? buf0 : (b.where == 1 ? buf1 : buf2)) + b.begin;
    const uint32_t* vsrc =
        VALS ? (b.where == 0 ? vbuf0 : (b.where == 1 ? vbuf1 : vbuf2)) + b.begin : nullptr;
    K* dst = out + b.begin;
    uint32_t* vdst = VALS ? vout + b.begin : nullptr;
    if (b.sort) {
        if constexpr (VALS) {
            auto& S = *reinterpret_cast<BlockSortSmem<K, VALS, T, IPT>*>(smem_raw);
            block_sort<K, VALS, T, IPT>(src, dst, vsrc, vdst, b.size, flip, S, (K)b.lo, b.bits);
        } else {
            block_sort_keys<K, T, IPT>(src, dst, b.size, flip, smem_raw, (K)b.lo, b.bits);
        }
    } else if (src != dst) {
        for (uint32_t i = threadIdx.x; i < b.size; i += T) {
            dst[i] = src[i];
            if constexpr (VALS) vdst[i] = vsrc[i];
        }
    }
}

template <typename K, bool VALS, int T, int IPT>
cudaError_t single_t(const void* kin, void* kout, const uint32_t* vin, uint32_t* vout, uint32_t n,
                     K flip, cudaStream_t st) {
    constexpr size_t kSmem = block_sort_smem_bytes<K, VALS, T, IPT>();
    auto fn = blocksort_single<K, VALS, T, IPT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e != cudaSuccess) return e;
    TraceScope ts("blocksort_single", n, st);
    fn<<<1, T, kSmem, st>>>(static_cast<const K*>(kin), static_cast<K*>(kout), vin, vout, n,
                                   flip);
    return cudaGetLastError();
}

template <typename K, bool VALS, int T, int IPT>
cudaError_t finish_class(const FinalBucket* d_list, uint32_t count, uint64_t keys, const void* b0,
                         const void* b1, const void* b2, void* out, const uint32_t* vb0,
                         const uint32_t* vb1, const uint32_t* vb2, uint32_t* vout, K flip,
                         cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    constexpr size_t kSmem = block_sort_smem_bytes<K, VALS, T, IPT>();
    auto fn = bucket_finish<K, VALS, T, IPT>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kSmem);
    if (e != cudaSuccess) return e;
    // Grids are limited to 2^31 - 1 blocks in x; bucket lists are far smaller.
    constexpr int CAP = T * IPT;
    TraceScope ts(CAP <= 1024 ? "bucket_sort_1k"
                  : CAP <= 2048 ? "bucket_sort_2k"
                  : CAP <= 3072 ? "bucket_sort_3k"
                  : CAP <= 4096 ? "bucket_sort_4k"
                  : CAP <= 4608 ? "bucket_sort_4.5k"
                  : CAP <= 6144 ? "bucket_sort_6k" : "bucket_sort_8k",
                  keys, st);
    fn<<<count, T, kSmem, st>>>(d_list, static_cast<const K*>(b0), static_cast<const K*>(b1),
                                       static_cast<const K*>(b2), static_cast<K*>(out), vb0, vb1,
                                       vb2, vout, flip);
    return cudaGetLastError();
}

template <typename K, bool VALS>
cudaError_t finish_t(const FinalBucket* d_lists[kBucketClasses], const uint32_t counts[kBucketClasses],
                     const uint64_t keys[kBucketClasses], const void* b0, const void* b1, const void* b2,
                     void* out, const uint32_t* vb0, const uint32_t* vb1, const uint32_t* vb2,
                     uint32_t* vout, K flip, cudaStream_t st) {
    cudaError_t e = finish_class<K, VALS, 128, 8>(d_lists[0], counts[0], keys[0], b0, b1, b2, out,
                                                  vb0, vb1, vb2, vout, flip, st);
    if (e == cudaSuccess)
        e = finish_class<K, VALS, 256, 8>(d_lists[1], counts[1], keys[1], b0, b1, b2, out, vb0,
                                          vb1, vb2, vout, flip, st);
    if (e == cudaSuccess)
        e = finish_class<K, VALS, 192, 16>(d_lists[2], counts[2], keys[2], b0, b1, b2, out, vb0,
                                           vb1, vb2, vout, flip, st);
    if (e == cudaSuccess)
        e = finish_class<K, VALS, 256, 16>(d_lists[3], counts[3], keys[3], b0, b1, b2, out, vb0,
                                           vb1, vb2, vout, flip, st);
    if (e == cudaSuccess)
        e = finish_class<K, VALS, 256, 18>(d_lists[4], counts[4], keys[4], b0, b1, b2, out, vb0,
                                           vb1, vb2, vout, flip, st);
    if (e == cudaSuccess)
        e = finish_class<K, VALS, 384, 16>(d_lists[5], counts[5], keys[5], b0, b1, b2, out, vb0,
                                           vb1, vb2, vout, flip, st);
    if (e == cudaSuccess)
        e = finish_class<K, VALS, 512, 16>(d_lists[6], counts[6], keys[6], b0, b1, b2, out, vb0,
                                           vb1, vb2, vout, flip, st);
    return e;
}

}  // namespace

uint64_t blocksort_capacity(uint32_t, bool) { return kBucketCap; }


cudaError_t launch_blocksort_single(const void* keys_in, void* keys_out, const uint32_t* vals_in,
                                    uint32_t* vals_out, uint64_t n, KeyDesc kd, cudaStream_t st) {
    const uint32_t m = (uint32_t)n;
    const bool v = vals_in != nullptr;
    if (kd.bytes == 4) {
        if (n <= 1024)
            return v ? single_t<uint32_t, true, 128, 8>(keys_in, keys_out, vals_in, vals_out, m, (uint32_t)kd.flip, st)
                     : single_t<uint32_t, false, 128, 8>(keys_in, keys_out, nullptr, nullptr, m, (uint32_t)kd.flip, st);
        return v ? single_t<uint32_t, true, 512, 16>(keys_in, keys_out, vals_in, vals_out, m, (uint32_t)kd.flip, st)
                 : single_t<uint32_t, false, 512, 16>(keys_in, keys_out, nullptr, nullptr, m, (uint32_t)kd.flip, st);
    }
    if (n <= 1024)
        return v ? single_t<uint64_t, true, 128, 8>(keys_in, keys_out, vals_in, vals_out, m, kd.flip, st)
                 : single_t<uint64_t, false, 128, 8>(keys_in, keys_out, nullptr, nullptr, m, kd.flip, st);
    return v ? single_t<uint64_t, true, 512, 16>(keys_in, keys_out, vals_in, vals_out, m, kd.flip, st)
             : single_t<uint64_t, false, 512, 16>(keys_in, keys_out, nullptr, nullptr, m, kd.flip, st);
}

cudaError_t launch_bucket_finish(const FinalBucket* d_lists[kBucketClasses],
                                 const uint32_t counts[kBucketClasses],
                                 const uint64_t keys[kBucketClasses], const void* buf0, const void* buf1,
                                 const void* buf2, void* out, const uint32_t* vbuf0,
                                 const uint32_t* vbuf1, const uint32_t* vbuf2, uint32_t* vout,
                                 KeyDesc kd, cudaStream_t st) {
    const bool v = vout != nullptr && vbuf2 != nullptr;
    if (kd.bytes == 4)
        return v ? finish_t<uint32_t, true>(d_lists, counts, keys, buf0, buf1, buf2, out, vbuf0,
                                           vbuf1, vbuf2, vout, (uint32_t)kd.flip, st)
                 : finish_t<uint32_t, false>(d_lists, counts, keys, buf0, buf1, buf2, out, nullptr,
                                            nullptr, nullptr, nullptr, (uint32_t)kd.flip, st);
    return v ? finish_t<uint64_t, true>(d_lists, counts, keys, buf0, buf1, buf2, out, vbuf0, vbuf1,
                                       vbuf2, vout, kd.flip, st)
             : finish_t<uint64_t, false>(d_lists, counts, keys, buf0, buf1, buf2, out, nullptr,
                                        nullptr, nullptr, nullptr, kd.flip, st);
}

}  // namespace ahs
