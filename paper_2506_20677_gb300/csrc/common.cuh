// Shared device-side helpers of the GB300 Adaptive Hybrid Sort library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define AHS_FULL_MASK 0xffffffffu

// Device self-checks (build with AHS_CHECKS=1): a failed check prints the
// site and the offending index and the access is skipped.
#ifdef AHS_DEVICE_CHECKS
#include <cstdio>
#define AHS_DCHECK(cond, what, idx)                                                         \
    ((cond) ? true                                                                          \
            : (printf("AHS check failed: %s at %s:%d block %d thread %d idx %llu\n", what, \
                      __FILE__, __LINE__, (int)blockIdx.x, (int)threadIdx.x,                \
                      (unsigned long long)(idx)),                                           \
               false))
#else
#define AHS_DCHECK(cond, what, idx) true
#endif

namespace ahs {

// Number of SMs on the device the kernels are sized for; the host passes the
// queried value, this is only the fallback.
constexpr int kDefaultSms = 152;

// Device error codes written to the context's error word (never trap).
enum DeviceError : uint32_t {
    kDevOk = 0,
    kDevLookbackTimeout = 1,   // a decoupled look-back wait ran out
    kDevBadState = 2,          // a status word held an impossible value
    kDevOverflow = 3,          // a bucket exceeded the capacity a kernel was sized for
};

// Key traits: keys move as their raw bits (K); digits, ranges and histograms
// are taken on the order-preserving unsigned image ord(x) = x ^ flip, where
// flip is the sign bit for signed types and 0 otherwise.
template <typename K> struct KeyBits;
template <> struct KeyBits<uint32_t> { static constexpr int kBits = 32; };
template <> struct KeyBits<uint64_t> { static constexpr int kBits = 64; };

// 16-byte vector of keys.
template <typename K> struct Vec16;
template <> struct Vec16<uint32_t> {
    static constexpr int kN = 4;
    union { uint4 v; uint32_t e[4]; };
};
template <> struct Vec16<uint64_t> {
    static constexpr int kN = 2;
    union { ulonglong2 v; uint64_t e[2]; };
};

template <typename K>
__device__ __forceinline__ Vec16<K> load_vec16(const K* p) {
    Vec16<K> r;
    if constexpr (sizeof(K) == 4) r.v = __ldg(reinterpret_cast<const uint4*>(p));
    else r.v = __ldg(reinterpret_cast<const ulonglong2*>(p));
    return r;
}

// Streaming (evict-first) 16-byte load for data read exactly once.
template <typename K>
__device__ __forceinline__ Vec16<K> load_vec16_stream(const K* p) {
    Vec16<K> r;
    if constexpr (sizeof(K) == 4) r.v = __ldcs(reinterpret_cast<const uint4*>(p));
    else r.v = __ldcs(reinterpret_cast<const ulonglong2*>(p));
    return r;
}

template <typename K>
__device__ __forceinline__ void store_vec16(K* p, const Vec16<K>& x) {
    if constexpr (sizeof(K) == 4) *reinterpret_cast<uint4*>(p) = x.v;
    else *reinterpret_cast<ulonglong2*>(p) = x.v;
}

// Elements before the first 16-byte boundary of p (p must be element-aligned).
template <typename K>
__host__ __device__ __forceinline__ uint64_t head_elems(const void* p, uint64_t n) {
    const uint64_t mis = (reinterpret_cast<uintptr_t>(p) & 15u) / sizeof(K);
    uint64_t h = mis ? (16 / sizeof(K)) - mis : 0;
    return h < n ? h : n;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm volatile("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

template <typename T>
__device__ __forceinline__ T warp_min(T v) {
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(AHS_FULL_MASK, v, o);
        v = u < v ? u : v;
    }
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
    for (int o = 16; o > 0; o >>= 1) {
        T u = __shfl_xor_sync(AHS_FULL_MASK, v, o);
        v = u > v ? u : v;
    }
    return v;
}
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(AHS_FULL_MASK, v, o);
    return v;
}

// Inclusive warp scan.
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v) {
    const uint32_t lane = lane_id();
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(AHS_FULL_MASK, v, o);
        if (lane >= (uint32_t)o) v += u;
    }
    return v;
}

// Block-wide exclusive scan of one value per thread (BLOCK threads, BLOCK/32
// warps <= 32).  scratch: BLOCK/32 + 1 elements of shared memory.  Returns the
// exclusive prefix; *total receives the block sum.  Contains __syncthreads.
template <int BLOCK, typename T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* scratch, T* total) {
    static_assert(BLOCK % 32 == 0 && BLOCK / 32 <= 32, "block size");
    constexpr int W = BLOCK / 32;
    const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
    T inc = warp_inclusive_scan(v);
    if (lane == 31) scratch[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T s = lane < (uint32_t)W ? scratch[lane] : T(0);
        T si = warp_inclusive_scan(s);
        if (lane < (uint32_t)W) scratch[lane] = si - s;
        if (lane == W - 1) scratch[W] = si;
    }
    __syncthreads();
    T r = scratch[warp] + inc - v;
    *total = scratch[W];
    __syncthreads();
    return r;
}

// Exclusive scan of NB per-digit counts with a block of BLOCK threads, for
// any BLOCK (each thread owns NB / BLOCK consecutive digits when NB >= BLOCK).
// start[d] = sum of count[d'] for d' < d.  Ends with __syncthreads, so start
// is visible to the whole block on return.
template <int BLOCK, int NB>
__device__ __forceinline__ void scan_digit_counts(const uint32_t* count, uint32_t* start,
                                                  uint32_t* scratch) {
    constexpr int PER = NB >= BLOCK ? NB / BLOCK : 1;
    static_assert(NB < BLOCK || NB % BLOCK == 0, "digit count must divide evenly");
    const uint32_t tid = threadIdx.x;
    uint32_t loc[PER];
    uint32_t sum = 0;
    if constexpr (NB >= BLOCK) {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            loc[r] = count[tid * PER + r];
            sum += loc[r];
        }
    } else {
        sum = tid < (uint32_t)NB ? count[tid] : 0u;
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<BLOCK>(sum, scratch, &total);
    if constexpr (NB >= BLOCK) {
#pragma unroll
        for (int r = 0; r < PER; ++r) {
            start[tid * PER + r] = run;
            run += loc[r];
        }
    } else {
        if (tid < (uint32_t)NB) start[tid] = run;
    }
    __syncthreads();
}

// Relaxed GPU-scope 32-bit load/store used for look-back status words: the
// flag and the count share one word, so a single access is all-or-nothing.
__device__ __forceinline__ uint32_t ld_relaxed_gpu(const uint32_t* p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_gpu(uint32_t* p, uint32_t v) {
    asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void report_error(uint32_t* err, uint32_t code) {
    if (err) atomicCAS(err, 0u, code);
}

__host__ __device__ __forceinline__ uint32_t bitlen64(uint64_t x) {
#ifdef __CUDA_ARCH__
    return x ? 64u - (uint32_t)__clzll((long long)x) : 0u;
#else
    return x ? 64u - (uint32_t)__builtin_clzll(x) : 0u;
#endif
}

__host__ __device__ __forceinline__ uint64_t ceil_div(uint64_t a, uint64_t b) {
    return (a + b - 1) / b;
}

}  // namespace ahs
