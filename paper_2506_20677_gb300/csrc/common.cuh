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
    kDevCopyTimeout = 4,       // a bulk-async copy did not complete
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
// 32-bit unsigned reductions in one warp-wide instruction.
template <>
__device__ __forceinline__ uint32_t warp_min<uint32_t>(uint32_t v) {
    return __reduce_min_sync(AHS_FULL_MASK, v);
}
template <>
__device__ __forceinline__ uint32_t warp_max<uint32_t>(uint32_t v) {
    return __reduce_max_sync(AHS_FULL_MASK, v);
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
// any BLOCK: thread t owns the PER = ceil(NB / BLOCK) consecutive digits from
// t * PER (threads past the end own none).  start[d] = sum of count[d'] for
// d' < d.  Ends with __syncthreads, so start is visible to the whole block on
// return.
template <int BLOCK, int NB>
__device__ __forceinline__ void scan_digit_counts(const uint32_t* count, uint32_t* start,
                                                  uint32_t* scratch) {
    constexpr int PER = (NB + BLOCK - 1) / BLOCK;
    const uint32_t tid = threadIdx.x;
    uint32_t loc[PER];
    uint32_t sum = 0;
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t d = tid * PER + r;
        loc[r] = d < (uint32_t)NB ? count[d] : 0u;
        sum += loc[r];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<BLOCK>(sum, scratch, &total);
#pragma unroll
    for (int r = 0; r < PER; ++r) {
        const uint32_t d = tid * PER + r;
        if (d < (uint32_t)NB) start[d] = run;
        run += loc[r];
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

// ------------------------------------------------------------------ bulk-async copies
// One-dimensional bulk copies (cp.async.bulk, the TMA engine) from global into
// shared memory, completed on an mbarrier that counts the bytes delivered.
// Source, destination and size must be multiples of 16 bytes.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gmem_src, uint32_t bytes,
                                          uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(smem_dst)),
        "l"(gmem_src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// later bulk-async writes into the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Wait for phase `parity` of the barrier; gives up after ~2^22 polls (seconds)
// and returns false, so a lost copy can never hang the GPU.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    for (uint32_t spin = 0; spin < (1u << 22); ++spin) {
        uint32_t done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// Asynchronous 4- or 8-byte global -> shared copy (cp.async), for the few
// keys of a run that bulk copies cannot move; completed by cp_async_wait_all
// in the issuing thread.
template <typename K>
__device__ __forceinline__ void cp_async_key(K* smem_dst, const K* gmem_src) {
    static_assert(sizeof(K) == 4 || sizeof(K) == 8, "4- or 8-byte keys");
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(smem_addr(smem_dst)),
                 "l"(gmem_src), "n"(sizeof(K))
                 : "memory");
}
// Asynchronous 16-byte global -> shared copy (both addresses 16-byte aligned).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(smem_dst)), "l"(gmem_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Wait until at most one (the most recent) cp.async group is pending.
__device__ __forceinline__ void cp_async_wait_prior() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// Split of a run of `size` keys at p into a head before the first 16-byte
// boundary, a body that bulk copies can move and a tail.  In a shared-memory
// buffer whose base is 16-byte aligned, key i of the run goes to
// buf[pad + i]: the body then starts 16-byte aligned.  The buffer needs
// size + 16 / sizeof(K) elements.
template <typename K>
struct TileSplit {
    uint32_t head, body, pad;
    __device__ __forceinline__ TileSplit(const K* p, uint32_t size) {
        constexpr uint32_t V = 16 / sizeof(K);
        const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(p) & 15u) / sizeof(K));
        head = mis ? V - mis : 0;
        if (head > size) head = size;
        body = ((size - head) / V) * V;
        pad = (V - head % V) % V;
    }
};

// One thread: start moving a run of `size` keys at src into buf (key i at
// buf[pad + i]): the body by a bulk copy completing on `bar` (which gets this
// thread's arrival either way), head and tail by cp.async as one commit group
// (the same thread waits for it before the block reads the buffer).
template <typename K>
__device__ __forceinline__ void issue_run(K* buf, const K* src, uint32_t size, uint64_t* bar,
                                          uint32_t extra_tx = 0) {
    const TileSplit<K> sp(src, size);
    for (uint32_t i = 0; i < sp.head; ++i) cp_async_key(&buf[sp.pad + i], src + i);
    for (uint32_t i = sp.head + sp.body; i < size; ++i) cp_async_key(&buf[sp.pad + i], src + i);
    cp_async_commit();
    const uint32_t tx = sp.body * (uint32_t)sizeof(K) + extra_tx;
    if (tx) mbar_arrive_expect_tx(bar, tx);
    else mbar_arrive(bar);
    if (sp.body) bulk_load(&buf[sp.pad + sp.head], src + sp.head, sp.body * (uint32_t)sizeof(K), bar);
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
