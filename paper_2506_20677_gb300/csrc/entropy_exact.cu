// Exact per-value entropy on the device (Section III-A): H = -sum over the
// distinct key values v of p_v log2 p_v, p_v = (keys equal to v) / n, and the
// number of distinct values k'.  The feature pass's histogram has 2^16 bins,
// so its entropy equals this one only for k <= 2^16; this mode sorts a copy
// of the keys with the library's own sort, then measures the runs of equal
// keys in the sorted copy.
//
// Runs: the thread at a run's first element finds its end by galloping then
// binary search (O(log c) reads for a run of c keys), so a heavy value costs
// no more than a short one.  Terms -(c/n) log2(c/n) are grouped by run length
// below kCocMax (count of counts, one fp64 log per distinct length) and
// evaluated directly above it.
#include <algorithm>
#include <cstring>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kRunThreads = 256;
constexpr uint32_t kCocMax = 4096;
constexpr uint32_t kRunItems = 8;      // elements per thread per block step

struct ExactRec {
    unsigned long long distinct;
    unsigned long long coc[kCocMax];   // runs of each length below kCocMax
    double big;                        // sum of the terms of longer runs
    double entropy;
    uint32_t done;
};

template <typename K>
__device__ __forceinline__ uint64_t run_end(const K* a, uint64_t n, uint64_t i) {
    const K x = a[i];
    // gallop: a[i + step - 1] == x for the last good step
    uint64_t lo = i + 1, step = 1;   // invariant: a[lo - 1] == x
    while (true) {
        const uint64_t probe = i + step;
        if (probe >= n || a[probe] != x) break;
        lo = probe + 1;
        step <<= 1;
    }
    uint64_t hi = i + step < n ? i + step : n;   // a[hi] != x or hi == n
    while (lo < hi) {                             // first index in [lo, hi) with a[j] != x
        const uint64_t mid = lo + (hi - lo) / 2;
        if (a[mid] == x) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

template <typename K>
__global__ void __launch_bounds__(kRunThreads)
runs_entropy(const K* __restrict__ a, uint64_t n, ExactRec* __restrict__ rec) {
    __shared__ uint32_t coc[kCocMax];
    __shared__ double s_big[kRunThreads / 32];
    __shared__ unsigned long long s_cnt[kRunThreads / 32];
    for (uint32_t i = threadIdx.x; i < kCocMax; i += kRunThreads) coc[i] = 0;
    __syncthreads();
    double big = 0.0;
    unsigned long long starts = 0;
    const double dn = (double)n;
    const uint64_t per_block = (uint64_t)kRunThreads * kRunItems;
    for (uint64_t base = (uint64_t)blockIdx.x * per_block; base < n; base += (uint64_t)gridDim.x * per_block) {
#pragma unroll
        for (uint32_t r = 0; r < kRunItems; ++r) {
            const uint64_t i = base + (uint64_t)r * kRunThreads + threadIdx.x;
            if (i >= n || (i > 0 && a[i] == a[i - 1])) continue;
            const uint64_t c = run_end(a, n, i) - i;
            ++starts;
            if (c < kCocMax) {
                atomicAdd(&coc[c], 1u);
            } else {
                const double p = (double)c / dn;
                big -= p * log2(p);
            }
        }
    }
    big = warp_sum(big);
    starts = warp_sum(starts);
    if (lane_id() == 0) {
        s_big[threadIdx.x >> 5] = big;
        s_cnt[threadIdx.x >> 5] = starts;
    }
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < kCocMax; c += kRunThreads)
        if (coc[c]) atomicAdd(&rec->coc[c], (unsigned long long)coc[c]);
    if (threadIdx.x == 0) {
        double b = 0.0;
        unsigned long long k = 0;
        for (int w = 0; w < kRunThreads / 32; ++w) {
            b += s_big[w];
            k += s_cnt[w];
        }
        atomicAdd(&rec->big, b);
        atomicAdd(&rec->distinct, k);
    }
}

// One block: H = sum over lengths c of coc[c] * (-(c/n) log2(c/n)) + big.
__global__ void __launch_bounds__(kRunThreads)
runs_entropy_final(uint64_t n, ExactRec* __restrict__ rec) {
    __shared__ double s_part[kRunThreads / 32];
    double h = 0.0;
    const double dn = (double)n;
    for (uint32_t c = threadIdx.x + 1; c < kCocMax; c += kRunThreads) {
        const unsigned long long m = rec->coc[c];
        if (m) {
            const double p = (double)c / dn;
            h += (double)m * (-p * log2(p));
        }
    }
    h = warp_sum(h);
    if (lane_id() == 0) s_part[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = rec->big;
        for (int w = 0; w < kRunThreads / 32; ++w) t += s_part[w];
        rec->entropy = t;
    }
}

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace
}  // namespace ahs

using namespace ahs;

extern "C" ahs_status ahs_entropy_exact(ahs_ctx* ctx, const void* d_keys, uint64_t n,
                                        ahs_key_type type, void* stream, double* h_entropy,
                                        uint64_t* h_distinct) {
    if (!ctx || ctx->device < 0 || !h_entropy || !h_distinct) return AHS_ERR_INVALID_ARG;
    if (type < AHS_U32 || type > AHS_I64) return AHS_ERR_DTYPE;
    if (n && !d_keys) return AHS_ERR_INVALID_ARG;
    *h_entropy = 0.0;
    *h_distinct = 0;
    if (n == 0) return AHS_OK;
    if (n > 0xffffffffull) return AHS_ERR_RANGE;
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const KeyDesc kd = key_desc(type);
    TracerGuard tg(&ctx->tracer);
    // The sorted copy and the record live in the context's side buffer.
    const size_t need = a256(n * kd.bytes) + a256(sizeof(ExactRec));
    if (need > ctx->side_bytes) {
        if (ctx->side) cudaFree(ctx->side);
        ctx->side = nullptr;
        ctx->side_bytes = 0;
        e = cudaMalloc(&ctx->side, need);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return cuda_status(ctx, e);
        }
        ctx->side_bytes = need;
    }
    void* sorted = ctx->side;
    ExactRec* rec = reinterpret_cast<ExactRec*>(static_cast<char*>(ctx->side) + a256(n * kd.bytes));
    // Sort the copy with the AUTO pipeline of the context's profile.
    ahs_features_t f;
    ahs_status rc = run_features(ctx, d_keys, n, kd, st, &f, sorted_identity(ctx) ? kSkipOrdered : 0u);
    if (rc != AHS_OK) return rc;
    uint32_t passes = 0, buckets = 0;
    rc = run_strategy(ctx, choose(ctx, f, kd.bytes, false), d_keys, sorted, nullptr, nullptr, n, kd,
                      f, st, &passes, &buckets);
    if (rc != AHS_OK) return rc;
    rc = check_device_error(ctx, st);
    if (rc != AHS_OK) return rc;
    e = cudaMemsetAsync(rec, 0, sizeof(ExactRec), st);
    const uint32_t grid = (uint32_t)std::min<uint64_t>(ceil_div(n, (uint64_t)kRunThreads * kRunItems),
                                                       8ull * (uint64_t)ctx->sms);
    if (e == cudaSuccess) {
        TraceScope ts("entropy_exact_runs", n, st);
        if (kd.bytes == 4) runs_entropy<uint32_t><<<grid, kRunThreads, 0, st>>>(
            static_cast<const uint32_t*>(sorted), n, rec);
        else runs_entropy<uint64_t><<<grid, kRunThreads, 0, st>>>(
            static_cast<const uint64_t*>(sorted), n, rec);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        runs_entropy_final<<<1, kRunThreads, 0, st>>>(n, rec);
        e = cudaGetLastError();
    }
    double h = 0.0;
    unsigned long long k = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, &rec->entropy, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&k, &rec->distinct, sizeof(k), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    *h_entropy = h;
    *h_distinct = k;
    return AHS_OK;
}
