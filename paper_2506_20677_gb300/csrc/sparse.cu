// Keys-only radix path for inputs with few distinct values.
//
// Section III-D sends wide-range, low-entropy inputs to radix sort.  Without
// a payload the sorted output of such an input is fixed by its distinct
// values and their counts alone, so when they fit a table the sort is the
// counting sort of Section III-C over a sparse set of values:
//   1. one read of the keys counts every distinct value in a per-CTA hash
//      table in shared memory, merged into one table in global memory;
//   2. each distinct value's rank among the others and the count of keys
//      below it give its run [start, start + count) of the output;
//   3. the output is written run by run (the counting fill), without reading
//      the keys again.
// A table that overflows (more distinct values than it holds) marks the
// attempt failed; the fill then writes nothing and the caller sorts by the
// histogram-guided partition passes instead.
#include <cstring>

#include "common.cuh"
#include "ctx.h"
#include "internal.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kSpThreads = 512;
constexpr int kSpUnroll = 2;
constexpr uint32_t kSpLocalLg = 12;   // 4,096 slots per CTA
constexpr uint32_t kSpLocal = 1u << kSpLocalLg;
constexpr uint32_t kSpGlobalLg = 13;   // 8,192 slots in the merged table
constexpr uint32_t kSpGlobal = 1u << kSpGlobalLg;
constexpr uint32_t kSpMaxProbe = 64;   // linear probes before a table counts as full
constexpr int kRankThreads = 256;
constexpr uint32_t kRankSplit = 8;   // CTAs that share one entry's comparisons

size_t a256(size_t x) { return (x + 255) & ~size_t(255); }

// Status words: [0] failure (1: a table was full, 2: the counts do not add up
// to n), [1] distinct values m.
constexpr uint32_t kStatusWords = 4;

// Fibonacci hashing (Knuth, TAOCP vol. 3, 6.4): the top lg bits of u times
// 2^w / phi.
__device__ __forceinline__ uint32_t sp_hash(uint32_t u, uint32_t lg) {
    return (u * 0x9E3779B1u) >> (32 - lg);
}
__device__ __forceinline__ uint32_t sp_hash(uint64_t u, uint32_t lg) {
    return (uint32_t)((u * 0x9E3779B97F4A7C15ull) >> (64 - lg));
}
__device__ __forceinline__ uint32_t sp_cas(uint32_t* p, uint32_t cmp, uint32_t val) {
    return atomicCAS(p, cmp, val);
}
__device__ __forceinline__ uint64_t sp_cas(uint64_t* p, uint64_t cmp, uint64_t val) {
    return (uint64_t)atomicCAS(reinterpret_cast<unsigned long long*>(p), (unsigned long long)cmp,
                               (unsigned long long)val);
}

// Slot of `key` (!= 0) in an open-addressed table of 2^LG slots (0 = empty),
// claimed if absent, plus kFresh when this call claimed it; -1 when
// kSpMaxProbe slots in a row hold other values.
constexpr int kFresh = 1 << 30;
template <typename K, uint32_t LG>
__device__ __forceinline__ int sp_slot(K* tab, K key) {
    static_assert(LG < 30, "slot and flag share an int");
    uint32_t h = sp_hash(key, LG);
    for (uint32_t p = 0; p < kSpMaxProbe; ++p) {
        K k = *reinterpret_cast<volatile K*>(&tab[h]);
        if (k == 0) {
            k = sp_cas(&tab[h], (K)0, key);
            if (k == 0) return (int)h | kFresh;
        }
        if (k == key) return (int)h;
        h = (h + 1) & ((1u << LG) - 1);
    }
    return -1;
}

// Step 1.  Keys are stored as u + 1, u = ord(x) - min (the caller checks
// that the span is below the largest K, so no key is 0).  list[i] is the
// merged table's slot of the i-th distinct value to arrive.
template <typename K>
__global__ void __launch_bounds__(kSpThreads, 2)
sp_count(const K* __restrict__ keys, uint64_t n, K flip, K mn, uint64_t head, uint64_t nvec,
         K* __restrict__ gkey, uint32_t* __restrict__ gcnt, uint32_t* __restrict__ list,
         uint32_t* __restrict__ status) {
    constexpr int V = Vec16<K>::kN;
    constexpr uint64_t kChunk = (uint64_t)kSpThreads * kSpUnroll;   // vectors
    __shared__ K skey[kSpLocal];
    __shared__ uint32_t scnt[kSpLocal];
    __shared__ uint32_t s_fail;
    for (uint32_t i = threadIdx.x; i < kSpLocal; i += kSpThreads) {
        skey[i] = 0;
        scnt[i] = 0;
    }
    if (threadIdx.x == 0) s_fail = 0;
    __syncthreads();
    const uint32_t lane = lane_id();
    // Once a CTA's table holds a value, nearly every later key of that value
    // finds it at its first slot: the keys of a batch are looked up there
    // together (independent loads; a stale read only sends a key to the
    // probing path, since a filled slot never changes), and only the rest
    // probe and claim slots one by one.
    auto slow = [&](K key) {
        const int h = sp_slot<K, kSpLocalLg>(skey, key);
        if (h < 0) s_fail = 1;
        else atomicAdd(&scnt[h & (kFresh - 1)], 1u);
    };
    auto encode = [&](K x) { return (K)((K)((K)(x ^ flip) - mn) + 1); };
    if (blockIdx.x == 0) {   // head and tail: fewer than V keys each
        const uint64_t tail0 = head + nvec * V, nt = n - tail0;
        if (threadIdx.x < head) slow(encode(keys[threadIdx.x]));
        if (threadIdx.x < nt) slow(encode(keys[tail0 + threadIdx.x]));
    }
    const K* body = keys + head;
    const uint64_t nchunks = ceil_div(nvec, kChunk);
    constexpr int B = kSpUnroll * V;
    // The next chunk's vectors are loaded before this chunk's keys are
    // counted, so that the loads stay in flight while the table works.
    auto load = [&](uint64_t c, Vec16<K> (&x)[kSpUnroll], bool (&ok)[kSpUnroll]) {
#pragma unroll
        for (int u = 0; u < kSpUnroll; ++u) {
            const uint64_t v = c * kChunk + (uint64_t)u * kSpThreads + threadIdx.x;
            ok[u] = c < nchunks && v < nvec;
            if (ok[u]) x[u] = load_vec16_stream(body + v * V);
        }
    };
    Vec16<K> xn[kSpUnroll];
    bool okn[kSpUnroll];
    load(blockIdx.x, xn, okn);
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        // Stop early once any table is full (the result is discarded then).
        uint32_t stop = 0;
        if (lane == 0) stop = *reinterpret_cast<volatile uint32_t*>(&s_fail) |
                              *reinterpret_cast<volatile uint32_t*>(&status[0]);
        if (__shfl_sync(AHS_FULL_MASK, stop, 0)) break;
        Vec16<K> x[kSpUnroll];
        bool ok[kSpUnroll];
#pragma unroll
        for (int u = 0; u < kSpUnroll; ++u) {
            x[u] = xn[u];
            ok[u] = okn[u];
        }
        load(c + gridDim.x, xn, okn);
        K key[B];
        uint32_t h[B];
#pragma unroll
        for (int u = 0; u < kSpUnroll; ++u)
#pragma unroll
            for (int e = 0; e < V; ++e) {
                key[u * V + e] = ok[u] ? encode(x[u].e[e]) : (K)0;
                h[u * V + e] = sp_hash(key[u * V + e], kSpLocalLg);
            }
        // The home slot and the next one (where a value lands when its home
        // was taken first) are read together.
        K at0[B], at1[B];
#pragma unroll
        for (int i = 0; i < B; ++i) {
            at0[i] = skey[h[i]];
            at1[i] = skey[(h[i] + 1) & (kSpLocal - 1)];
        }
#pragma unroll
        for (int i = 0; i < B; ++i) {
            if (key[i] == 0) continue;   // past the end
            const bool hit0 = at0[i] == key[i];
            if (hit0 || at1[i] == key[i])
                atomicAdd(&scnt[hit0 ? h[i] : (h[i] + 1) & (kSpLocal - 1)], 1u);
            else
                slow(key[i]);
        }
    }
    __syncthreads();
    if (s_fail) {
        if (threadIdx.x == 0) atomicExch(&status[0], 1u);
        return;
    }
    // Merge into the global table.
    for (uint32_t i = threadIdx.x; i < kSpLocal; i += kSpThreads) {
        const K key = skey[i];
        if (key == 0) continue;
        const int hf = sp_slot<K, kSpGlobalLg>(gkey, key);
        if (hf < 0) {
            atomicExch(&status[0], 1u);
            continue;
        }
        const uint32_t h = (uint32_t)(hf & (kFresh - 1));
        if (hf & kFresh) {
            const uint32_t idx = atomicAdd(&status[1], 1u);   // < kSpGlobal: one per slot
            if (AHS_DCHECK(idx < kSpGlobal, "sparse list", idx)) list[idx] = h;
        }
        atomicAdd(&gcnt[h], scnt[i]);
    }
}

// Step 2a.  For distinct value i (blockIdx.x * 256 + threadIdx.x < m): how
// many values, and how many keys, lie below it among the entries of the
// blockIdx.y-th part of the list.
template <typename K>
__global__ void __launch_bounds__(kRankThreads)
sp_rank(const K* __restrict__ gkey, const uint32_t* __restrict__ gcnt,
        const uint32_t* __restrict__ list, const uint32_t* __restrict__ status,
        uint32_t* __restrict__ rank, unsigned long long* __restrict__ below) {
    if (status[0] != 0) return;
    const uint32_t m = status[1];
    if (blockIdx.x * kRankThreads >= m) return;   // block-uniform
    __shared__ K tk[kRankThreads];
    __shared__ uint32_t tc[kRankThreads];
    const uint32_t i = blockIdx.x * kRankThreads + threadIdx.x;
    const K mine = i < m ? gkey[list[i]] : (K)0;
    const uint32_t per = (m + kRankSplit - 1) / kRankSplit;
    const uint32_t j0 = blockIdx.y * per, j1 = j0 + per < m ? j0 + per : m;
    uint32_t r = 0;
    unsigned long long s = 0;
    for (uint32_t t0 = j0; t0 < j1; t0 += kRankThreads) {
        __syncthreads();
        const uint32_t j = t0 + threadIdx.x;
        if (j < j1) {
            const uint32_t h = list[j];
            tk[threadIdx.x] = gkey[h];
            tc[threadIdx.x] = gcnt[h];
        }
        __syncthreads();
        const uint32_t cnt = j1 - t0 < (uint32_t)kRankThreads ? j1 - t0 : (uint32_t)kRankThreads;
        for (uint32_t q = 0; q < cnt; ++q) {
            const bool lt = tk[q] < mine;
            r += lt ? 1u : 0u;
            s += lt ? tc[q] : 0u;
        }
    }
    if (i < m) {
        if (r) atomicAdd(&rank[i], r);
        if (s) atomicAdd(&below[i], s);
    }
}

// Step 2b.  Run rank[i] holds value u_i at [below[i], below[i] + count_i);
// prefix[m] closes the last run and must equal n.
template <typename K>
__global__ void __launch_bounds__(kRankThreads)
sp_place(const K* __restrict__ gkey, const uint32_t* __restrict__ gcnt,
         const uint32_t* __restrict__ list, uint32_t* __restrict__ status,
         const uint32_t* __restrict__ rank, const unsigned long long* __restrict__ below,
         K* __restrict__ vals, unsigned long long* __restrict__ prefix, uint64_t n,
         uint32_t* __restrict__ err) {
    if (status[0] != 0) return;
    const uint32_t m = status[1];
    const uint32_t i = blockIdx.x * kRankThreads + threadIdx.x;
    if (i >= m) return;
    const uint32_t h = list[i], r = rank[i];
    if (!AHS_DCHECK(r < m, "sparse rank", r)) return;
    vals[r] = gkey[h] - 1;
    prefix[r] = below[i];
    if (r == m - 1) {
        const unsigned long long end = below[i] + gcnt[h];
        prefix[m] = end;
        if (end != n) {   // the counts do not describe these keys: no fill
            atomicExch(&status[0], 2u);
            report_error(err, kDevBadState);
        }
    }
}

template <typename K>
size_t sp_layout(size_t* o_key, size_t* o_cnt, size_t* o_list, size_t* o_rank, size_t* o_below,
                 size_t* o_status, size_t* zero_end, size_t* o_vals, size_t* o_prefix) {
    size_t o = 0;
    *o_key = o;    o += a256(kSpGlobal * sizeof(K));
    *o_cnt = o;    o += a256(kSpGlobal * 4);
    *o_rank = o;   o += a256(kSpGlobal * 4);
    *o_below = o;  o += a256(kSpGlobal * 8);
    *o_status = o; o += a256(kStatusWords * 4);
    *zero_end = o;
    *o_list = o;   o += a256(kSpGlobal * 4);
    *o_vals = o;   o += a256(kSpGlobal * sizeof(K));
    *o_prefix = o; o += a256((kSpGlobal + 1) * 8);
    return o;
}

template <typename K>
ahs_status sparse_t(ahs_ctx* ctx, const K* kin, K* kout, uint64_t n, K flip, K mn, cudaStream_t st,
                    bool* done, uint32_t* distinct) {
    size_t o_key, o_cnt, o_list, o_rank, o_below, o_status, zero_end, o_vals, o_prefix;
    const size_t bytes = sp_layout<K>(&o_key, &o_cnt, &o_list, &o_rank, &o_below, &o_status,
                                      &zero_end, &o_vals, &o_prefix);
    ahs_status rc = ensure_aux(ctx, bytes);
    if (rc == AHS_OK) rc = ensure_stage(ctx, kStatusWords * 4);
    if (rc != AHS_OK) return rc;
    char* a = static_cast<char*>(ctx->aux);
    K* gkey = reinterpret_cast<K*>(a + o_key);
    uint32_t* gcnt = reinterpret_cast<uint32_t*>(a + o_cnt);
    uint32_t* list = reinterpret_cast<uint32_t*>(a + o_list);
    uint32_t* rank = reinterpret_cast<uint32_t*>(a + o_rank);
    unsigned long long* below = reinterpret_cast<unsigned long long*>(a + o_below);
    uint32_t* status = reinterpret_cast<uint32_t*>(a + o_status);
    K* vals = reinterpret_cast<K*>(a + o_vals);
    unsigned long long* prefix = reinterpret_cast<unsigned long long*>(a + o_prefix);

    cudaError_t e = launch_zero32(a, zero_end / 4, ctx->sms, st);
    constexpr int V = Vec16<K>::kN;
    const uint64_t head = head_elems<K>(kin, n);
    const uint64_t nvec = (n - head) / V;
    if (e == cudaSuccess) {
        const uint64_t chunks = ceil_div(nvec, (uint64_t)kSpThreads * kSpUnroll);
        const uint64_t cap = 2ull * (uint64_t)ctx->sms;
        const uint32_t g = (uint32_t)(chunks < 1 ? 1 : (chunks < cap ? chunks : cap));
        TraceScope ts("sparse_count", n, st);
        sp_count<K><<<g, kSpThreads, 0, st>>>(kin, n, flip, mn, head, nvec, gkey, gcnt, list, status);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        TraceScope ts("sparse_rank", 0, st);
        sp_rank<K><<<dim3(kSpGlobal / kRankThreads, kRankSplit), kRankThreads, 0, st>>>(
            gkey, gcnt, list, status, rank, below);
        sp_place<K><<<kSpGlobal / kRankThreads, kRankThreads, 0, st>>>(
            gkey, gcnt, list, status, rank, below, vals, prefix, n, ctx->d_err);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
        KeyDesc kd;
        kd.bytes = sizeof(K);
        kd.flip = flip;
        e = launch_sparse_fill(kout, n, kd, prefix, vals, status, (uint64_t)mn, ctx->sms, st);
    }
    // The outcome decides whether the caller sorts another way.
    if (e == cudaSuccess) e = launch_transfer(ctx->h_stage, status, kStatusWords * 4, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(ctx, e);
    uint32_t hs[kStatusWords];
    std::memcpy(hs, ctx->h_stage, sizeof(hs));
    *done = hs[0] == 0;
    *distinct = hs[1];
    return AHS_OK;
}

}  // namespace

bool sparse_radix_fits(uint64_t n, uint32_t key_bytes, uint64_t span, const HistView& hist) {
    if (n < kSparseMinKeys || n > 0xffffffffull) return false;
    const uint64_t kmax = key_bytes == 4 ? 0xffffffffull : ~0ull;
    if (span >= kmax) return false;   // u + 1 must not wrap to 0
    uint32_t nonzero = 0;
    for (uint32_t b = 0; b < hist.nbins; ++b) nonzero += hist.counts[b] ? 1u : 0u;
    return nonzero <= kSparseMaxBins;
}

ahs_status run_sparse_radix(ahs_ctx* ctx, const void* kin, void* kout, uint64_t n, KeyDesc kd,
                            uint64_t min_ord, cudaStream_t st, bool* done, uint32_t* distinct) {
    *done = false;
    *distinct = 0;
    if (kd.bytes == 4)
        return sparse_t<uint32_t>(ctx, static_cast<const uint32_t*>(kin), static_cast<uint32_t*>(kout),
                                  n, (uint32_t)kd.flip, (uint32_t)min_ord, st, done, distinct);
    return sparse_t<uint64_t>(ctx, static_cast<const uint64_t*>(kin), static_cast<uint64_t*>(kout), n,
                              kd.flip, min_ord, st, done, distinct);
}

}  // namespace ahs
