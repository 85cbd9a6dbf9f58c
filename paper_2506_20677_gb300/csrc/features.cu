// Feature extraction: the state vector v = (n, k, H) of Section III-A.
//
//  K1  k1_minmax_descents  one read of the keys: min / max of the order-
//                          preserving image, and the count of descents
//                          (key[i] > key[i+1]); last block reduces the
//                          per-block partials and fixes the histogram binning.
//  K2  k2_histogram        one read of the keys: c_j = #{x : (ord(x)-min) >> s == j}
//                          in shared memory (<= 2^16 bins), one CTA per SM,
//                          flushed to a per-CTA slab in global memory.
//  K3  k3_entropy          sums the slabs into the exact u64 histogram and
//                          reduces H = -sum_j (c_j/n) log2(c_j/n) in fp64.
#include "common.cuh"
#include "internal.h"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kK1Threads = 512;
template <typename K>
struct K1Unroll { static constexpr int kU = 4; };
// 64-bit keys: two vectors in flight per thread keep the counters and the
// neighbours' keys in registers (three or four spill).
template <>
struct K1Unroll<uint64_t> { static constexpr int kU = 2; };
constexpr int kK2Unroll = 4;
// Up to this many bins K3 gives each bin a warp's lanes in eight warps that
// split the slabs, instead of one thread per bin walking every slab: with few
// bins that walk is a chain of L2 latencies on a handful of threads.
constexpr uint32_t kK3DirectBins = 4096;
constexpr uint32_t kU32Bins = kHistSmemBytes / 4;           // bins that fit as u32 counters

template <typename K>
__device__ __forceinline__ void k1_scalar(const K* keys, uint64_t i, uint64_t n, K flip, K& mn,
                                          K& mx, unsigned long long& desc, unsigned long long& asc) {
    const K o = keys[i] ^ flip;
    mn = o < mn ? o : mn;
    mx = o > mx ? o : mx;
    if (i + 1 < n) {
        const K on = (K)(keys[i + 1] ^ flip);
        desc += (o > on) ? 1ull : 0ull;
        asc += (o < on) ? 1ull : 0ull;
    }
}

// An input K1 found presorted under the caller's skip flags: K2 and K3 have
// nothing to do (block-uniform).
__device__ __forceinline__ bool presorted_skip(const DevFeatures* rec, uint32_t flags) {
    return ((flags & kSkipOrdered) && rec->descents == 0) ||
           ((flags & kSkipReversed) && rec->ascents == 0) ||
           ((flags & kSkipStrictReversed) && rec->n >= 2 && rec->descents == rec->n - 1);
}

template <typename K>
__global__ void __launch_bounds__(kK1Threads, 2)
k1_minmax_descents(const K* __restrict__ keys, uint64_t n, K flip, uint64_t head, uint64_t nvec,
                   unsigned long long* __restrict__ partials, DevFeatures* __restrict__ rec) {
    constexpr int V = Vec16<K>::kN;
    K mn = ~K(0), mx = 0;
    unsigned long long desc = 0, asc = 0;
    const uint32_t lane = lane_id();
    const uint64_t gtid = (uint64_t)blockIdx.x * kK1Threads + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * kK1Threads;

    // Elements before the first 16-byte boundary, and after the last full vector.
    const uint64_t tail0 = head + nvec * V;
    if (gtid < head) k1_scalar(keys, gtid, n, flip, mn, mx, desc, asc);
    if (gtid < n - tail0) k1_scalar(keys, tail0 + gtid, n, flip, mn, mx, desc, asc);

    // Vector body: each warp reads kK1Unroll * 32 consecutive vectors per
    // iteration (one contiguous stretch), vector u * 32 + lane to each lane, so
    // the pair that straddles two vectors is closed with a shuffle from the
    // next lane, or for lane 31 from lane 0's next vector.  The last lane of
    // the stretch (and the owner of the last vector) needs the next key from
    // memory: it is loaded together with the vectors so its latency overlaps
    // theirs.
    const K* body = keys + head;
    uint32_t dloc = 0, aloc = 0;   // descents, ascents of this thread (< 2^32 keys per thread)
    constexpr int kK1Unroll = K1Unroll<K>::kU;
    constexpr uint64_t kRun = 32ull * kK1Unroll;   // vectors of a warp's stretch
    const uint64_t nwarps = stride >> 5;
    for (uint64_t cb = (gtid >> 5) * kRun; cb < nvec; cb += nwarps * kRun) {
        Vec16<K> x[kK1Unroll];
        K first[kK1Unroll];
        K succ = K(0);
#pragma unroll
        for (int u = 0; u < kK1Unroll; ++u) {
            const uint64_t v = cb + (uint64_t)u * 32 + lane;
            if (v < nvec) x[u] = load_vec16_stream(body + v * V);
            const uint64_t e_next = head + (v + 1) * V;
            if (v < nvec && (v + 1 == nvec || (lane == 31 && u == kK1Unroll - 1)) && e_next < n)
                succ = keys[e_next];
        }
#pragma unroll
        for (int u = 0; u < kK1Unroll; ++u) {
            const uint64_t v = cb + (uint64_t)u * 32 + lane;
            first[u] = v < nvec ? (K)(x[u].e[0] ^ flip) : K(0);
        }
#pragma unroll
        for (int u = 0; u < kK1Unroll; ++u) {
            const uint64_t v = cb + (uint64_t)u * 32 + lane;
            const K down = __shfl_down_sync(AHS_FULL_MASK, first[u], 1);
            const K wrap = u + 1 < kK1Unroll ? __shfl_sync(AHS_FULL_MASK, first[u + 1 < kK1Unroll ? u + 1 : u], 0)
                                             : K(0);
            if (v < nvec) {
                K o[V];
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    o[j] = x[u].e[j] ^ flip;
                    mn = o[j] < mn ? o[j] : mn;
                    mx = o[j] > mx ? o[j] : mx;
                }
#pragma unroll
                for (int j = 0; j + 1 < V; ++j) {
                    dloc += (o[j] > o[j + 1]) ? 1u : 0u;
                    aloc += (o[j] < o[j + 1]) ? 1u : 0u;
                }
                if (head + (v + 1) * V < n) {
                    K on;
                    if (v + 1 == nvec) on = (K)(succ ^ flip);
                    else if (lane < 31) on = down;
                    else on = u + 1 < kK1Unroll ? wrap : (K)(succ ^ flip);
                    dloc += (o[V - 1] > on) ? 1u : 0u;
                    aloc += (o[V - 1] < on) ? 1u : 0u;
                }
            }
        }
    }
    desc += dloc;
    asc += aloc;

    // Block reduction.
    __shared__ unsigned long long s_min[kK1Threads / 32], s_max[kK1Threads / 32],
        s_desc[kK1Threads / 32], s_asc[kK1Threads / 32];
    __shared__ bool s_last;
    unsigned long long bmn = warp_min((unsigned long long)mn);
    unsigned long long bmx = warp_max((unsigned long long)mx);
    unsigned long long bd = warp_sum(desc);
    unsigned long long ba = warp_sum(asc);
    const uint32_t warp = threadIdx.x >> 5;
    if (lane == 0) { s_min[warp] = bmn; s_max[warp] = bmx; s_desc[warp] = bd; s_asc[warp] = ba; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kK1Threads / 32; ++w) {
            bmn = s_min[w] < bmn ? s_min[w] : bmn;
            bmx = s_max[w] > bmx ? s_max[w] : bmx;
            bd += s_desc[w];
            ba += s_asc[w];
        }
        partials[4 * blockIdx.x + 0] = bmn;
        partials[4 * blockIdx.x + 1] = bmx;
        partials[4 * blockIdx.x + 2] = bd;
        partials[4 * blockIdx.x + 3] = ba;
        __threadfence();
        const uint32_t ticket = atomicAdd(&rec->k1_done, 1u);
        s_last = (ticket == gridDim.x - 1);
    }
    __syncthreads();
    if (!s_last) return;

    // Last block: combine all blocks and fix the binning (Section III-A reading:
    // s = max(0, bitlen(span) - 16), nbins = (span >> s) + 1).
    unsigned long long gmn = ~0ull, gmx = 0, gd = 0, ga = 0;
    for (uint32_t b = threadIdx.x; b < gridDim.x; b += kK1Threads) {
        const unsigned long long a = __ldcg(partials + 4 * b + 0);
        const unsigned long long c = __ldcg(partials + 4 * b + 1);
        gmn = a < gmn ? a : gmn;
        gmx = c > gmx ? c : gmx;
        gd += __ldcg(partials + 4 * b + 2);
        ga += __ldcg(partials + 4 * b + 3);
    }
    gmn = warp_min(gmn);
    gmx = warp_max(gmx);
    gd = warp_sum(gd);
    ga = warp_sum(ga);
    if (lane == 0) { s_min[warp] = gmn; s_max[warp] = gmx; s_desc[warp] = gd; s_asc[warp] = ga; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < kK1Threads / 32; ++w) {
            gmn = s_min[w] < gmn ? s_min[w] : gmn;
            gmx = s_max[w] > gmx ? s_max[w] : gmx;
            gd += s_desc[w];
            ga += s_asc[w];
        }
        const unsigned long long span = gmx - gmn;
        const uint32_t bl = bitlen64(span);
        const uint32_t s = bl > 16 ? bl - 16 : 0;
        rec->min_ord = gmn;
        rec->max_ord = gmx;
        rec->descents = gd;
        rec->ascents = ga;
        rec->k2_wrapped = 0;
        rec->n = n;
        rec->span = span;
        rec->shift = s;
        rec->nbins = (uint32_t)((span >> s) + 1);
        rec->k1_done = 0;
    }
}

// K2: per-CTA shared-memory histograms of u32 counters, flushed to per-slab
// counts in global memory.  Two layouts, chosen on the device from nbins:
//  - nbins <= kU32Bins (43,692): every CTA counts all bins of the keys it
//    reads, in R copies (warp w uses copy w % R) that spread the same-bin
//    atomics of skewed inputs; one slab per CTA.
//  - larger (up to 65,536 bins), input in runs: the two CTAs of a cluster
//    read the same chunks and each counts only its half of the bins (32,768
//    u32 counters, 128 KB), so no counter needs more than 32 bits and no
//    atomic is wider than 32 bits; the second read of a chunk is served by
//    L2.  One slab per cluster.
//  - larger, input not in runs: the packed layout (k2_packed below).
template <typename K>
__device__ __forceinline__ void k2_load(const K* __restrict__ body, uint64_t c, uint64_t nvec,
                                        Vec16<K> (&x)[kK2Unroll], bool (&ok)[kK2Unroll]) {
    constexpr uint64_t kChunkVecs = (uint64_t)kHistThreads * kK2Unroll;
#pragma unroll
    for (int u = 0; u < kK2Unroll; ++u) {
        const uint64_t v = c * kChunkVecs + (uint64_t)u * kHistThreads + threadIdx.x;
        ok[u] = v < nvec;
        if (ok[u]) x[u] = load_vec16(body + v * Vec16<K>::kN);
    }
}

template <typename K>
__device__ __forceinline__ void k2_replicated(const K* __restrict__ keys, uint64_t n, K flip,
                                              uint64_t head, uint64_t nvec, K mn, uint32_t s,
                                              uint32_t nb, uint32_t* __restrict__ slabs,
                                              uint32_t* sm) {
    constexpr int V = Vec16<K>::kN;
    constexpr uint64_t kChunkVecs = (uint64_t)kHistThreads * kK2Unroll;
    uint32_t R = kU32Bins / nb;
    R = R > 32 ? 32 : R;
    for (uint32_t i = threadIdx.x; i < R * nb; i += kHistThreads) sm[i] = 0;
    __syncthreads();
    uint32_t* mine = sm + ((threadIdx.x >> 5) % R) * nb;
    auto add = [&](K x) {
        const uint32_t bin = (uint32_t)(((K)(x ^ flip) - mn) >> s);
        if (AHS_DCHECK(bin < nb, "k2 bin", bin)) atomicAdd(&mine[bin], 1u);
    };
    if (blockIdx.x == 0) {
        const uint64_t tail0 = head + nvec * V;
        if (threadIdx.x < head) add(keys[threadIdx.x]);
        if (threadIdx.x < n - tail0) add(keys[tail0 + threadIdx.x]);
    }
    const K* body = keys + head;
    const uint64_t nchunks = ceil_div(nvec, kChunkVecs);
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        Vec16<K> x[kK2Unroll];
        bool ok[kK2Unroll];
        k2_load(body, c, nvec, x, ok);
#pragma unroll
        for (int u = 0; u < kK2Unroll; ++u)
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < V; ++j) add(x[u].e[j]);
            }
    }
    __syncthreads();
    uint32_t* slab = slabs + (size_t)blockIdx.x * kMaxBins;
    for (uint32_t j = threadIdx.x; j < nb; j += kHistThreads) {
        uint32_t c = 0;
        for (uint32_t r = 0; r < R; ++r) c += sm[r * nb + j];
        slab[j] = c;
    }
}

template <typename K>
__device__ __forceinline__ void k2_split(const K* __restrict__ keys, uint64_t n, K flip,
                                         uint64_t head, uint64_t nvec, K mn, uint32_t s,
                                         uint32_t nb, uint32_t* __restrict__ slabs, uint32_t* sm) {
    constexpr int V = Vec16<K>::kN;
    constexpr uint64_t kChunkVecs = (uint64_t)kHistThreads * kK2Unroll;
    const uint32_t h = blockIdx.x & 1u, pair = blockIdx.x >> 1, npairs = gridDim.x >> 1;
    const uint32_t half = (nb + 1) >> 1;
    const uint32_t lo = h * half;
    const uint32_t len = h ? nb - half : half;
    for (uint32_t i = threadIdx.x; i < len; i += kHistThreads) sm[i] = 0;
    __syncthreads();
    auto add = [&](K x) {
        const uint32_t b = (uint32_t)(((K)(x ^ flip) - mn) >> s) - lo;   // wraps below lo
        if (b < len) atomicAdd(&sm[b], 1u);
    };
    if (pair == 0) {
        const uint64_t tail0 = head + nvec * V;
        if (threadIdx.x < head) add(keys[threadIdx.x]);
        if (threadIdx.x < n - tail0) add(keys[tail0 + threadIdx.x]);
    }
    const K* body = keys + head;
    const uint64_t nchunks = ceil_div(nvec, kChunkVecs);
    for (uint64_t c = pair; c < nchunks; c += npairs) {
        Vec16<K> x[kK2Unroll];
        bool ok[kK2Unroll];
        k2_load(body, c, nvec, x, ok);
#pragma unroll
        for (int u = 0; u < kK2Unroll; ++u)
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < V; ++j) add(x[u].e[j]);
            }
    }
    __syncthreads();
    uint32_t* slab = slabs + (size_t)pair * kMaxBins + lo;
    for (uint32_t j = threadIdx.x; j < len; j += kHistThreads) slab[j] = sm[j];
}

// Above kU32Bins bins, for an input not in runs (k2_packed_layout): every
// CTA counts all bins of its own keys in 16-bit counters, two to a word
// (128 KB).  A counter that reaches 2^15 gives 2^15 back at once and lists its
// bin (the list adds 2^15 to the bin when the CTA writes its slab), so a
// counter never holds more than 2^15 plus the additions that land before
// that subtraction.  An addition that would carry out of 16 bits is seen by
// the thread that makes it (old value 0xffff): the CTA marks the record and
// the host counts again in the split layout, so the histogram is exact either
// way.  One slab per CTA.  Inputs in runs (few descents or few ascents:
// neighbouring keys share a bin) keep the split layout, whose additions need
// no returned value: returning additions serialise when a warp's keys share a
// counter.
constexpr uint32_t kK2Words = kMaxBins / 2;
constexpr uint32_t kK2OvfCap = 1024;   // flushes a CTA can list (2^15 keys each)
static_assert((kK2Words + kK2OvfCap) * 4 <= kHistSmemBytes, "packed counters fit the shared memory");

// K2's layout above kU32Bins: packed (one slab per CTA) or split (one slab
// per cluster pair).  K3 asks the same question of the same record.
__device__ __forceinline__ bool k2_packed_layout(const DevFeatures* rec, int split) {
    const unsigned long long q = rec->n / 4;
    return !split && rec->nbins > kU32Bins && rec->descents >= q && rec->ascents >= q;
}

template <typename K>
__device__ __forceinline__ void k2_packed(const K* __restrict__ keys, uint64_t n, K flip,
                                          uint64_t head, uint64_t nvec, K mn, uint32_t s,
                                          uint32_t nb, uint32_t* __restrict__ slabs, uint32_t* sm,
                                          uint32_t* wrapped) {
    constexpr int V = Vec16<K>::kN;
    constexpr uint64_t kChunkVecs = (uint64_t)kHistThreads * kK2Unroll;
    __shared__ uint32_t s_novf, s_bad;
    uint32_t* ovf = sm + kK2Words;
    const uint32_t words = (nb + 1) >> 1;
    for (uint32_t i = threadIdx.x; i < words; i += kHistThreads) sm[i] = 0;
    if (threadIdx.x == 0) {
        s_novf = 0;
        s_bad = 0;
    }
    __syncthreads();
    auto add = [&](K x) {
        const uint32_t bin = (uint32_t)(((K)(x ^ flip) - mn) >> s);
        if (!AHS_DCHECK(bin < nb, "k2 bin", bin)) return;
        const uint32_t sh = (bin & 1u) << 4;
        const uint32_t old = (atomicAdd(&sm[bin >> 1], 1u << sh) >> sh) & 0xffffu;
        if (old == 0x7fffu) {
            atomicSub(&sm[bin >> 1], 0x8000u << sh);
            const uint32_t i = atomicAdd(&s_novf, 1u);
            if (i < kK2OvfCap) ovf[i] = bin;
            else s_bad = 1;
        } else if (old == 0xffffu) {
            s_bad = 1;
        }
    };
    if (blockIdx.x == 0) {
        const uint64_t tail0 = head + nvec * V;
        if (threadIdx.x < head) add(keys[threadIdx.x]);
        if (threadIdx.x < n - tail0) add(keys[tail0 + threadIdx.x]);
    }
    const K* body = keys + head;
    const uint64_t nchunks = ceil_div(nvec, kChunkVecs);
    for (uint64_t c = blockIdx.x; c < nchunks; c += gridDim.x) {
        Vec16<K> x[kK2Unroll];
        bool ok[kK2Unroll];
        k2_load(body, c, nvec, x, ok);
#pragma unroll
        for (int u = 0; u < kK2Unroll; ++u)
            if (ok[u]) {
#pragma unroll
                for (int j = 0; j < V; ++j) add(x[u].e[j]);
            }
    }
    __syncthreads();
    uint32_t* slab = slabs + (size_t)blockIdx.x * kMaxBins;
    for (uint32_t j = threadIdx.x; j < words; j += kHistThreads) {
        const uint32_t w = sm[j];
        slab[2 * j] = w & 0xffffu;
        if (2 * j + 1 < nb) slab[2 * j + 1] = w >> 16;
    }
    __syncthreads();   // the slab's plain stores come before the listed halves
    const uint32_t novf = s_novf < kK2OvfCap ? s_novf : kK2OvfCap;
    for (uint32_t i = threadIdx.x; i < novf; i += kHistThreads) atomicAdd(&slab[ovf[i]], 0x8000u);
    if (threadIdx.x == 0 && s_bad) atomicExch(wrapped, 1u);
}

template <typename K>
__global__ void __launch_bounds__(kHistThreads, 1)
k2_histogram(const K* __restrict__ keys, uint64_t n, K flip, uint64_t head, uint64_t nvec,
             DevFeatures* __restrict__ rec, uint32_t* __restrict__ slabs, int skip_sorted, int split) {
    extern __shared__ __align__(16) uint32_t sm32[];
    if (presorted_skip(rec, (uint32_t)skip_sorted)) return;   // block-uniform
    const K mn = (K)rec->min_ord;
    const uint32_t s = rec->shift;
    const uint32_t nb = rec->nbins;
    if (nb <= kU32Bins) k2_replicated<K>(keys, n, flip, head, nvec, mn, s, nb, slabs, sm32);
    else if (k2_packed_layout(rec, split))
        k2_packed<K>(keys, n, flip, head, nvec, mn, s, nb, slabs, sm32, &rec->k2_wrapped);
    else k2_split<K>(keys, n, flip, head, nvec, mn, s, nb, slabs, sm32);
}

// host_rec / host_hist (optional): pinned host mirrors of the record and of
// the histogram, written here so that the host reads them without a copy.
__global__ void __launch_bounds__(256)
k3_entropy(const uint32_t* __restrict__ slabs, uint32_t k2_grid, uint64_t n,
           DevFeatures* __restrict__ rec, unsigned long long* __restrict__ hist,
           double* __restrict__ partials, DevFeatures* host_rec,
           unsigned long long* host_hist, int skip_sorted, int split) {
    if (presorted_skip(rec, (uint32_t)skip_sorted)) {
        // K2 counted nothing: no histogram, and the entropy is marked missing.
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            rec->entropy = __longlong_as_double(0x7ff8000000000000ll);
            rec->entropy_norm = rec->entropy;
            if (host_rec) *host_rec = *rec;
        }
        return;
    }
    const uint32_t nb = rec->nbins;
    // One slab per CTA (replicated and packed layouts) or per pair (split).
    const uint32_t nslabs = (nb > kU32Bins && !k2_packed_layout(rec, split)) ? k2_grid / 2 : k2_grid;
    __shared__ double s_part[8];
    __shared__ bool s_last;
    __shared__ unsigned long long s_acc[8][32];
    // Blocks past the bins have nothing to add: they leave at once, and the
    // last of the active blocks reduces their partial sums.
    const bool direct = nb <= kK3DirectBins;
    const uint32_t active = direct ? (nb + 31) / 32 : (nb + 255) / 256;
    if (blockIdx.x >= active) return;
    double term = 0.0;
    if (direct) {
        // Few bins: block b takes bins [32 b, 32 b + 32) and its eight warps
        // split the slabs between them, so every thread has a few loads in
        // flight instead of one thread walking all ~150 slabs of a bin.
        const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
        const uint32_t bin = blockIdx.x * 32 + lane;
        unsigned long long acc = 0;
        if (bin < nb)
            for (uint32_t c = warp; c < nslabs; c += 8) acc += slabs[(size_t)c * kMaxBins + bin];
        s_acc[warp][lane] = acc;
        __syncthreads();
        if (warp == 0 && bin < nb) {
            unsigned long long tot = 0;
            for (int w = 0; w < 8; ++w) tot += s_acc[w][lane];
            hist[bin] = tot;
            if (host_hist) host_hist[bin] = tot;
            if (tot) {
                const double p = (double)tot / (double)n;
                term = -p * log2(p);
            }
        }
    } else {
        const uint32_t j = blockIdx.x * 256 + threadIdx.x;
        if (j < nb) {
            unsigned long long tot = 0;
            uint32_t c = 0;
            for (; c + 4 <= nslabs; c += 4) {
                const uint32_t a0 = slabs[(size_t)(c + 0) * kMaxBins + j];
                const uint32_t a1 = slabs[(size_t)(c + 1) * kMaxBins + j];
                const uint32_t a2 = slabs[(size_t)(c + 2) * kMaxBins + j];
                const uint32_t a3 = slabs[(size_t)(c + 3) * kMaxBins + j];
                tot += (unsigned long long)a0 + a1 + a2 + a3;
            }
            for (; c < nslabs; ++c) tot += slabs[(size_t)c * kMaxBins + j];
            hist[j] = tot;
            if (host_hist) host_hist[j] = tot;
            if (tot) {
                const double p = (double)tot / (double)n;
                term = -p * log2(p);
            }
        }
    }
    term = warp_sum(term);
    if (lane_id() == 0) s_part[threadIdx.x >> 5] = term;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < 8; ++w) b += s_part[w];
        partials[blockIdx.x] = b;
        __threadfence();
        s_last = (atomicAdd(&rec->k3_done, 1u) == active - 1);
    }
    __syncthreads();
    if (!s_last) return;
    // Last active block: the partial sums, one per thread, then the block.
    double h = threadIdx.x < active ? __ldcg(partials + threadIdx.x) : 0.0;
    h = warp_sum(h);
    if (lane_id() == 0) s_part[threadIdx.x >> 5] = h;
    __syncthreads();
    if (threadIdx.x != 0) return;
    double H = 0.0;
    for (int w = 0; w < 8; ++w) H += s_part[w];
    rec->entropy = H;
    rec->entropy_norm = nb > 1 ? H / log2((double)nb) : 0.0;
    rec->k3_done = 0;
    if (host_rec) *host_rec = *rec;
}

template <typename K>
cudaError_t k2_k3_t(const K* keys, uint64_t n, K flip, uint64_t head, uint64_t nvec,
                    const FeatureScratch& s, int sms, cudaStream_t st, bool split);

template <typename K>
cudaError_t features_t(const void* keys_v, uint64_t n, K flip, const FeatureScratch& s, int sms,
                       cudaStream_t st) {
    const K* keys = static_cast<const K*>(keys_v);
    constexpr int V = Vec16<K>::kN;
    const uint64_t head = head_elems<K>(keys, n);
    const uint64_t nvec = (n - head) / V;
    const uint32_t g1 = k1_blocks(n, sms);
    {
        TraceScope ts("features_minmax", n, st);
        k1_minmax_descents<K><<<g1, kK1Threads, 0, st>>>(keys, n, flip, head, nvec, s.k1_partials,
                                                          s.rec);
    }
    return k2_k3_t<K>(keys, n, flip, head, nvec, s, sms, st, false);
}

// K2 and K3.  One CTA per SM (shared memory holds one histogram), launched as
// clusters of two so that a pair of the split layout shares a GPC and its
// duplicated reads hit L2.  split: the split layout above kU32Bins whatever
// the input (the exact count after a packed counter wrapped).
template <typename K>
cudaError_t k2_k3_t(const K* keys, uint64_t n, K flip, uint64_t head, uint64_t nvec,
                    const FeatureScratch& s, int sms, cudaStream_t st, bool split) {
    const uint32_t g2 = (uint32_t)(sms & ~1);
    {
        TraceScope ts("features_histogram", n, st);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g2);
        cfg.blockDim = dim3(kHistThreads);
        cfg.dynamicSmemBytes = kHistSmemBytes;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 2;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, k2_histogram<K>, keys, n, flip, head, nvec, s.rec,
                                           s.slabs, (int)s.skip_sorted, (int)split);
        if (e != cudaSuccess) return e;
    }
    {
        TraceScope ts("features_entropy", 0, st);
        k3_entropy<<<kEntropyBlocks, 256, 0, st>>>(s.slabs, g2, n, s.rec, s.hist, s.ent_partials,
                                                   s.host_rec, s.host_hist, (int)s.skip_sorted,
                                                   (int)split);
    }
    return cudaGetLastError();
}

template <typename K>
cudaError_t split_retry_t(const void* keys_v, uint64_t n, K flip, const FeatureScratch& s, int sms,
                          cudaStream_t st) {
    const K* keys = static_cast<const K*>(keys_v);
    constexpr int V = Vec16<K>::kN;
    const uint64_t head = head_elems<K>(keys, n);
    const uint64_t nvec = (n - head) / V;
    return k2_k3_t<K>(keys, n, flip, head, nvec, s, sms, st, true);
}

}  // namespace

uint32_t k1_blocks(uint64_t n, int sms) {
    const uint64_t per = (uint64_t)kK1Threads * 8 * 4;
    uint64_t b = ceil_div(n ? n : 1, per);
    const uint64_t cap = 2ull * (uint64_t)sms;   // two resident blocks per SM: one wave
    return (uint32_t)(b < cap ? b : cap);
}

size_t features_scratch_bytes(int sms) {
    return 3 * sizeof(unsigned long long) * 4 * (size_t)sms + 256 +
           (size_t)sms * kMaxBins * sizeof(uint32_t) + 256 +
           kMaxBins * sizeof(unsigned long long) + 256 + kEntropyBlocks * sizeof(double) + 256;
}

cudaError_t launch_features(const void* keys, uint64_t n, KeyDesc kd, const FeatureScratch& s,
                            int sms, cudaStream_t st) {
    // The dynamic shared-memory limit is a per-device attribute of the kernel:
    // set it on every call (a cheap host call) so that every device, and every
    // thread that launches, finds it set.
    if (kd.bytes == 4) {
        cudaError_t e = cudaFuncSetAttribute(k2_histogram<uint32_t>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             kHistSmemBytes);
        if (e != cudaSuccess) return e;
        return features_t<uint32_t>(keys, n, (uint32_t)kd.flip, s, sms, st);
    }
    cudaError_t e = cudaFuncSetAttribute(k2_histogram<uint64_t>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kHistSmemBytes);
    if (e != cudaSuccess) return e;
    return features_t<uint64_t>(keys, n, kd.flip, s, sms, st);
}

cudaError_t launch_features_split_retry(const void* keys, uint64_t n, KeyDesc kd,
                                        const FeatureScratch& s, int sms, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(&s.rec->k2_wrapped, 0, sizeof(uint32_t), st);
    if (e != cudaSuccess) return e;
    if (kd.bytes == 4) return split_retry_t<uint32_t>(keys, n, (uint32_t)kd.flip, s, sms, st);
    return split_retry_t<uint64_t>(keys, n, kd.flip, s, sms, st);
}

}  // namespace ahs
