// LSD radix sort (Listing 3, Section III-G) over u = ord(x) - min.
//
// The paper distributes keys into base-b buckets digit by digit, least
// significant first, appending in input order (stable), with d = ceil(log_b k)
// passes (Eq. 4).  Here b = 2^8 and each pass is one "onesweep" kernel: a tile
// of keys is ranked by digit in shared memory (warp match + cross-warp scan),
// the tile's per-digit counts are published and the exclusive prefix over all
// earlier tiles is found by decoupled look-back (Merrill & Garland 2016;
// one-sweep formulation of Adinets & Merrill 2022), and the tile is staged in
// shared memory in digit order so every digit's run is written contiguously.
// The global digit offsets of all passes come from one histogram kernel that
// reads the keys once before the first pass.
#include "common.cuh"
#include "internal.h"
#include "rank.cuh"
#include "trace.h"

namespace ahs {
namespace {

constexpr int kRadixMax = 2048;               // widest digit: 11 bits
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagIncl = 2u << 30;
constexpr uint32_t kCountMask = (1u << 30) - 1;
constexpr uint32_t kSpinLimit = 1u << 22;     // ~1 s with the backoff below

constexpr int kHistThreadsR = 512;

struct PassDesc {
    uint32_t passes;
    uint32_t shift[kMaxRadixPasses];
    uint32_t bits[kMaxRadixPasses];
};

// Replicated shared histograms spread the atomics of skewed digits; wide
// digits leave room for fewer copies.
template <int NB>
constexpr int hist_replicas() { return NB <= 256 ? 4 : (NB <= 512 ? 2 : 1); }
template <int NB>
constexpr size_t digit_hist_smem() { return (size_t)hist_replicas<NB>() * kMaxRadixPasses * NB * 4; }

// Histogram of every pass's digit in one read (dhist zeroed beforehand); the
// last block turns the counts into per-pass exclusive digit offsets.  NB is
// the digit alphabet (2^width); dhist and dbase rows are kRadixMax apart.
template <typename K, int NB>
__global__ void __launch_bounds__(kHistThreadsR)
radix_digit_hist(const K* __restrict__ keys, uint64_t n, K mn, K flip, uint64_t head,
                 uint64_t nvec, PassDesc pd, unsigned long long* __restrict__ dhist,
                 uint32_t* __restrict__ dbase, DevFeatures* __restrict__ rec) {
    constexpr int V = Vec16<K>::kN;
    constexpr int R = hist_replicas<NB>();
    extern __shared__ __align__(16) uint32_t sh[];   // [R][kMaxRadixPasses][NB]
    __shared__ bool s_last;
    const uint32_t P = pd.passes;
    for (uint32_t i = threadIdx.x; i < (uint32_t)R * kMaxRadixPasses * NB; i += kHistThreadsR) sh[i] = 0;
    __syncthreads();
    uint32_t* mine = sh + ((threadIdx.x >> 5) % R) * kMaxRadixPasses * NB;
    auto add = [&](K x) {
        const K u = (K)(x ^ flip) - mn;
        for (uint32_t p = 0; p < P; ++p)
            atomicAdd(&mine[p * NB + ((uint32_t)(u >> pd.shift[p]) & ((1u << pd.bits[p]) - 1))], 1u);
    };
    const uint64_t gtid = (uint64_t)blockIdx.x * kHistThreadsR + threadIdx.x;
    const uint64_t stride = (uint64_t)gridDim.x * kHistThreadsR;
    const uint64_t tail0 = head + nvec * V;
    if (gtid < head) add(keys[gtid]);
    if (gtid < n - tail0) add(keys[tail0 + gtid]);
    const K* body = keys + head;
    for (uint64_t v = gtid; v < nvec; v += 2 * stride) {
        Vec16<K> a = load_vec16(body + v * V);
        const bool ok2 = v + stride < nvec;
        Vec16<K> b;
        if (ok2) b = load_vec16(body + (v + stride) * V);
#pragma unroll
        for (int j = 0; j < V; ++j) add(a.e[j]);
        if (ok2) {
#pragma unroll
            for (int j = 0; j < V; ++j) add(b.e[j]);
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < P * NB; i += kHistThreadsR) {
        const uint32_t p = i / NB, d = i % NB;
        uint32_t c = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) c += sh[(r * kMaxRadixPasses + p) * NB + d];
        if (c) atomicAdd(&dhist[p * kRadixMax + d], (unsigned long long)c);
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) s_last = (atomicAdd(&rec->rh_done, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!s_last) return;
    // Last block: exclusive prefix per pass (one warp per pass), then clear.
    const uint32_t warp = threadIdx.x >> 5, lane = lane_id();
    if (warp < P) {
        unsigned long long run = 0;
        for (int base = 0; base < NB; base += 32) {
            const unsigned long long c =
                base + lane < (uint32_t)NB ? atomicAdd(&dhist[warp * kRadixMax + base + lane], 0ull) : 0ull;
            const unsigned long long inc = warp_inclusive_scan(c);
            if (base + lane < (uint32_t)NB) dbase[warp * kRadixMax + base + lane] = (uint32_t)(run + inc - c);
            run += __shfl_sync(AHS_FULL_MASK, inc, 31);
        }
    }
    if (threadIdx.x == 0) rec->rh_done = 0;
}

// Per-warp digit counters.  Up to 512 digits: one 32-bit counter per digit.
// Wider digits: two 16-bit counters per word (a warp's count of one digit in a
// tile, and every prefix of them over the warps, stays below 2^16, so packed
// words add without carries between the halves).
template <int NB>
struct WarpCounters {
    static constexpr bool kPacked = NB > 512;
    static constexpr int kWords = kPacked ? NB / 2 : NB;
    __device__ static __forceinline__ uint32_t add(uint32_t* wh, uint32_t d, uint32_t c) {
        if constexpr (kPacked) {
            const uint32_t sh = 16u * (d & 1u);
            return (atomicAdd(&wh[d >> 1], c << sh) >> sh) & 0xffffu;
        } else {
            return atomicAdd(&wh[d], c);
        }
    }
    __device__ static __forceinline__ uint32_t get(const uint32_t* wh, uint32_t d) {
        if constexpr (kPacked) return (wh[d >> 1] >> (16u * (d & 1u))) & 0xffffu;
        else return wh[d];
    }
};

// Stable rank of each item among the warp's items with the same digit (input
// order: item i of lane l precedes item i of lane l + 1 and item i + 1 of any
// lane).  Peers are found by one ballot per digit bit (multisplit); the group's
// lowest lane adds the group size to the warp's counter.  Digit NB marks an
// item past the end.
template <int IPT, int NB>
__device__ __forceinline__ void rank_warp(const uint32_t (&dig)[IPT], uint32_t (&rank)[IPT],
                                          uint32_t* wh) {
    constexpr int BITS = NB <= 2 ? 1 : 32 - __builtin_clz(NB - 1);
    const uint32_t lt = lanemask_lt(), lane = lane_id();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t d = dig[i];
        const bool valid = d < (uint32_t)NB;
        uint32_t peers = __ballot_sync(AHS_FULL_MASK, valid);
#pragma unroll
        for (int b = 0; b < BITS; ++b) {
            const bool bit = (d >> b) & 1u;
            const uint32_t m = __ballot_sync(AHS_FULL_MASK, bit);
            peers &= bit ? m : ~m;
        }
        const uint32_t leader = valid ? __ffs(peers) - 1 : lane;
        uint32_t old = 0;
        if (valid && lane == leader) old = WarpCounters<NB>::add(wh, d, __popc(peers));
        old = __shfl_sync(AHS_FULL_MASK, old, leader);
        rank[i] = old + __popc(peers & lt);
    }
}

template <typename K, bool VALS, int THREADS, int IPT, int NB>
struct OnesweepSmem {
    static constexpr int W = THREADS / 32;
    static constexpr int TILE = THREADS * IPT;
    static_assert(TILE < 65536 || NB <= 512, "packed counters hold tile prefixes below 2^16");
    uint32_t warp_hist[W][WarpCounters<NB>::kWords];
    uint32_t tile_count[NB];   // this tile's digit counts, then the write offsets
    uint32_t tile_start[NB];
    uint32_t scan[W + 1];
    uint32_t tile_id;
    K keys[TILE];
    uint32_t vals[VALS ? TILE : 1];
    alignas(16) uint32_t vraw[VALS ? TILE : 1];   // the tile's payload in input order
};

template <typename K, bool VALS, int THREADS, int IPT, int MINB, int NB>
__global__ void __launch_bounds__(THREADS, MINB)
onesweep_pass(const K* __restrict__ keys_in, K* __restrict__ keys_out,
              const uint32_t* __restrict__ vals_in, uint32_t* __restrict__ vals_out, uint32_t n,
              K mn, K flip, uint32_t shift, uint32_t bits, const uint32_t* __restrict__ dbase,
              uint32_t* __restrict__ status, uint32_t* __restrict__ tile_counter,
              uint32_t* __restrict__ err, uint32_t stall_tile) {
    using Smem = OnesweepSmem<K, VALS, THREADS, IPT, NB>;
    using WC = WarpCounters<NB>;
    static_assert(THREADS % 32 == 0 && THREADS <= 1024, "whole warps");
    constexpr int W = Smem::W;
    constexpr int TILE = Smem::TILE;
    constexpr int WARP_ITEMS = 32 * IPT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Smem& S = *reinterpret_cast<Smem*>(smem_raw);

    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t mask = (1u << bits) - 1;

    if (tid == 0) S.tile_id = atomicAdd(tile_counter, 1u);
    for (uint32_t i = tid; i < W * WC::kWords; i += THREADS) (&S.warp_hist[0][0])[i] = 0;
    __syncthreads();
    const uint32_t tile = S.tile_id;
    if (!AHS_DCHECK(tile < gridDim.x, "onesweep tile id", tile)) return;
    const uint32_t tile_base = tile * (uint32_t)TILE;
    const uint32_t wbase = tile_base + warp * WARP_ITEMS;

    // The tile's payload goes to shared memory by asynchronous copies that
    // run while the keys are ranked (loading it into registers with the keys
    // measured slower on GB300, 1.51 against 1.25 ms per pass at 2^27 keys:
    // register pressure).
    if constexpr (VALS) {
        const uint32_t tile_n = (n - tile_base) < (uint32_t)TILE ? (n - tile_base) : (uint32_t)TILE;
        const uint32_t* src = vals_in + tile_base;
        const bool vec = (reinterpret_cast<uintptr_t>(src) & 15u) == 0;
        const uint32_t nv = vec ? tile_n / 4 : 0;
        for (uint32_t q = tid; q < nv; q += THREADS) cp_async16(&S.vraw[4 * q], src + 4 * q);
        for (uint32_t q = 4 * nv + tid; q < tile_n; q += THREADS) cp_async_key(&S.vraw[q], src + q);
        cp_async_commit();
    }

    // Load warp-striped: item i of lane l is key wbase + 32 i + l.
    K key[IPT];
    uint32_t dig[IPT];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t idx = wbase + 32 * i + lane;
        if (idx < n) {
            key[i] = keys_in[idx];
            dig[i] = (uint32_t)(((K)(key[i] ^ flip) - mn) >> shift) & mask;
        } else {
            key[i] = 0;
            dig[i] = NB;   // past the end: ranked nowhere
        }
    }

    // Rank within the warp in input order (stable): peers share a digit.
    uint32_t rank[IPT];
    rank_warp<IPT, NB>(dig, rank, S.warp_hist[warp]);
    __syncthreads();

    // Per digit (per counter word): exclusive prefix over warps, and the
    // tile's count, published for the look-back as early as possible.
    for (uint32_t q = tid; q < (uint32_t)WC::kWords; q += THREADS) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
            const uint32_t c = S.warp_hist[w][q];
            S.warp_hist[w][q] = run;
            run += c;
        }
        const uint32_t flag = tile == 0 ? kFlagIncl : kFlagAgg;
        if constexpr (WC::kPacked) {
            S.tile_count[2 * q] = run & 0xffffu;
            S.tile_count[2 * q + 1] = run >> 16;
            if (tile != stall_tile) {
                st_relaxed_gpu(&status[(size_t)tile * NB + 2 * q], flag | (run & 0xffffu));
                st_relaxed_gpu(&status[(size_t)tile * NB + 2 * q + 1], flag | (run >> 16));
            }
        } else {
            S.tile_count[q] = run;
            if (tile != stall_tile) st_relaxed_gpu(&status[(size_t)tile * NB + q], flag | run);
        }
    }
    if constexpr (VALS) cp_async_wait_all();   // this thread's payload copies; the barrier shows all
    __syncthreads();
    scan_digit_counts<THREADS, NB>(S.tile_count, S.tile_start, S.scan);

    // Stage the tile in digit order.
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        if (dig[i] < (uint32_t)NB) {
            const uint32_t lp = S.tile_start[dig[i]] + WC::get(S.warp_hist[warp], dig[i]) + rank[i];
            if (AHS_DCHECK(lp < (uint32_t)TILE, "onesweep stage", lp)) S.keys[lp] = key[i];
        }
    }
    if constexpr (VALS) {
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            if (dig[i] < (uint32_t)NB) {
                const uint32_t lp = S.tile_start[dig[i]] + WC::get(S.warp_hist[warp], dig[i]) + rank[i];
                if (AHS_DCHECK(lp < (uint32_t)TILE, "onesweep vstage", lp))
                    S.vals[lp] = S.vraw[warp * WARP_ITEMS + 32 * i + lane];
            }
        }
    }

    // Decoupled look-back: exclusive prefix of each digit over earlier tiles.
    // The same thread then turns the digit's count into its write offset.
    for (uint32_t d = tid; d < (uint32_t)NB; d += THREADS) {
        uint32_t excl = 0;
        const uint32_t cnt = S.tile_count[d];
        if (tile > 0) {
            int64_t j = (int64_t)tile - 1;
            uint32_t spins = 0;
            while (j >= 0) {
                const uint32_t s = ld_relaxed_gpu(&status[(size_t)j * NB + d]);
                const uint32_t flag = s & ~kCountMask;
                if (flag == 0) {
                    if (++spins > kSpinLimit) { report_error(err, kDevLookbackTimeout); break; }
                    // Another tile gave up already: stop waiting too.
                    if ((spins & 1023u) == 0 && ld_relaxed_gpu(err) != 0) break;
                    if (spins > 64) __nanosleep(spins > 4096 ? 256 : 32);
                    continue;
                }
                excl += s & kCountMask;
                if (flag == kFlagIncl) break;
                --j;
            }
            if (tile != stall_tile)
                st_relaxed_gpu(&status[(size_t)tile * NB + d], kFlagIncl | (excl + cnt));
        }
        S.tile_count[d] = dbase[d] + excl - S.tile_start[d];
    }
    __syncthreads();

    // Write the staged tile: runs of one digit go to consecutive addresses.
    const uint32_t tile_n = (n - tile_base) < (uint32_t)TILE ? (n - tile_base) : (uint32_t)TILE;
    for (uint32_t j = tid; j < tile_n; j += THREADS) {
        const K k = S.keys[j];
        const uint32_t d = (uint32_t)(((K)(k ^ flip) - mn) >> shift) & mask;
        const uint32_t gp = S.tile_count[d] + j;
        if (gp >= n) { report_error(err, kDevBadState); continue; }   // only after a failed wait
        keys_out[gp] = k;
        if constexpr (VALS) vals_out[gp] = S.vals[j];
    }
}

// Tile shapes (threads x keys per thread, minimum resident CTAs per SM).
template <typename K, bool VALS>
struct OnesweepCfg;
template <> struct OnesweepCfg<uint32_t, false> { static constexpr int T = 512, IPT = 16, MINB = 2; };
template <> struct OnesweepCfg<uint32_t, true> { static constexpr int T = 512, IPT = 12, MINB = 2; };
template <> struct OnesweepCfg<uint64_t, false> { static constexpr int T = 512, IPT = 12, MINB = 2; };
template <> struct OnesweepCfg<uint64_t, true> { static constexpr int T = 512, IPT = 8, MINB = 2; };

template <typename K, bool VALS>
constexpr int tile_keys() { return OnesweepCfg<K, VALS>::T * OnesweepCfg<K, VALS>::IPT; }

// Resident CTAs per SM a digit width allows with this tile shape (shared memory).
template <typename K, bool VALS, int NB>
constexpr int onesweep_minb() {
    constexpr int T = OnesweepCfg<K, VALS>::T, IPT = OnesweepCfg<K, VALS>::IPT;
    return sizeof(OnesweepSmem<K, VALS, T, IPT, NB>) * 2 <= 220 * 1024 ? OnesweepCfg<K, VALS>::MINB : 1;
}

template <typename K, bool VALS, int NB>
cudaError_t radix_passes_t(const K* kin, K* kout, const uint32_t* vin, uint32_t* vout, uint64_t n,
                           K flip, K mn, const RadixPlan& plan, const RadixScratch& rs,
                           DevFeatures* rec, uint32_t* err, int sms, cudaStream_t st,
                           uint32_t stall_tile) {
    constexpr int T = OnesweepCfg<K, VALS>::T, IPT = OnesweepCfg<K, VALS>::IPT;
    constexpr int MINB = onesweep_minb<K, VALS, NB>();
    constexpr int TILE = T * IPT;
    using Smem = OnesweepSmem<K, VALS, T, IPT, NB>;
    K* ktmp = static_cast<K*>(rs.keys_tmp);
    const uint32_t P = plan.passes;
    const uint64_t tiles = ceil_div(n, TILE);
    cudaError_t e;

    // Histogram of all passes' digits, and their exclusive offsets.
    PassDesc pd{};
    pd.passes = P;
    for (uint32_t p = 0; p < P; ++p) { pd.shift[p] = plan.shift[p]; pd.bits[p] = plan.bits[p]; }
    uint32_t* dbase = reinterpret_cast<uint32_t*>(rs.digit_hist + kMaxRadixPasses * kRadixMax);
    // One zeroing launch covers the digit counts, the look-back status words
    // of every pass and the tile counters (carved contiguously).
    {
        const uint64_t words = (uint64_t)(rs.tile_counters + kMaxRadixPasses -
                                          reinterpret_cast<uint32_t*>(rs.digit_hist));
        e = launch_zero32(rs.digit_hist, words, sms, st);
        if (e != cudaSuccess) return e;
    }
    {
        constexpr int V = Vec16<K>::kN;
        const uint64_t head = head_elems<K>(kin, n);
        const uint64_t nvec = (n - head) / V;
        uint64_t g = ceil_div(nvec ? nvec : 1, (uint64_t)kHistThreadsR * 4);
        const uint64_t cap = 2ull * sms;
        g = g < cap ? g : cap;
        e = cudaFuncSetAttribute(radix_digit_hist<K, NB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)digit_hist_smem<NB>());
        if (e != cudaSuccess) return e;
        TraceScope ts("radix_digit_hist", n, st);
        radix_digit_hist<K, NB><<<(uint32_t)g, kHistThreadsR, digit_hist_smem<NB>(), st>>>(
            kin, n, mn, flip, head, nvec, pd, rs.digit_hist, dbase, rec);
    }

    // A per-device attribute of the kernel: set on every call, for every
    // device and launching thread.
    e = cudaFuncSetAttribute(onesweep_pass<K, VALS, T, IPT, MINB, NB>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(Smem));
    if (e != cudaSuccess) return e;

    // Buffer schedule: the last pass writes kout.  When sorting in place with
    // an odd pass count, first move the keys into the temporary buffer.
    const bool inplace = (static_cast<const void*>(kin) == static_cast<const void*>(kout));
    const K* src = kin;
    const uint32_t* vsrc = vin;
    if (inplace && (P % 2 == 1)) {
        e = launch_copy32(ktmp, kin, n * sizeof(K) / 4, sms, st);
        if (e != cudaSuccess) return e;
        if (VALS) {
            e = launch_copy32(rs.vals_tmp, vin, n, sms, st);
            if (e != cudaSuccess) return e;
        }
        src = ktmp;
        vsrc = rs.vals_tmp;
    }
    for (uint32_t p = 0; p < P; ++p) {
        const bool to_out = ((P - 1 - p) % 2) == 0;
        K* dst = to_out ? kout : ktmp;
        uint32_t* vdst = to_out ? vout : rs.vals_tmp;
        uint32_t* status = rs.status + (size_t)p * tiles * NB;
        TraceScope ts("radix_onesweep", n, st);
        onesweep_pass<K, VALS, T, IPT, MINB, NB><<<(uint32_t)tiles, T, sizeof(Smem), st>>>(
            src, dst, vsrc, vdst, (uint32_t)n, mn, flip, plan.shift[p], plan.bits[p],
            dbase + p * kRadixMax, status, rs.tile_counters + p, err, stall_tile);
        src = dst;
        vsrc = vdst;
    }
    return cudaGetLastError();
}

template <typename K, bool VALS>
cudaError_t radix_t(const void* kin_v, void* kout_v, const uint32_t* vin, uint32_t* vout,
                    uint64_t n, K flip, K mn, const RadixPlan& plan, const RadixScratch& rs,
                    DevFeatures* rec, uint32_t* err, int sms, cudaStream_t st, uint32_t stall_tile) {
    const K* kin = static_cast<const K*>(kin_v);
    K* kout = static_cast<K*>(kout_v);
    switch (plan.radix) {
    case 16:
        return radix_passes_t<K, VALS, 16>(kin, kout, vin, vout, n, flip, mn, plan, rs, rec, err, sms,
                                           st, stall_tile);
    case 256:
        return radix_passes_t<K, VALS, 256>(kin, kout, vin, vout, n, flip, mn, plan, rs, rec, err,
                                            sms, st, stall_tile);
    case 512:
        return radix_passes_t<K, VALS, 512>(kin, kout, vin, vout, n, flip, mn, plan, rs, rec, err,
                                            sms, st, stall_tile);
    case 1024:
        return radix_passes_t<K, VALS, 1024>(kin, kout, vin, vout, n, flip, mn, plan, rs, rec, err,
                                             sms, st, stall_tile);
    case 2048:
        return radix_passes_t<K, VALS, 2048>(kin, kout, vin, vout, n, flip, mn, plan, rs, rec, err,
                                             sms, st, stall_tile);
    default:
        return cudaErrorInvalidValue;
    }
}

uint64_t tile_keys_for(uint32_t key_bytes, bool has_vals) {
    if (key_bytes == 4) return has_vals ? tile_keys<uint32_t, true>() : tile_keys<uint32_t, false>();
    return has_vals ? tile_keys<uint64_t, true>() : tile_keys<uint64_t, false>();
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

// Eq. 4 with digits of at most max_bits bits: d = ceil(bitlen(span) / max_bits)
// passes, the bits shared as evenly as possible (so 36 bits at max_bits = 11
// take 4 passes of 9 bits), each pass's alphabet the smallest compiled one
// (16, 256, 512, 1024 or 2048 digits) that holds its width.
RadixPlan radix_plan(uint64_t span, uint32_t max_bits) {
    RadixPlan p{};
    if (max_bits < 1) max_bits = 1;
    if (max_bits > 11) max_bits = 11;
    const uint32_t D = bitlen64(span);
    p.passes = (D + max_bits - 1) / max_bits;
    if (p.passes > kMaxRadixPasses) p.passes = kMaxRadixPasses;   // only for max_bits < 8 on 64-bit keys
    const uint32_t width = p.passes ? (D + p.passes - 1) / p.passes : 0;
    p.radix = width <= 4 ? 16 : (width <= 8 ? 256 : (width <= 9 ? 512 : (width <= 10 ? 1024 : 2048)));
    for (uint32_t i = 0; i < p.passes; ++i) {
        p.shift[i] = width * i;
        const uint32_t hi = width * i + width < D ? width * i + width : D;
        p.bits[i] = hi - width * i;
    }
    return p;
}

size_t radix_scratch_bytes(uint64_t n, uint32_t key_bytes, bool has_vals, const RadixPlan& plan) {
    const uint64_t tiles = ceil_div(n, tile_keys_for(key_bytes, has_vals));
    return align256(n * key_bytes) + (has_vals ? align256(n * 4) : 0) +
           align256(kMaxRadixPasses * kRadixMax * (sizeof(unsigned long long) + sizeof(uint32_t))) +
           align256(((size_t)plan.passes * tiles * plan.radix + kMaxRadixPasses) * sizeof(uint32_t)) + 256;
}

RadixScratch radix_carve(void* base, uint64_t n, uint32_t key_bytes, bool has_vals,
                         const RadixPlan& plan) {
    RadixScratch r{};
    char* p = static_cast<char*>(base);
    r.tiles = ceil_div(n, tile_keys_for(key_bytes, has_vals));
    r.keys_tmp = p;
    p += align256(n * key_bytes);
    if (has_vals) {
        r.vals_tmp = reinterpret_cast<uint32_t*>(p);
        p += align256(n * 4);
    }
    r.digit_hist = reinterpret_cast<unsigned long long*>(p);   // digit bases follow it
    p += align256(kMaxRadixPasses * kRadixMax * (sizeof(unsigned long long) + sizeof(uint32_t)));
    r.status = reinterpret_cast<uint32_t*>(p);
    r.tile_counters = r.status + (size_t)plan.passes * r.tiles * plan.radix;
    return r;
}

cudaError_t launch_radix_sort(const void* keys_in, void* keys_out, const uint32_t* vals_in,
                              uint32_t* vals_out, uint64_t n, KeyDesc kd, uint64_t min_ord,
                              const RadixPlan& plan, const RadixScratch& rs, DevFeatures* rec,
                              uint32_t* err, int sms, cudaStream_t st, uint32_t stall_tile) {
    const bool v = vals_in != nullptr;
    if (kd.bytes == 4) {
        if (v) return radix_t<uint32_t, true>(keys_in, keys_out, vals_in, vals_out, n,
                                              (uint32_t)kd.flip, (uint32_t)min_ord, plan, rs, rec,
                                              err, sms, st, stall_tile);
        return radix_t<uint32_t, false>(keys_in, keys_out, nullptr, nullptr, n, (uint32_t)kd.flip,
                                        (uint32_t)min_ord, plan, rs, rec, err, sms, st, stall_tile);
    }
    if (v) return radix_t<uint64_t, true>(keys_in, keys_out, vals_in, vals_out, n, kd.flip,
                                          min_ord, plan, rs, rec, err, sms, st, stall_tile);
    return radix_t<uint64_t, false>(keys_in, keys_out, nullptr, nullptr, n, kd.flip, min_ord, plan,
                                    rs, rec, err, sms, st, stall_tile);
}

}  // namespace ahs
