// One-CTA stable sort of up to THREADS*IPT keys (optional uint32 payload) in
// registers and shared memory: LSD passes of 8-bit digits over u = ord(x) -
// min, with min and the digit count taken from the keys themselves (so a
// segment whose keys are all equal costs no pass).  Used for small inputs
// (the paper's insertion-sort regime, Section III-E) and for the buckets of the
// general path.  Without a payload a counting pass on the leading bits and
// per-thread insertion sorts take its place (block_sort_keys, below).
#pragma once

#include "common.cuh"
#include "rank.cuh"

namespace ahs {

constexpr int kBsRadix = 256;

template <typename K, bool VALS, int THREADS, int IPT>
struct BlockSortSmem {
    static constexpr int W = THREADS / 32;
    static constexpr int CAP = THREADS * IPT;
    uint32_t warp_hist[W][kBsRadix];
    uint32_t warp_mask[kRankBlockSort == kRankAtomicOr ? W : 1][kBsRadix];
    uint32_t tile_count[kBsRadix];
    uint32_t tile_start[kBsRadix];
    uint32_t scan[W + 1];
    unsigned long long red[2][W];
    K keys[CAP];
    uint32_t vals[VALS ? CAP : 1];
};

// Sort keys_in[0..m) (m <= CAP) into keys_out[0..m); vals likewise.  All
// threads of the block must call it.  keys_in may equal keys_out.
// bits < 64: the caller guarantees lo_known <= ord(x) < lo_known + 2^bits for
// every key, so the digits start from lo_known and no block-wide min / max
// has to be waited for before the first pass (the pass count still shrinks
// to what the keys' actual largest offset needs).
template <typename K, bool VALS, int THREADS, int IPT>
__device__ __forceinline__ void block_sort(const K* keys_in, K* keys_out,
                                           const uint32_t* vals_in, uint32_t* vals_out,
                                           uint32_t m, K flip,
                                           BlockSortSmem<K, VALS, THREADS, IPT>& S,
                                           K lo_known = 0, uint32_t bits = 0xffu) {
    constexpr int W = THREADS / 32;
    constexpr int WARP_ITEMS = 32 * IPT;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t wbase = warp * WARP_ITEMS;
    const bool known = bits < 64;

    K key[IPT];
    uint32_t val[IPT];
    K lo = ~K(0), hi = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t p = wbase + 32 * i + lane;
        if (p < m) {
            key[i] = keys_in[p];
            if constexpr (VALS) val[i] = vals_in[p];
            const K o = key[i] ^ flip;
            lo = o < lo ? o : lo;
            hi = o > hi ? o : hi;
        } else {
            key[i] = 0;
            if constexpr (VALS) val[i] = 0;
        }
    }
    uint32_t passes;
    if (known) {
        // Warp maxima go to shared memory now; the first pass's barrier
        // publishes them and the pass count is trimmed there.
        lo = lo_known;
        const unsigned long long b = warp_max((unsigned long long)hi);
        if (lane == 0) S.red[1][warp] = b;
        passes = (bits + 7) / 8;
    } else {
        // Block min / max of ord(x).
        unsigned long long a = warp_min((unsigned long long)lo), b = warp_max((unsigned long long)hi);
        if (lane == 0) { S.red[0][warp] = a; S.red[1][warp] = b; }
        __syncthreads();
        a = S.red[0][0];
        b = S.red[1][0];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            a = S.red[0][w] < a ? S.red[0][w] : a;
            b = S.red[1][w] > b ? S.red[1][w] : b;
        }
        lo = (K)a;
        hi = (K)b;
        __syncthreads();
        const uint32_t D = m ? bitlen64((unsigned long long)(K)(hi - lo)) : 0;
        passes = (D + 7) / 8;
    }

    if constexpr (kRankBlockSort == kRankAtomicOr) {
        for (uint32_t i = tid; i < W * kBsRadix; i += THREADS) (&S.warp_mask[0][0])[i] = 0;
    }
    for (uint32_t pass = 0; pass < passes; ++pass) {
        const uint32_t shift = 8 * pass;
        for (uint32_t i = tid; i < W * kBsRadix; i += THREADS) (&S.warp_hist[0][0])[i] = 0;
        __syncthreads();
        if (known && pass == 0) {
            // Largest key of the block (warp maxima published by the barrier
            // above): passes beyond the digits of its offset from lo are no-ops.
            unsigned long long b = S.red[1][0];
#pragma unroll
            for (int w = 1; w < W; ++w) b = S.red[1][w] > b ? S.red[1][w] : b;
            const uint32_t need = m ? (bitlen64((unsigned long long)(K)((K)b - lo)) + 7) / 8 : 0;
            passes = need < passes ? need : passes;
            if (passes == 0) break;
        }
        uint32_t dr[IPT];
        {
            uint32_t dig[IPT];
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                const uint32_t p = wbase + 32 * i + lane;
                dig[i] = p < m ? (uint32_t)(((K)(key[i] ^ flip) - lo) >> shift) & 0xffu : (uint32_t)kBsRadix;
            }
            if (!VALS && pass == 0) {
                // Keys only: the first LSD pass need not be stable (keys with
                // equal low digits are reordered only among themselves, and
                // every later pass is stable), so one returning atomic ranks.
                constexpr int SH = RankPack<kBsRadix>::kShift;
#pragma unroll
                for (int i = 0; i < IPT; ++i)
                    dr[i] = dig[i] < (uint32_t)kBsRadix
                                ? (atomicAdd(&S.warp_hist[warp][dig[i]], 1u) << SH) | dig[i]
                                : (uint32_t)kBsRadix;
            } else {
                warp_rank<IPT, kBsRadix, kRankBlockSort>(dig, dr, S.warp_hist[warp],
                                                    S.warp_mask[kRankBlockSort == kRankAtomicOr ? warp : 0]);
            }
        }
        __syncthreads();
        for (uint32_t d = tid; d < (uint32_t)kBsRadix; d += THREADS) {
            uint32_t run = 0;
#pragma unroll
            for (int w = 0; w < W; ++w) {
                const uint32_t c = S.warp_hist[w][d];
                S.warp_hist[w][d] = run;
                run += c;
            }
            S.tile_count[d] = run;
        }
        __syncthreads();
        scan_digit_counts<THREADS, kBsRadix>(S.tile_count, S.tile_start, S.scan);
        constexpr int SH = RankPack<kBsRadix>::kShift;
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const uint32_t d = dr[i] & RankPack<kBsRadix>::kMask;
            if (d < (uint32_t)kBsRadix) {
                const uint32_t lp = S.tile_start[d] + S.warp_hist[warp][d] + (dr[i] >> SH);
                if (AHS_DCHECK(lp < m, "blocksort stage", lp)) {
                    S.keys[lp] = key[i];
                    if constexpr (VALS) S.vals[lp] = val[i];
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < IPT; ++i) {
            const uint32_t p = wbase + 32 * i + lane;
            if (p < m) {
                key[i] = S.keys[p];
                if constexpr (VALS) val[i] = S.vals[p];
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t p = wbase + 32 * i + lane;
        if (p < m) {
            keys_out[p] = key[i];
            if constexpr (VALS) vals_out[p] = val[i];
        }
    }
}

// ------------------------------------------------------------ keys only
//
// Without a payload equal keys need no order among themselves, so a bucket
// can be sorted by one counting pass instead of LSD passes: count the keys by
// the top DB bits of u = ord(x) - min (DB chosen so there is about one
// counter per key), place each key at its counter's slot in shared memory,
// then let each thread insertion-sort a range of about IPT staged keys made
// of whole sub-buckets (already in order among themselves).  This is
// the counting sort of Section III-C over the leading bits with an insertion
// sort for the rest.  A sub-bucket of more than kCountRankMax keys with
// different offsets would make the insertion sort quadratic; such a bucket is
// sorted by block_sort's LSD passes instead.
constexpr uint32_t kCountRankMax = 32;

__host__ __device__ constexpr uint32_t log2_floor(uint32_t x) {
    return x > 1 ? 1 + log2_floor(x >> 1) : 0;
}

__host__ __device__ constexpr uint32_t pow2_at_least(uint32_t x) {
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Counter index with one padding word per 32: a thread that scans a run of
// consecutive counters then meets no bank conflict with its neighbours.
__device__ __forceinline__ uint32_t cnt_pad(uint32_t i) { return i + (i >> 5); }

// A run of C counters (C a power of two up to 32) starting at a multiple of C
// lies inside one padded group of 32: its words are consecutive.
template <uint32_t C>
__device__ __forceinline__ uint32_t run_sum(const uint32_t* cnt, uint32_t c0, uint32_t& mx) {
    const uint32_t* p = cnt + cnt_pad(c0);
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < C; ++k) {
        const uint32_t v = p[k];
        sum += v;
        mx = v > mx ? v : mx;
    }
    return sum;
}
template <uint32_t C>
__device__ __forceinline__ void run_starts(uint32_t* cnt, uint32_t c0, uint32_t run) {
    uint32_t* p = cnt + cnt_pad(c0);
#pragma unroll
    for (uint32_t k = 0; k < C; ++k) {
        const uint32_t v = p[k];
        p[k] = run;
        run += v;
    }
}

template <typename K, int THREADS, int IPT>
struct BlockCountSmem {
    static constexpr int W = THREADS / 32;
    static constexpr uint32_t CAP = THREADS * IPT;
    static constexpr uint32_t NB = pow2_at_least(CAP);
    static_assert(NB % 128 == 0, "counters are cleared as 16-byte words");
    alignas(16) uint32_t cnt[NB + NB / 32 + 4];   // counts, then run starts; [cnt_pad(nb)] = m
    uint32_t scan[W + 1];
    unsigned long long red[2][W];
    K keys[CAP];
};

// Dynamic shared memory a bucket kernel needs: the keys-only sort can fall
// back to block_sort in the same bytes.
template <typename K, bool VALS, int THREADS, int IPT>
constexpr size_t block_sort_smem_bytes() {
    return VALS || sizeof(BlockSortSmem<K, VALS, THREADS, IPT>) > sizeof(BlockCountSmem<K, THREADS, IPT>)
               ? sizeof(BlockSortSmem<K, VALS, THREADS, IPT>)
               : sizeof(BlockCountSmem<K, THREADS, IPT>);
}

// block_sort as a separate call, so that its registers are not added to the
// counting path's.
template <typename K, int THREADS, int IPT>
__device__ __noinline__ void block_sort_keys_lsd(const K* keys_in, K* keys_out, uint32_t m, K flip,
                                                 unsigned char* smem, K lo_known, uint32_t bits) {
    block_sort<K, false, THREADS, IPT>(keys_in, keys_out, nullptr, nullptr, m, flip,
                                       *reinterpret_cast<BlockSortSmem<K, false, THREADS, IPT>*>(smem),
                                       lo_known, bits);
}

// Sort keys_in[0..m) (m <= THREADS*IPT) into keys_out[0..m), keys only.
// smem holds block_sort_smem_bytes<K, false, THREADS, IPT>() bytes.
// keys_in may equal keys_out.  lo_known / bits are passed to block_sort
// when it takes over.
template <typename K, int THREADS, int IPT>
__device__ __forceinline__ void block_sort_keys(const K* keys_in, K* keys_out, uint32_t m, K flip,
                                                unsigned char* smem, K lo_known = 0,
                                                uint32_t bits = 0xffu) {
    using CS = BlockCountSmem<K, THREADS, IPT>;
    CS& S = *reinterpret_cast<CS*>(smem);
    constexpr int W = THREADS / 32;
    constexpr int WARP_ITEMS = 32 * IPT;
    const uint32_t tid = threadIdx.x, lane = lane_id(), warp = tid >> 5;
    const uint32_t wbase = warp * WARP_ITEMS;

    // About one counter per key: at most 2^lgc counters, 0.8 m <= 2^lgc < 1.6 m
    // (fewer counters to clear and scan; the insertion sort below meets
    // slightly larger sub-buckets).  Zero them before the first barrier.
    const uint32_t lgc = m > 1 ? bitlen64(m - 1 - m / 5) : 0u;
    {
        uint4* z = reinterpret_cast<uint4*>(S.cnt);
        for (uint32_t i = tid; i < (cnt_pad(1u << lgc) + 3) / 4; i += THREADS)
            z[i] = make_uint4(0u, 0u, 0u, 0u);
    }

    K key[IPT];
    K lo = ~K(0), hi = 0;
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t p = wbase + 32 * i + lane;
        if (p < m) {
            key[i] = keys_in[p];
            const K o = key[i] ^ flip;
            lo = o < lo ? o : lo;
            hi = o > hi ? o : hi;
        } else {
            key[i] = 0;
        }
    }
    {
        const K a = warp_min(lo), b = warp_max(hi);
        if (lane == 0) { S.red[0][warp] = a; S.red[1][warp] = b; }
    }
    __syncthreads();
    {
        unsigned long long a = S.red[0][0], b = S.red[1][0];
#pragma unroll
        for (int w = 1; w < W; ++w) {
            a = S.red[0][w] < a ? S.red[0][w] : a;
            b = S.red[1][w] > b ? S.red[1][w] : b;
        }
        lo = (K)a;
        hi = (K)b;
    }
    const uint32_t D = m ? bitlen64((unsigned long long)(K)(hi - lo)) : 0u;
    if (D == 0) {   // at most one distinct key (block-uniform)
        if (keys_in != keys_out) {
#pragma unroll
            for (int i = 0; i < IPT; ++i) {
                const uint32_t p = wbase + 32 * i + lane;
                if (p < m) keys_out[p] = key[i];
            }
        }
        return;
    }
    const uint32_t DB = D < lgc ? D : lgc;   // lgc >= 1 here, since m >= 2
    const uint32_t R = D - DB;
    const uint32_t nb = 1u << DB;

    // Each key's slot in its counter (< 2^16), two to a register.
    static_assert(THREADS * IPT <= 65536 && IPT % 2 == 0, "slots are packed in 16 bits");
    uint32_t slot[IPT / 2];
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t p = wbase + 32 * i + lane;
        uint32_t r = 0;
        if (p < m) {
            const uint32_t d = (uint32_t)((K)((key[i] ^ flip) - lo) >> R);
            r = atomicAdd(&S.cnt[cnt_pad(d)], 1u);
        }
        if (i & 1) slot[i / 2] |= r << 16;
        else slot[i / 2] = r;
    }
    __syncthreads();

    // Exclusive scan of the nb counters: thread t owns a run of C of them.
    // With a power-of-two block and nb >= THREADS, C = nb / THREADS is a
    // power of two (at most 32) and the runs are unrolled.
    const uint32_t C = (nb + THREADS - 1) / THREADS;
    const uint32_t c0 = tid * C < nb ? tid * C : nb;
    const uint32_t c1 = c0 + C < nb ? c0 + C : nb;
    constexpr uint32_t kLgT = log2_floor(THREADS);
    const int lgC = ((THREADS & (THREADS - 1)) == 0 && nb >= THREADS) ? (int)(DB - kLgT) : -1;
    uint32_t sum = 0, mx = 0;
    switch (lgC) {
        case 0: sum = run_sum<1>(S.cnt, c0, mx); break;
        case 1: sum = run_sum<2>(S.cnt, c0, mx); break;
        case 2: sum = run_sum<4>(S.cnt, c0, mx); break;
        case 3: sum = run_sum<8>(S.cnt, c0, mx); break;
        case 4: sum = run_sum<16>(S.cnt, c0, mx); break;
        case 5: sum = run_sum<32>(S.cnt, c0, mx); break;
        default:
            for (uint32_t c = c0; c < c1; ++c) {
                const uint32_t v = S.cnt[cnt_pad(c)];
                sum += v;
                mx = v > mx ? v : mx;
            }
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan<THREADS>(sum, S.scan, &total);
    switch (lgC) {
        case 0: run_starts<1>(S.cnt, c0, run); break;
        case 1: run_starts<2>(S.cnt, c0, run); break;
        case 2: run_starts<4>(S.cnt, c0, run); break;
        case 3: run_starts<8>(S.cnt, c0, run); break;
        case 4: run_starts<16>(S.cnt, c0, run); break;
        case 5: run_starts<32>(S.cnt, c0, run); break;
        default:
            for (uint32_t c = c0; c < c1; ++c) {
                const uint32_t v = S.cnt[cnt_pad(c)];
                S.cnt[cnt_pad(c)] = run;
                run += v;
            }
    }
    if (tid == 0) S.cnt[cnt_pad(nb)] = m;
    if (__syncthreads_or(R > 0 && mx > kCountRankMax)) {
        // Every thread is past its reads of the counters: the bytes are free.
        block_sort_keys_lsd<K, THREADS, IPT>(keys_in, keys_out, m, flip, smem, lo_known, bits);
        return;
    }

#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t p = wbase + 32 * i + lane;
        if (p < m) {
            const uint32_t d = (uint32_t)((K)((key[i] ^ flip) - lo) >> R);
            const uint32_t lp = S.cnt[cnt_pad(d)] + ((slot[i / 2] >> (16 * (i & 1))) & 0xffffu);
            if (AHS_DCHECK(lp < m, "count sort stage", lp)) S.keys[lp] = key[i];
        }
    }
    __syncthreads();
    if (R > 0) {
        // The staged keys are ordered by their leading DB bits; each
        // sub-bucket is in arbitrary order.  Thread t insertion-sorts the
        // staged keys from the first sub-bucket start at or after t (IPT + 1)
        // to the first at or after (t + 1)(IPT + 1): whole sub-buckets, about
        // IPT + 1 keys a thread, and an odd stride, so that the lanes of a
        // warp read and write different banks.  (THREADS ranges cover m keys:
        // m <= THREADS * IPT.)
        constexpr uint32_t kStride = IPT + 1;
        auto cut = [&](uint32_t q) -> uint32_t {
            if (q >= m) return m;
            const uint32_t d = (uint32_t)((K)((S.keys[q] ^ flip) - lo) >> R);
            const uint32_t b = S.cnt[cnt_pad(d)];
            return b == q ? q : S.cnt[cnt_pad(d + 1)];
        };
        const uint32_t s0 = cut(tid * kStride), s1 = cut(tid * kStride + kStride);
        // In ordered values, the three largest keys so far stay in registers
        // (w0 <= w1 <= w2): each key joins them and the smallest of the four
        // goes to shared memory three places back, without a branch.  Only a
        // key below the last one written (a sub-bucket of five keys or more)
        // is inserted by shifting keys in memory.  The window starts with
        // three copies of the smallest ordered value, whose places fall
        // before s0 and are not written.
        K w0 = 0, w1 = 0, w2 = 0, last = 0;
        for (uint32_t i = s0; i < s1; ++i) {
            const K o = S.keys[i] ^ flip;
            if (o < last) {   // then i - 4 >= s0, and o < w0 <= w1 <= w2
                uint32_t j = i - 3;
                do {
                    S.keys[j] = S.keys[j - 1];
                    --j;
                } while (j > s0 && (K)(S.keys[j - 1] ^ flip) > o);
                S.keys[j] = o ^ flip;
                continue;
            }
            const bool c0 = o < w0, c1 = o < w1, c2 = o < w2;
            const K out = c0 ? o : w0;
            w0 = c0 ? w0 : (c1 ? o : w1);
            w1 = c1 ? w1 : (c2 ? o : w2);
            w2 = c2 ? w2 : o;
            if (i >= s0 + 3) S.keys[i - 3] = out ^ flip;
            last = out;
        }
        if (s1 >= s0 + 3) S.keys[s1 - 3] = w0 ^ flip;
        if (s1 >= s0 + 2) S.keys[s1 - 2] = w1 ^ flip;
        if (s1 >= s0 + 1) S.keys[s1 - 1] = w2 ^ flip;
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t p = wbase + 32 * i + lane;
        if (p < m) keys_out[p] = S.keys[p];
    }
}

}  // namespace ahs
