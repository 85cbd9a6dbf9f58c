// Stable warp-level ranking by digit: the core of every partition kernel.
//
// A warp holds IPT items per lane in "warp-striped" order (item i of lane l
// is the (32 i + l)-th of the warp's keys, so i-major then lane order is input
// order).  For each item it finds the peers with the same digit among the 32
// lanes, adds the group size to the warp's private counter of that digit, and
// returns the item's rank = counter before the group + peers of lower lane.
// Items whose digit is NB (past the end of the data) are skipped.
//
// Three ways of finding the peers, selected at compile time:
//  kRankMatch    the warp match instruction;
//  kRankBallot   one ballot per digit bit, intersected (multisplit);
//  kRankAtomicOr each lane ORs its lane bit into a per-digit mask in shared
//                memory; after a warp barrier the mask is the peer set, and the
//                group leader clears it after the counter update.
// The result is packed as (rank << SHIFT) | digit, SHIFT = bits to hold NB.
#pragma once

#include "common.cuh"

namespace ahs {

enum RankAlgo { kRankMatch = 0, kRankBallot = 1, kRankAtomicOr = 2 };

// Algorithm of each kernel family, chosen by measurement on GB300 (match,
// ballot and atomic-or variants timed on the same inputs).
constexpr int kRankOnesweep = kRankBallot;
constexpr int kRankScatter = kRankBallot;
constexpr int kRankBlockSort = kRankAtomicOr;

template <int NB>
struct RankPack {
    static constexpr int kShift = NB <= 256 ? 9 : (NB <= 512 ? 10 : 12);
    static constexpr uint32_t kMask = (1u << kShift) - 1;
};

// PACK: write (rank << SHIFT) | digit into out[i]; otherwise write the rank.
template <int IPT, int NB, int ALGO, bool PACK = true>
__device__ __forceinline__ void warp_rank(const uint32_t (&dig)[IPT], uint32_t (&out)[IPT],
                                          uint32_t* wh, uint32_t* wmask) {
    constexpr int SH = RankPack<NB>::kShift;
    const uint32_t lane = lane_id();
    const uint32_t lt = lanemask_lt();
#pragma unroll
    for (int i = 0; i < IPT; ++i) {
        const uint32_t d = dig[i];
        const bool valid = d < (uint32_t)NB;
        uint32_t peers;
        if constexpr (ALGO == kRankMatch) {
            peers = __match_any_sync(AHS_FULL_MASK, d);
        } else if constexpr (ALGO == kRankBallot) {
            constexpr int BITS = NB <= 2 ? 1 : 32 - __builtin_clz(NB - 1);
            peers = __ballot_sync(AHS_FULL_MASK, valid);
#pragma unroll
            for (int b = 0; b < BITS; ++b) {
                const bool bit = (d >> b) & 1u;
                const uint32_t m = __ballot_sync(AHS_FULL_MASK, bit);
                peers &= bit ? m : ~m;
            }
        } else {
            if (valid) atomicOr(&wmask[d], 1u << lane);
            __syncwarp();
            peers = valid ? wmask[d] : 0u;
            __syncwarp();
        }
        uint32_t leader = valid ? __ffs(peers) - 1 : lane;
        uint32_t old = 0;
        if (valid && lane == leader) {
            old = atomicAdd(&wh[d], __popc(peers));
            if constexpr (ALGO == kRankAtomicOr) wmask[d] = 0;
        }
        if constexpr (ALGO == kRankAtomicOr) __syncwarp();
        old = __shfl_sync(AHS_FULL_MASK, old, leader);
        if constexpr (PACK) out[i] = ((old + __popc(peers & lt)) << SH) | (valid ? d : (uint32_t)NB);
        else out[i] = old + __popc(peers & lt);
    }
}

}  // namespace ahs
