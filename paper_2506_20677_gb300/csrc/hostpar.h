// Host-side parallel loops for planning work lists: the batched form plans
// tens of thousands of segments between GPU launches, and the host time it
// takes is time the GPU waits.
#pragma once

#include <algorithm>
#include <cstddef>
#include <thread>
#include <vector>

namespace ahs {

// Run fn(chunk, lo, hi) over `chunks` contiguous chunks of [0, n), each on its
// own thread (the first on the caller's).  chunks_for() picks the count.
template <typename F>
void parallel_chunks(size_t n, size_t chunks, F&& fn) {
    if (chunks <= 1 || n < 2) {
        fn(size_t(0), size_t(0), n);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(chunks - 1);
    const size_t per = (n + chunks - 1) / chunks;
    for (size_t c = 1; c < chunks; ++c) {
        const size_t lo = std::min(n, c * per), hi = std::min(n, lo + per);
        th.emplace_back([&fn, c, lo, hi] { fn(c, lo, hi); });
    }
    fn(size_t(0), size_t(0), std::min(n, per));
    for (auto& t : th) t.join();
}

// Threads worth starting for n items of about `grain` items of work each.
inline size_t chunks_for(size_t n, size_t grain) {
    const size_t hw = std::max(1u, std::thread::hardware_concurrency());
    return std::max<size_t>(1, std::min<size_t>({n / std::max<size_t>(grain, 1), hw, 8}));
}

}  // namespace ahs
