// libstdc++ std::sort and std::stable_sort on uint32 keys -- TEST
// INFRASTRUCTURE ONLY, timed beside the oracle as the host's library routine
// for context.  It implements nothing of the method; only tests/ and
// bench.py's CPU-baseline leg may load it.
#include <algorithm>
#include <cstdint>
#include <cstring>

extern "C" int orc_std_sort_u32(const uint32_t* in, uint32_t* out, uint64_t n, int stable) {
    if (n && (!in || !out)) return 1;
    if (n) std::memcpy(out, in, n * sizeof(uint32_t));
    if (stable) std::stable_sort(out, out + n);
    else std::sort(out, out + n);
    return 0;
}
