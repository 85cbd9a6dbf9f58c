// Loader and lookups of the tuned-shape table (see tuning.h).
#include "tuning.h"

#include <algorithm>
#include <cstdio>
#include <cstring>

namespace ahs {

void Tuning::clear() {
    loaded_ = false;
    radix_.clear();
    batch_small_cutoff_ = kDefaultBatchSmallCutoff;
}

bool Tuning::load(const char* path, std::string* why) {
    FILE* fp = path ? std::fopen(path, "r") : nullptr;
    if (!fp) {
        if (why) *why = "cannot open";
        return false;
    }
    std::vector<RadixRow> rows;
    uint32_t cutoff = kDefaultBatchSmallCutoff;
    bool ok = false, header = false;
    char line[512];
    while (std::fgets(line, sizeof line, fp)) {
        char word[64] = {0};
        if (std::sscanf(line, "%63s", word) != 1 || word[0] == '#') continue;
        if (!header) {
            int version = 0;
            header = std::sscanf(line, "%63s %d", word, &version) == 2 &&
                     std::strcmp(word, "ahs-tuning") == 0 && version == 1;
            if (!header) break;
            ok = true;
            continue;
        }
        if (std::strcmp(word, "radix_bits") == 0) {
            unsigned kb = 0, pay = 0, span = 0, bits = 0;
            if (std::sscanf(line, "%63s %u %u %u %u", word, &kb, &pay, &span, &bits) != 5 ||
                (kb != 4 && kb != 8) || pay > 1 || span < 1 || span > 64 || bits < 1 || bits > 11) {
                ok = false;
                break;
            }
            rows.push_back({kb, pay, span, bits});
        } else if (std::strcmp(word, "batch_small_cutoff") == 0) {
            unsigned c = 0;
            if (std::sscanf(line, "%63s %u", word, &c) != 2 || c > 8192) {
                ok = false;
                break;
            }
            cutoff = c;
        } else {
            ok = false;
            break;
        }
    }
    std::fclose(fp);
    if (!ok) {
        if (why) *why = "malformed tuning table";
        return false;
    }
    std::stable_sort(rows.begin(), rows.end(), [](const RadixRow& a, const RadixRow& b) {
        return a.span_bits < b.span_bits;
    });
    radix_ = std::move(rows);
    batch_small_cutoff_ = cutoff;
    loaded_ = true;
    return true;
}

uint32_t Tuning::radix_digit_bits(uint32_t key_bytes, bool payload, uint32_t span_bits) const {
    for (const RadixRow& r : radix_)
        if (r.key_bytes == key_bytes && r.payload == (payload ? 1u : 0u) && span_bits <= r.span_bits)
            return r.digit_bits;
    return kDefaultRadixDigitBits;
}

}  // namespace ahs
