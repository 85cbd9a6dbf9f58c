// Tuned kernel shapes: a small table written by the autotuner
// (paper_2506_20677_gb300/autotune.py) from CUDA-event timings on the GPU,
// loaded by a context at creation.  Without a table, or for a case the table
// does not cover, the compiled defaults apply.
#pragma once

#include <stdint.h>

#include <string>
#include <vector>

namespace ahs {

// Compiled defaults.
constexpr uint32_t kDefaultRadixDigitBits = 8;   // Listing 3's base 256
constexpr uint32_t kDefaultBatchSmallCutoff = 0;  // 0: the selector decides alone

class Tuning {
public:
    // One row of the radix table: for keys of `key_bytes`, with or without a
    // payload, and key ranges of at most `span_bits` bits, digits of at most
    // `digit_bits` bits (1..11).
    struct RadixRow {
        uint32_t key_bytes;
        uint32_t payload;
        uint32_t span_bits;
        uint32_t digit_bits;
    };
    // Text format (whitespace separated, '#' starts a comment line):
    //   ahs-tuning 1
    //   radix_bits <key_bytes 4|8> <payload 0|1> <span_bits 1..64> <digit_bits 1..11>
    //   batch_small_cutoff <keys 0..8192>
    // Rows of one (key_bytes, payload) are matched in order of increasing
    // span_bits.  A malformed file loads nothing and returns false.
    bool load(const char* path, std::string* why);
    void clear();
    bool loaded() const { return loaded_; }
    uint32_t radix_digit_bits(uint32_t key_bytes, bool payload, uint32_t span_bits) const;
    uint32_t batch_small_cutoff() const { return batch_small_cutoff_; }

private:
    bool loaded_ = false;
    std::vector<RadixRow> radix_;
    uint32_t batch_small_cutoff_ = kDefaultBatchSmallCutoff;
};

}  // namespace ahs
