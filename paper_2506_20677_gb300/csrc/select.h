// Host-side strategy selection (Section III-A FSM, Section III-H tree model).
#pragma once

#include <string>
#include <vector>

#include "../../include/ahs.h"

namespace ahs {

// n_t of the GB300 profile: inputs this small are sorted by one CTA in
// shared memory (every key type, with or without payload, fits).
constexpr uint64_t kGb300SmallCutoff = 4096;
constexpr int kModelFeatures = 5;
// Section III-H / Table IV: the learned model decides from n = 1000 on; below
// it static thresholds do, counting sort for k <= 500 among them.
constexpr uint64_t kModelMinN = 1000;
constexpr uint64_t kModelSmallCountingK = 500;
// Counting sort reads its histogram from the feature pass: k <= 2^16.
constexpr uint64_t kMaxBinsCounting = 65536;

ahs_status profile_thresholds(ahs_select_mode mode, ahs_thresholds_t* t);
ahs_strategy select_fsm(const ahs_features_t& f, const ahs_thresholds_t& p);
// Section III-I: Lemma 3.2 and Table V above k_max, the FSM's chain below.
ahs_strategy select_lemma32(const ahs_features_t& f, const ahs_thresholds_t& p);

class TreeModel {
public:
    struct Node {
        int feature = -1;
        double threshold = 0.0;
        int left = 0, right = 0;
        std::vector<double> value;
    };
    bool load(const char* path, std::string* why);
    bool loaded() const { return !trees_.empty(); }
    int predict(const double* x) const;

private:
    std::vector<int> classes_;
    int n_features_ = 0;
    std::vector<std::vector<Node>> trees_;
};

void model_features(const ahs_features_t& f, uint32_t key_bytes, int32_t has_payload, double* x);
ahs_strategy select_model(const TreeModel& m, const ahs_features_t& f, uint32_t key_bytes,
                          int32_t has_payload);

}  // namespace ahs
