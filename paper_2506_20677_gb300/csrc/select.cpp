// Host-side strategy selection: the finite-state machine of Section III-A
// (with Listing 6 as a profile) and a tree-ensemble evaluator for the learned
// selector of Section III-H.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "select.h"

namespace ahs {

ahs_status profile_thresholds(ahs_select_mode mode, ahs_thresholds_t* t) {
    if (!t) return AHS_ERR_INVALID_ARG;
    // Section III-A text, Listing 6 and Table II: n_t = 20, k_t = 1000, k_max = 10^6,
    // radix only when H < 0.7 log2 k.
    t->n_t = 20;
    t->k_t = 1000;
    t->k_max = 1000000;
    t->h_max = 0.7;
    t->use_entropy = 1;
    t->sorted_identity = 0;
    switch (mode) {
    case AHS_SEL_PAPER:
        return AHS_OK;
    case AHS_SEL_LISTING6:
        t->use_entropy = 0;
        return AHS_OK;
    case AHS_SEL_LEMMA32:
        return AHS_OK;   // its rules above k_max are not thresholds
    case AHS_SEL_GB300:
    case AHS_SEL_MODEL:
        // Eq. 2 sizes k_max from the cache a thread owns; on this GPU the
        // counting histogram lives in one CTA's shared memory and is the
        // feature histogram itself, so k_t = 2^16.  Small inputs go to the
        // one-block shared-memory sort, and an input already in order is
        // returned as is (the descent count is a by-product of the min/max pass).
        t->n_t = kGb300SmallCutoff;
        t->k_t = 65536;
        t->sorted_identity = 1;
        return AHS_OK;
    default:
        return AHS_ERR_INVALID_ARG;
    }
}

ahs_strategy select_fsm(const ahs_features_t& f, const ahs_thresholds_t& p) {
    if (f.n <= 1) return AHS_IDENTITY;
    if (p.sorted_identity && f.descents == 0) return AHS_IDENTITY;
    if (f.n <= p.n_t) return AHS_SMALL;
    if (f.span == 0) return AHS_IDENTITY;
    // k = span + 1 may be 2^64: compare on span to stay in 64 bits.
    //   k <= k_t   <=>  span <= k_t - 1        (k_t >= 1)
    //   k >  k_max <=>  span >= k_max          (k_max >= 0)
    if (p.k_t >= 1 && f.span <= p.k_t - 1) return AHS_COUNTING;
    if (f.span >= p.k_max && (!p.use_entropy || f.entropy_norm < p.h_max)) return AHS_RADIX;
    return AHS_GENERAL;
}

ahs_strategy select_lemma32(const ahs_features_t& f, const ahs_thresholds_t& p) {
    using u128 = unsigned __int128;
    if (f.n <= 1) return AHS_IDENTITY;
    if (f.n <= p.n_t) return AHS_SMALL;
    if (f.span == 0) return AHS_IDENTITY;
    const u128 k = (u128)f.span + 1, n = f.n;
    if (k <= p.k_t) return AHS_COUNTING;
    if (k <= p.k_max) return AHS_GENERAL;
    // Table V: high density (k / n < 5) and skewed ranges (few distinct
    // values, k' << k, taken as k' <= k_t) are counted.
    if (k < 5 * n) return AHS_COUNTING;
    if (f.distinct != 0 && f.distinct <= p.k_t) return AHS_COUNTING;
    // Lemma 3.2: radix when its d passes cost less space than counting's
    // n + k, i.e. d < 1 + k / n, with d = ceil(log_256 k) (Eq. 4).
    u128 reach = 1;
    uint32_t d = 0;
    while (reach < k) {
        reach <<= 8;
        ++d;
    }
    return (u128)(d - 1) * n < k ? AHS_RADIX : AHS_GENERAL;
}

// ------------------------------------------------------------ tree ensemble
//
// Text format (one token stream, whitespace separated):
//   ahs-trees 1
//   classes C  <C strategy codes>
//   features F
//   trees T
//   then per tree:  nodes M  followed by M lines
//      feature threshold left right v_0 .. v_{C-1}
//   feature = -1 marks a leaf (its v_c are the class scores added);
//   internal nodes go left when float32(x[feature]) <= threshold (the rule of
//   the scikit-learn trees the table is written from).
// The predicted class is the argmax of the summed leaf scores (first max wins).

bool TreeModel::load(const char* path, std::string* why) {
    FILE* fp = std::fopen(path, "r");
    if (!fp) { if (why) *why = "cannot open"; return false; }
    char magic[32] = {0};
    int version = 0;
    bool ok = std::fscanf(fp, "%31s %d", magic, &version) == 2 &&
              std::strcmp(magic, "ahs-trees") == 0 && version == 1;
    int C = 0, F = 0, T = 0;
    char word[32];
    ok = ok && std::fscanf(fp, "%31s %d", word, &C) == 2 && C > 0 && C <= 8;
    std::vector<int> cls(C > 0 ? C : 0);
    for (int c = 0; ok && c < C; ++c) ok = std::fscanf(fp, "%d", &cls[c]) == 1;
    ok = ok && std::fscanf(fp, "%31s %d", word, &F) == 2 && F > 0 && F <= 16;
    ok = ok && std::fscanf(fp, "%31s %d", word, &T) == 2 && T > 0 && T <= 4096;
    std::vector<std::vector<Node>> trees;
    for (int t = 0; ok && t < T; ++t) {
        int M = 0;
        ok = std::fscanf(fp, "%31s %d", word, &M) == 2 && M > 0 && M <= 1 << 16;
        std::vector<Node> nodes(ok ? M : 0);
        for (int m = 0; ok && m < M; ++m) {
            Node& nd = nodes[m];
            nd.value.assign(C, 0.0);
            ok = std::fscanf(fp, "%d %lf %d %d", &nd.feature, &nd.threshold, &nd.left, &nd.right) == 4;
            for (int c = 0; ok && c < C; ++c) ok = std::fscanf(fp, "%lf", &nd.value[c]) == 1;
            if (ok && nd.feature >= 0)
                ok = nd.feature < F && nd.left > m && nd.left < M && nd.right > m && nd.right < M;
        }
        if (ok) trees.push_back(std::move(nodes));
    }
    std::fclose(fp);
    if (!ok) { if (why) *why = "malformed tree table"; return false; }
    classes_ = cls;
    n_features_ = F;
    trees_ = std::move(trees);
    return true;
}

int TreeModel::predict(const double* x) const {
    const int C = (int)classes_.size();
    std::vector<double> score(C, 0.0);
    for (const auto& tree : trees_) {
        int m = 0;
        while (tree[m].feature >= 0) {
            const double xv = (double)(float)x[tree[m].feature];
            m = xv <= tree[m].threshold ? tree[m].left : tree[m].right;
        }
        for (int c = 0; c < C; ++c) score[c] += tree[m].value[c];
    }
    int best = 0;
    for (int c = 1; c < C; ++c)
        if (score[c] > score[best]) best = c;
    return classes_[best];
}

// Model inputs (Section III-H uses n, k, H; trees are invariant to monotone
// transforms, so log2 n and log2 k carry the same information).
void model_features(const ahs_features_t& f, uint32_t key_bytes, int32_t has_payload, double* x) {
    x[0] = std::log2((double)(f.n ? f.n : 1));
    x[1] = std::log2((double)f.span + 1.0);
    x[2] = f.entropy_norm;
    x[3] = (double)key_bytes;
    x[4] = has_payload ? 1.0 : 0.0;
}

ahs_strategy select_model(const TreeModel& m, const ahs_features_t& f, uint32_t key_bytes,
                          int32_t has_payload) {
    ahs_thresholds_t t;
    profile_thresholds(AHS_SEL_GB300, &t);
    const bool ordered = t.sorted_identity && f.descents == 0;
    if (f.n < kModelMinN || !m.loaded()) {
        // Table IV's static thresholds for small inputs (insertion sort up to
        // n = 20, counting sort up to k = 500), the GB300 chain after them.
        if (f.n <= 1 || ordered) return AHS_IDENTITY;
        if (f.n <= 20) return AHS_SMALL;
        if (f.span == 0) return AHS_IDENTITY;
        if (f.span < kModelSmallCountingK) return AHS_COUNTING;   // k = span + 1 <= 500
        return select_fsm(f, t);
    }
    if (f.span == 0 || ordered) return AHS_IDENTITY;
    double x[kModelFeatures];
    model_features(f, key_bytes, has_payload, x);
    int s = m.predict(x);
    if (s == AHS_COUNTING && f.span >= kMaxBinsCounting) s = AHS_GENERAL;   // k <= 2^16 only
    if (s == AHS_SMALL && f.n > t.n_t) s = AHS_GENERAL;
    if (s < AHS_IDENTITY || s > AHS_GENERAL) s = AHS_GENERAL;
    return (ahs_strategy)s;
}

}  // namespace ahs
