/* Adaptive Hybrid Sort (arXiv 2506.20677): CPU oracle — TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-threaded statement of what the method computes, used
 * to check the GPU library against.  It shares no code, header, table or constant with
 * the library under paper_2506_20677_gb300/, and the library never loads it.
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs may load or execute it.
 *
 * Keys are handled as their mathematical integer values (__int128), so every
 * key type (uint32, uint64, int32, int64) and every range k <= 2^64 is exact.
 *
 * Parity pins: every function here is pinned by tests in tests/test_oracle_*.py
 * against library sorts (Python's sorted / numpy), brute force over all
 * permutations of small multisets, closed-form entropies, and the paper's
 * decision thresholds.  Exception, "parity unpinned": the paper's printed
 * dataset entropies (Table VII) fit no stated definition and are not used.
 */
#ifndef AHS_ORACLE_H
#define AHS_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* key types */
enum { ORC_U32 = 0, ORC_U64 = 1, ORC_I32 = 2, ORC_I64 = 3 };
/* strategies (Section III-A: insertion / counting / radix / quick; plus identity) */
enum { ORC_AUTO = 0, ORC_IDENTITY = 1, ORC_SMALL = 2, ORC_COUNTING = 3,
       ORC_RADIX = 4, ORC_GENERAL = 5, ORC_REVERSE = 6 };
/* status */
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ERANGE = -3 };

/* The state vector v = (n, k, H) of Section III-A, plus the binning used for H. */
typedef struct {
    uint64_t n;          /* number of keys */
    uint64_t min_bits;   /* smallest key, its bit pattern in the key type (zero-extended) */
    uint64_t max_bits;   /* largest key, same */
    uint64_t span;       /* max - min as an integer (k = span + 1) */
    uint32_t shift;      /* s = max(0, bitlen(span) - 16) */
    uint32_t nbins;      /* (span >> s) + 1 */
    double   entropy;    /* H = -sum_j p_j log2 p_j, p_j = c_j / n, over c_j > 0 */
    double   entropy_norm; /* h = H / log2(nbins), 0 when nbins == 1 */
    uint64_t descents;   /* number of i with key[i] > key[i+1] (0: already sorted) */
    uint64_t ascents;    /* number of i with key[i] < key[i+1] (0: in reverse order) */
} orc_features_t;

/* Decision thresholds of the finite-state machine (Section III-A, Table II). */
typedef struct {
    uint64_t n_t;          /* n <= n_t -> insertion sort */
    uint64_t k_t;          /* k <= k_t -> counting sort */
    uint64_t k_max;        /* k > k_max and entropy test -> radix sort */
    double   h_max;        /* entropy test: h < h_max (0.7) */
    int32_t  use_entropy;  /* 0: Listing 6 (range test only) */
    int32_t  sorted_identity; /* 1: an already sorted input needs no work */
} orc_fsm_t;

int orc_features(const void* keys, uint64_t n, int key_type, orc_features_t* out);

/* Exact per-value entropy (sum over all k values; diagnostic). */
int orc_entropy_exact(const void* keys, uint64_t n, int key_type, double* out);

int orc_select(const orc_features_t* f, const orc_fsm_t* p);

/* k' = the number of distinct key values. */
int orc_distinct(const void* keys, uint64_t n, int key_type, uint64_t* out);

/* Section III-I (Lemma 3.2, Table V): the memory-aware choice for k > k_max
 * (counting for k/n < 5 or k' <= k_t, radix for d < 1 + k/n, else general);
 * the FSM's rules at and below k_max.  distinct = k', 0 if unknown. */
int orc_select_lemma32(const orc_features_t* f, const orc_fsm_t* p, uint64_t distinct);

/* Radix passes of base 256 over k values: d = ceil(log_256 k) (Eq. 4). */
uint32_t orc_radix_passes(uint64_t span);

/* Forced strategies.  vals may be NULL (keys only).  Outputs may not alias inputs. */
int orc_insertion_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                       uint64_t n, int key_type);
int orc_counting_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                      uint64_t n, int key_type);
int orc_radix_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                   uint64_t n, int key_type);
int orc_radix_sort_signed_listing7(const void* keys, void* out, uint64_t n, int key_type);
int orc_quicksort(const void* keys, void* out, uint64_t n, int key_type);
int orc_merge_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                   uint64_t n, int key_type);

/* Learned selector (Section III-H): a tree table (see the format in
 * paper_2506_20677_gb300/selector/train_trees.py) evaluated on
 * x = (log2 n, log2 k, h, key bytes, has payload).  An inner node goes left
 * when float32(x[f]) <= threshold; the class with the largest summed leaf
 * score wins, the first on ties. */
typedef struct orc_model orc_model;
orc_model* orc_model_load(const char* path);
void orc_model_free(orc_model* m);
int orc_model_predict(const orc_model* m, const double* x);
/* Section III-H / Table IV: below n = 1000 the static thresholds (n <= 20
 * insertion, k <= 500 counting) and then the profile's rules (`rules`); from
 * n = 1000 the model, after the rules' identity cases (k == 1, an ordered input
 * under a profile that returns it as it is).  Counting only for k <= 2^16 and
 * the one-block sort only up to n_t and small_capacity, otherwise the general
 * path. */
int orc_select_model(const orc_features_t* f, const orc_model* m, uint32_t key_bytes, int payload,
                     const orc_fsm_t* rules, uint64_t small_capacity);

/* Features -> select (unless forced) -> run.  *chosen receives the strategy run. */
int orc_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
             uint64_t n, int key_type, int force, const orc_fsm_t* fsm,
             int* chosen, orc_features_t* feat);

#ifdef __cplusplus
}
#endif
#endif
