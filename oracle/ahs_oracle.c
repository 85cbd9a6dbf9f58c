/* Adaptive Hybrid Sort (arXiv 2506.20677): CPU oracle — TEST INFRASTRUCTURE ONLY.
 * See ahs_oracle.h for who may load this file.  Plain C99 + __int128, one
 * thread, no blocking or fusion beyond what each cited definition states.
 */
#include "ahs_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef __int128 val_t;              /* the mathematical value of a key */
typedef unsigned __int128 uval_t;

/* ---------------------------------------------------------------- helpers */

static int valid_type(int t) { return t >= ORC_U32 && t <= ORC_I64; }

static val_t load_key(const void* keys, uint64_t i, int t) {
    switch (t) {
    case ORC_U32: return (val_t)((const uint32_t*)keys)[i];
    case ORC_U64: return (val_t)((const uint64_t*)keys)[i];
    case ORC_I32: return (val_t)((const int32_t*)keys)[i];
    default:      return (val_t)((const int64_t*)keys)[i];
    }
}

static void store_key(void* keys, uint64_t i, int t, val_t v) {
    switch (t) {
    case ORC_U32: ((uint32_t*)keys)[i] = (uint32_t)v; break;
    case ORC_U64: ((uint64_t*)keys)[i] = (uint64_t)v; break;
    case ORC_I32: ((int32_t*)keys)[i] = (int32_t)v; break;
    default:      ((int64_t*)keys)[i] = (int64_t)v; break;
    }
}

static uint64_t key_bits(val_t v, int t) {
    switch (t) {
    case ORC_U32: return (uint64_t)(uint32_t)v;
    case ORC_I32: return (uint64_t)(uint32_t)(int32_t)v;
    default:      return (uint64_t)v; /* two's complement bits of u64 / i64 */
    }
}

static val_t* load_all(const void* keys, uint64_t n, int t) {
    val_t* a = (val_t*)malloc((n ? n : 1) * sizeof(val_t));
    if (!a) return NULL;
    for (uint64_t i = 0; i < n; ++i) a[i] = load_key(keys, i, t);
    return a;
}

static void store_all(void* keys, const val_t* a, uint64_t n, int t) {
    for (uint64_t i = 0; i < n; ++i) store_key(keys, i, t, a[i]);
}

static uint32_t bitlen_u64(uint64_t x) {
    uint32_t b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

/* --------------------------------------------- Section III-A: the state vector */

/* n = |arr|; k = max - min + 1; H = -sum_i p_i log2 p_i (Section III-A, III-H).
 * The sum runs over the bins j = (x - min) >> s of a histogram with at most
 * 2^16 bins, s = max(0, bitlen(max - min) - 16): for k <= 2^16 these bins are
 * the key values themselves and H is the paper's per-value entropy. */
int orc_features(const void* keys, uint64_t n, int t, orc_features_t* f) {
    if (!f || !valid_type(t) || (n && !keys)) return ORC_EINVAL;
    memset(f, 0, sizeof(*f));
    f->n = n;
    if (n == 0) { f->nbins = 0; return ORC_OK; }

    val_t mn = load_key(keys, 0, t), mx = mn;
    uint64_t descents = 0, ascents = 0;
    for (uint64_t i = 0; i < n; ++i) {
        val_t x = load_key(keys, i, t);
        if (x < mn) mn = x;
        if (x > mx) mx = x;
        if (i + 1 < n) {
            val_t y = load_key(keys, i + 1, t);
            if (x > y) ++descents;
            if (x < y) ++ascents;
        }
    }
    uint64_t span = (uint64_t)(mx - mn);
    uint32_t bl = bitlen_u64(span);
    uint32_t s = bl > 16 ? bl - 16 : 0;
    uint64_t nbins = (span >> s) + 1;

    uint64_t* c = (uint64_t*)calloc(nbins, sizeof(uint64_t));
    if (!c) return ORC_ENOMEM;
    for (uint64_t i = 0; i < n; ++i) {
        uint64_t u = (uint64_t)(load_key(keys, i, t) - mn);
        c[u >> s] += 1;
    }
    double H = 0.0;
    for (uint64_t j = 0; j < nbins; ++j) {
        if (c[j] == 0) continue;           /* 0 log 0 = 0 */
        double p = (double)c[j] / (double)n;
        H -= p * log2(p);
    }
    free(c);

    f->min_bits = key_bits(mn, t);
    f->max_bits = key_bits(mx, t);
    f->span = span;
    f->shift = s;
    f->nbins = (uint32_t)nbins;
    f->entropy = H;
    f->entropy_norm = nbins > 1 ? H / log2((double)nbins) : 0.0;
    f->descents = descents;
    f->ascents = ascents;
    return ORC_OK;
}

static int cmp_val(const void* a, const void* b) {
    val_t x = *(const val_t*)a, y = *(const val_t*)b;
    return (x > y) - (x < y);
}

/* The per-value entropy over all k values (no binning): sort, then count runs. */
int orc_entropy_exact(const void* keys, uint64_t n, int t, double* out) {
    if (!out || !valid_type(t)) return ORC_EINVAL;
    *out = 0.0;
    if (n == 0) return ORC_OK;
    val_t* a = load_all(keys, n, t);
    if (!a) return ORC_ENOMEM;
    qsort(a, n, sizeof(val_t), cmp_val);
    double H = 0.0;
    uint64_t run = 1;
    for (uint64_t i = 1; i <= n; ++i) {
        if (i < n && a[i] == a[i - 1]) { ++run; continue; }
        double p = (double)run / (double)n;
        H -= p * log2(p);
        run = 1;
    }
    free(a);
    *out = H;
    return ORC_OK;
}

/* k' = the number of distinct key values (Table V's k'): sorted copy, runs. */
int orc_distinct(const void* keys, uint64_t n, int t, uint64_t* out) {
    if (!out || !valid_type(t)) return ORC_EINVAL;
    *out = 0;
    if (n == 0) return ORC_OK;
    val_t* a = load_all(keys, n, t);
    if (!a) return ORC_ENOMEM;
    qsort(a, n, sizeof(val_t), cmp_val);
    uint64_t k = 1;
    for (uint64_t i = 1; i < n; ++i) k += a[i] != a[i - 1];
    free(a);
    *out = k;
    return ORC_OK;
}

/* ------------------------------------- Section III-A, Listing 6: the decision FSM */

int orc_select(const orc_features_t* f, const orc_fsm_t* p) {
    if (f->n <= 1) return ORC_IDENTITY;                          /* Section I, III-K */
    if (p->sorted_identity && f->descents == 0) return ORC_IDENTITY;
    if (f->n <= p->n_t) return ORC_SMALL;                       /* n <= 20: insertion */
    if (f->span == 0) return ORC_IDENTITY;                       /* k == 1 (III-K) */
    uval_t k = (uval_t)f->span + 1;
    if (k <= (uval_t)p->k_t) return ORC_COUNTING;               /* k <= 1000 */
    if (k > (uval_t)p->k_max && (!p->use_entropy || f->entropy_norm < p->h_max))
        return ORC_RADIX;                                        /* k > 10^6, H < 0.7 log2 k */
    return ORC_GENERAL;                                          /* quicksort */
}

/* Section III-I, Lemma 3.2 and Table V: for large ranges (k > k_max) the
 * memory-aware choice -- counting when k/n < 5 (high density) or when the
 * distinct values are few (k' <= k_t, "k' << k"; distinct = 0 when unknown),
 * radix when d < 1 + k/n with d from Eq. 4, else the general sort.  Below
 * k_max the FSM of Section III-A decides. */
int orc_select_lemma32(const orc_features_t* f, const orc_fsm_t* p, uint64_t distinct) {
    if (f->n <= 1) return ORC_IDENTITY;
    if (f->n <= p->n_t) return ORC_SMALL;
    if (f->span == 0) return ORC_IDENTITY;
    uval_t k = (uval_t)f->span + 1, n = (uval_t)f->n;
    if (k <= (uval_t)p->k_t) return ORC_COUNTING;
    if (k <= (uval_t)p->k_max) return ORC_GENERAL;
    if (k < 5 * n) return ORC_COUNTING;                          /* k / n < 5 */
    if (distinct != 0 && distinct <= p->k_t) return ORC_COUNTING;  /* k' << k */
    uval_t d = orc_radix_passes(f->span);
    if (k > (d - 1) * n) return ORC_RADIX;                      /* d < 1 + k / n */
    return ORC_GENERAL;
}

/* Eq. 4: d = ceil(log_256 k), computed by repeated division. */
uint32_t orc_radix_passes(uint64_t span) {
    uval_t k = (uval_t)span + 1;
    uint32_t d = 0;
    uval_t reach = 1;            /* 256^d */
    while (reach < k) { reach *= 256; ++d; }
    return d;
}

/* ----------------------------------------------- Section III-E: insertion sort */

static void insertion_core(val_t* a, uint32_t* v, uint64_t n) {
    for (uint64_t i = 1; i < n; ++i) {
        val_t key = a[i];
        uint32_t kv = v ? v[i] : 0;
        uint64_t j = i;                      /* a[0, i) is sorted; find key's place */
        while (j > 0 && a[j - 1] > key) {    /* strict > keeps equal keys in order */
            a[j] = a[j - 1];
            if (v) v[j] = v[j - 1];
            --j;
        }
        a[j] = key;
        if (v) v[j] = kv;
    }
}

int orc_insertion_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                       uint64_t n, int t) {
    if (!valid_type(t)) return ORC_EINVAL;
    val_t* a = load_all(keys, n, t);
    if (!a) return ORC_ENOMEM;
    if (vals) memcpy(vals_out, vals, n * sizeof(uint32_t));
    insertion_core(a, vals ? vals_out : NULL, n);
    store_all(out, a, n, t);
    free(a);
    return ORC_OK;
}

/* ------------------------------------------------- Section III-F: counting sort */

/* Section III-F defines counting sort by the frequency of each value,
 * Count[c] = #{j : A[j] - min = c}, and places every key by the accumulated
 * counts of the values before it.  Written from that definition: start[c] =
 * sum of Count[c'] over c' < c is where the first key of value min + c goes,
 * and the keys of one value take start[c], start[c] + 1, ... in input order,
 * so the order is stable. */
int orc_counting_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                      uint64_t n, int t) {
    if (!valid_type(t)) return ORC_EINVAL;
    if (n == 0) return ORC_OK;
    val_t* a = load_all(keys, n, t);
    if (!a) return ORC_ENOMEM;
    val_t mn = a[0], mx = a[0];
    for (uint64_t i = 0; i < n; ++i) { if (a[i] < mn) mn = a[i]; if (a[i] > mx) mx = a[i]; }
    uval_t range = (uval_t)(mx - mn) + 1;
    if (range > ((uval_t)1 << 28)) { free(a); return ORC_ERANGE; }
    uint64_t* start = (uint64_t*)calloc((size_t)range, sizeof(uint64_t));
    val_t* o = (val_t*)malloc(n * sizeof(val_t));
    if (!start || !o) { free(a); free(start); free(o); return ORC_ENOMEM; }
    for (uint64_t i = 0; i < n; ++i) start[(uint64_t)(a[i] - mn)] += 1;   /* Count[c] */
    uint64_t before = 0;                     /* keys of smaller values */
    for (uint64_t c = 0; c < (uint64_t)range; ++c) {
        uint64_t count = start[c];
        start[c] = before;
        before += count;
    }
    for (uint64_t i = 0; i < n; ++i) {       /* input order: equal keys stay in order */
        uint64_t pos = start[(uint64_t)(a[i] - mn)]++;
        o[pos] = a[i];
        if (vals) vals_out[pos] = vals[i];
    }
    store_all(out, o, n, t);
    free(a); free(start); free(o);
    return ORC_OK;
}

/* -------------------------------------------------- Section III-G: LSD radix sort */

/* LSD over u = x - min in base 256 (the base the paper uses for k > 10^6),
 * d = ceil(log_256 k) passes (Eq. 4).  Each pass distributes the keys into 256
 * buckets in input order and concatenates the buckets (stable). */
static int radix_core(val_t* a, uint32_t* v, uint64_t n) {
    if (n == 0) return ORC_OK;
    val_t mn = a[0], mx = a[0];
    for (uint64_t i = 0; i < n; ++i) { if (a[i] < mn) mn = a[i]; if (a[i] > mx) mx = a[i]; }
    uint32_t d = orc_radix_passes((uint64_t)(mx - mn));
    val_t* ta = (val_t*)malloc(n * sizeof(val_t));
    uint32_t* tv = v ? (uint32_t*)malloc(n * sizeof(uint32_t)) : NULL;
    if (!ta || (v && !tv)) { free(ta); free(tv); return ORC_ENOMEM; }
    for (uint32_t digit = 0; digit < d; ++digit) {
        uint64_t bucket_size[256] = {0}, bucket_start[256];
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t u = (uint64_t)(a[i] - mn);
            bucket_size[(u >> (8 * digit)) & 255] += 1;
        }
        uint64_t acc = 0;
        for (int b = 0; b < 256; ++b) { bucket_start[b] = acc; acc += bucket_size[b]; }
        for (uint64_t i = 0; i < n; ++i) {           /* append in input order */
            uint64_t u = (uint64_t)(a[i] - mn);
            uint64_t pos = bucket_start[(u >> (8 * digit)) & 255]++;
            ta[pos] = a[i];
            if (v) tv[pos] = v[i];
        }
        memcpy(a, ta, n * sizeof(val_t));            /* the flattened buckets */
        if (v) memcpy(v, tv, n * sizeof(uint32_t));
    }
    free(ta); free(tv);
    return ORC_OK;
}

int orc_radix_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                   uint64_t n, int t) {
    if (!valid_type(t)) return ORC_EINVAL;
    val_t* a = load_all(keys, n, t);
    if (!a) return ORC_ENOMEM;
    if (vals) memcpy(vals_out, vals, n * sizeof(uint32_t));
    int rc = radix_core(a, vals ? vals_out : NULL, n);
    if (rc == ORC_OK) store_all(out, a, n, t);
    free(a);
    return rc;
}

/* Section III-K, Listing 7 (keys only): split negatives and non-negatives,
 * sort the absolute values of the negatives and the non-negatives separately,
 * reverse the former, restore their sign and concatenate.  Negation is exact
 * in 128 bits. */
int orc_radix_sort_signed_listing7(const void* keys, void* out, uint64_t n, int t) {
    if (!valid_type(t)) return ORC_EINVAL;
    val_t* a = load_all(keys, n, t);
    val_t* neg = (val_t*)malloc((n ? n : 1) * sizeof(val_t));
    val_t* pos = (val_t*)malloc((n ? n : 1) * sizeof(val_t));
    if (!a || !neg || !pos) { free(a); free(neg); free(pos); return ORC_ENOMEM; }
    uint64_t nn = 0, np = 0;
    for (uint64_t i = 0; i < n; ++i) {
        if (a[i] < 0) neg[nn++] = -a[i];
        else pos[np++] = a[i];
    }
    int rc = radix_core(neg, NULL, nn);
    if (rc == ORC_OK) rc = radix_core(pos, NULL, np);
    if (rc == ORC_OK) {
        uint64_t o = 0;
        for (uint64_t i = nn; i-- > 0;) a[o++] = -neg[i];
        for (uint64_t i = 0; i < np; ++i) a[o++] = pos[i];
        store_all(out, a, n, t);
    }
    free(a); free(neg); free(pos);
    return rc;
}

/* ----------------------------- Section III-G(1): quicksort, median-of-three pivot */

static val_t median_of_three(const val_t* a, uint64_t n) {
    val_t x = a[0], y = a[n / 2], z = a[n - 1];
    /* the middle value of the three */
    if (x > y) { val_t tmp = x; x = y; y = tmp; }
    if (y > z) { val_t tmp = y; y = z; z = tmp; }
    if (x > y) { val_t tmp = x; x = y; y = tmp; }
    return y;
}

/* Partition into (< pivot), (== pivot), (> pivot), each in input order; the
 * (== pivot) group keeps every copy of the pivot. */
static void quick_core(val_t* a, val_t* tmp, uint64_t n) {
    while (n > 1) {
        val_t pivot = median_of_three(a, n);
        uint64_t nl = 0, ne = 0, ng = 0;
        for (uint64_t i = 0; i < n; ++i) {
            if (a[i] < pivot) ++nl;
            else if (a[i] == pivot) ++ne;
        }
        ng = n - nl - ne;
        uint64_t il = 0, ie = nl, ig = nl + ne;
        for (uint64_t i = 0; i < n; ++i) {
            if (a[i] < pivot) tmp[il++] = a[i];
            else if (a[i] == pivot) tmp[ie++] = a[i];
            else tmp[ig++] = a[i];
        }
        memcpy(a, tmp, n * sizeof(val_t));
        /* recurse into the smaller side, iterate on the larger (bounded stack) */
        if (nl < ng) {
            quick_core(a, tmp, nl);
            a += nl + ne; tmp += nl + ne; n = ng;
        } else {
            quick_core(a + nl + ne, tmp + nl + ne, ng);
            n = nl;
        }
    }
}

int orc_quicksort(const void* keys, void* out, uint64_t n, int t) {
    if (!valid_type(t)) return ORC_EINVAL;
    val_t* a = load_all(keys, n, t);
    val_t* tmp = (val_t*)malloc((n ? n : 1) * sizeof(val_t));
    if (!a || !tmp) { free(a); free(tmp); return ORC_ENOMEM; }
    quick_core(a, tmp, n);
    store_all(out, a, n, t);
    free(a); free(tmp);
    return ORC_OK;
}

/* ------------------------------------- stable merge sort (general path, payload) */

static void merge_core(val_t* a, uint32_t* v, val_t* ta, uint32_t* tv, uint64_t n) {
    if (n < 2) return;
    uint64_t h = n / 2;
    merge_core(a, v, ta, tv, h);
    merge_core(a + h, v ? v + h : NULL, ta, tv, n - h);
    uint64_t i = 0, j = h, o = 0;
    while (i < h && j < n) {
        if (a[j] < a[i]) { ta[o] = a[j]; if (v) tv[o] = v[j]; ++j; }   /* ties take the left */
        else             { ta[o] = a[i]; if (v) tv[o] = v[i]; ++i; }
        ++o;
    }
    while (i < h) { ta[o] = a[i]; if (v) tv[o] = v[i]; ++i; ++o; }
    while (j < n) { ta[o] = a[j]; if (v) tv[o] = v[j]; ++j; ++o; }
    memcpy(a, ta, n * sizeof(val_t));
    if (v) memcpy(v, tv, n * sizeof(uint32_t));
}

int orc_merge_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
                   uint64_t n, int t) {
    if (!valid_type(t)) return ORC_EINVAL;
    val_t* a = load_all(keys, n, t);
    val_t* ta = (val_t*)malloc((n ? n : 1) * sizeof(val_t));
    uint32_t* tv = vals ? (uint32_t*)malloc((n ? n : 1) * sizeof(uint32_t)) : NULL;
    if (!a || !ta || (vals && !tv)) { free(a); free(ta); free(tv); return ORC_ENOMEM; }
    if (vals) memcpy(vals_out, vals, n * sizeof(uint32_t));
    merge_core(a, vals ? vals_out : NULL, ta, tv, n);
    store_all(out, a, n, t);
    free(a); free(ta); free(tv);
    return ORC_OK;
}

/* --------------------------------------- Section III-H: the learned selector */

struct orc_model {
    int n_classes, n_features, n_trees;
    int* classes;
    int* tree_start;     /* first node of each tree */
    int* feature;        /* per node (-1: leaf) */
    double* threshold;
    int* left;
    int* right;
    double* value;       /* n_classes per node */
};

void orc_model_free(orc_model* m) {
    if (!m) return;
    free(m->classes); free(m->tree_start); free(m->feature); free(m->threshold);
    free(m->left); free(m->right); free(m->value); free(m);
}

orc_model* orc_model_load(const char* path) {
    FILE* fp = fopen(path, "r");
    if (!fp) return NULL;
    orc_model* m = (orc_model*)calloc(1, sizeof(orc_model));
    char word[64];
    int version = 0, ok = 1, cap = 1024, used = 0;
    ok = m && fscanf(fp, "%63s %d", word, &version) == 2 && strcmp(word, "ahs-trees") == 0 && version == 1;
    ok = ok && fscanf(fp, "%63s %d", word, &m->n_classes) == 2 && m->n_classes > 0 && m->n_classes <= 16;
    if (ok) m->classes = (int*)malloc(sizeof(int) * m->n_classes);
    for (int c = 0; ok && c < m->n_classes; ++c) ok = fscanf(fp, "%d", &m->classes[c]) == 1;
    ok = ok && fscanf(fp, "%63s %d", word, &m->n_features) == 2 && m->n_features > 0;
    ok = ok && fscanf(fp, "%63s %d", word, &m->n_trees) == 2 && m->n_trees > 0;
    if (ok) {
        m->tree_start = (int*)malloc(sizeof(int) * (m->n_trees + 1));
        m->feature = (int*)malloc(sizeof(int) * cap);
        m->threshold = (double*)malloc(sizeof(double) * cap);
        m->left = (int*)malloc(sizeof(int) * cap);
        m->right = (int*)malloc(sizeof(int) * cap);
        m->value = (double*)malloc(sizeof(double) * cap * m->n_classes);
    }
    for (int t = 0; ok && t < m->n_trees; ++t) {
        int nodes = 0;
        ok = fscanf(fp, "%63s %d", word, &nodes) == 2 && nodes > 0;
        m->tree_start[t] = used;
        for (int i = 0; ok && i < nodes; ++i) {
            if (used == cap) {
                cap *= 2;
                m->feature = (int*)realloc(m->feature, sizeof(int) * cap);
                m->threshold = (double*)realloc(m->threshold, sizeof(double) * cap);
                m->left = (int*)realloc(m->left, sizeof(int) * cap);
                m->right = (int*)realloc(m->right, sizeof(int) * cap);
                m->value = (double*)realloc(m->value, sizeof(double) * cap * m->n_classes);
            }
            ok = fscanf(fp, "%d %lf %d %d", &m->feature[used], &m->threshold[used], &m->left[used],
                        &m->right[used]) == 4;
            for (int c = 0; ok && c < m->n_classes; ++c)
                ok = fscanf(fp, "%lf", &m->value[(size_t)used * m->n_classes + c]) == 1;
            if (ok && m->feature[used] >= 0)      /* children are local indices of this tree */
                ok = m->feature[used] < m->n_features && m->left[used] > i && m->left[used] < nodes &&
                     m->right[used] > i && m->right[used] < nodes;
            ++used;
        }
    }
    if (ok) m->tree_start[m->n_trees] = used;
    fclose(fp);
    if (!ok) { orc_model_free(m); return NULL; }
    return m;
}

int orc_model_predict(const orc_model* m, const double* x) {
    double score[16] = {0};
    for (int t = 0; t < m->n_trees; ++t) {
        const int base = m->tree_start[t];
        int i = 0;                                   /* local node index */
        while (m->feature[base + i] >= 0) {
            const float xf = (float)x[m->feature[base + i]];
            i = ((double)xf <= m->threshold[base + i]) ? m->left[base + i] : m->right[base + i];
        }
        for (int c = 0; c < m->n_classes; ++c) score[c] += m->value[(size_t)(base + i) * m->n_classes + c];
    }
    int best = 0;
    for (int c = 1; c < m->n_classes; ++c)
        if (score[c] > score[best]) best = c;
    return m->classes[best];
}

int orc_select_model(const orc_features_t* f, const orc_model* m, uint32_t key_bytes, int payload,
                     const orc_fsm_t* rules, uint64_t small_capacity) {
    int s;
    uval_t k = (uval_t)f->span + 1;
    if (f->n < 1000 || !m) {
        /* Section III-H, Table IV: below n = 1000 static thresholds decide --
         * n <= 20 insertion sort, k <= 500 counting sort -- and the profile's
         * rules decide what those two leave. */
        if (f->n <= 1) s = ORC_IDENTITY;
        else if (rules->sorted_identity && f->descents == 0) s = ORC_IDENTITY;
        else if (f->n <= 20) s = ORC_SMALL;
        else if (f->span == 0) s = ORC_IDENTITY;
        else if (k <= 500) s = ORC_COUNTING;
        else s = orc_select(f, rules);
    } else if (f->span == 0 || (rules->sorted_identity && f->descents == 0)) {
        s = ORC_IDENTITY;
    } else {
        double x[5];
        x[0] = log2((double)f->n);
        x[1] = log2((double)f->span + 1.0);
        x[2] = f->entropy_norm;
        x[3] = (double)key_bytes;
        x[4] = payload ? 1.0 : 0.0;
        s = orc_model_predict(m, x);
        if (s == ORC_COUNTING && k > 65536) s = ORC_GENERAL;
        if (s == ORC_SMALL && f->n > rules->n_t) s = ORC_GENERAL;
        if (s < ORC_IDENTITY || s > ORC_GENERAL) s = ORC_GENERAL;
    }
    if (s == ORC_SMALL && f->n > small_capacity) s = ORC_GENERAL;
    return s;
}

/* -------------------------------------------------------- the whole pipeline */

int orc_sort(const void* keys, void* out, const uint32_t* vals, uint32_t* vals_out,
             uint64_t n, int t, int force, const orc_fsm_t* fsm,
             int* chosen, orc_features_t* feat) {
    if (!valid_type(t) || force < ORC_AUTO || force > ORC_GENERAL) return ORC_EINVAL;
    orc_features_t f;
    int rc = orc_features(keys, n, t, &f);
    if (rc != ORC_OK) return rc;
    if (feat) *feat = f;
    int s = force;
    if (s == ORC_AUTO) {
        if (!fsm) return ORC_EINVAL;
        /* The descending presorted edge case (Section III-B): under rules that
         * return presorted inputs by a copy, an input with no ascent and at
         * least one descent is returned reversed -- with a payload only when
         * strictly decreasing, where the reversal is the stable order. */
        if (fsm->sorted_identity && n >= 2 && f.descents > 0 && f.ascents == 0 &&
            (!vals || f.descents == n - 1))
            s = ORC_REVERSE;
        else
            s = orc_select(&f, fsm);
    }
    if (chosen) *chosen = s;
    size_t w = (t == ORC_U32 || t == ORC_I32) ? 4 : 8;
    switch (s) {
    case ORC_IDENTITY:
        if (n) memmove(out, keys, n * w);
        if (vals && n) memmove(vals_out, vals, n * sizeof(uint32_t));
        return ORC_OK;
    case ORC_REVERSE:
        for (uint64_t i = 0; i < n; ++i) {
            memcpy((char*)out + (n - 1 - i) * w, (const char*)keys + i * w, w);
            if (vals) vals_out[n - 1 - i] = vals[i];
        }
        return ORC_OK;
    case ORC_SMALL:    return orc_insertion_sort(keys, out, vals, vals_out, n, t);
    case ORC_COUNTING: return orc_counting_sort(keys, out, vals, vals_out, n, t);
    case ORC_RADIX:    return orc_radix_sort(keys, out, vals, vals_out, n, t);
    default:
        if (vals) return orc_merge_sort(keys, out, vals, vals_out, n, t);
        return orc_quicksort(keys, out, n, t);
    }
}
