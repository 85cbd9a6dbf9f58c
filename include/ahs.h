/* ahs.h — C ABI of the GB300 (sm_103a) Adaptive Hybrid Sort library.
 *
 * Adaptive Hybrid Sort (arXiv 2506.20677) sorts an array of integer keys by
 * first extracting the state vector v = (n, k, H) (Section III-A: size, value
 * range k = max - min + 1, Shannon entropy H of the key histogram), then
 * choosing a strategy with a finite-state machine (Section III-A, Listing 6)
 * or a trained tree classifier (Section III-H), then running insertion,
 * counting (Listing 2), LSD radix (Listing 3) or a general comparison-class
 * sort (Listing 4: quicksort; here a splitter-based sample sort).
 *
 * Conventions for every function below:
 *  - All functions are extern "C", never throw, and return ahs_status.
 *  - "d_" pointers are CUDA device pointers on the context's device; "h_"
 *    pointers are host pointers.  The caller owns every key / payload buffer.
 *  - Keys are exact integers: AHS_U32, AHS_I32 (4 bytes) or AHS_U64, AHS_I64
 *    (8 bytes), contiguous, any alignment of the element type.  Signed keys
 *    sort in signed order.  An optional payload is uint32 per key.
 *  - Non-integer inputs are refused (Section III-K): bindings map float
 *    dtypes to AHS_ERR_DTYPE; an unknown ahs_key_type is AHS_ERR_DTYPE.
 *  - Streams are cudaStream_t values passed as void* (NULL = legacy default
 *    stream).  Work is enqueued on that stream; functions that return host
 *    results synchronise that stream and say so.
 *  - A context is single-threaded: calls on one ctx must not overlap, except
 *    ahs_serve_submit / ahs_serve_poll, which are thread-safe.
 *  - Device-side waits (decoupled look-back) are bounded; a wait that runs out
 *    returns AHS_ERR_DEVICE_TIMEOUT and leaves the context usable.
 */
#ifndef AHS_H
#define AHS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AHS_VERSION_MAJOR 0
#define AHS_VERSION_MINOR 1

typedef enum {
    AHS_OK = 0,
    AHS_ERR_INVALID_ARG = 1,    /* bad pointer, size, enum value or combination */
    AHS_ERR_DTYPE = 2,          /* keys are not one of the four integer types (Section III-K) */
    AHS_ERR_OOM = 3,            /* device workspace could not be allocated */
    AHS_ERR_BUDGET = 4,         /* a served request can never fit the HBM budget */
    AHS_ERR_CUDA = 5,           /* a CUDA runtime call failed (see ahs_last_cuda_error) */
    AHS_ERR_DEVICE_TIMEOUT = 6, /* a bounded device-side wait ran out */
    AHS_ERR_AGAIN = 7,          /* a served request is not finished yet */
    AHS_ERR_NOT_FOUND = 8,      /* unknown ticket / file */
    AHS_ERR_UNIMPLEMENTED = 9,  /* strategy / type combination not provided */
    AHS_ERR_RANGE = 10          /* forced strategy cannot handle this input's range or size */
} ahs_status;

typedef enum { AHS_U32 = 0, AHS_U64 = 1, AHS_I32 = 2, AHS_I64 = 3 } ahs_key_type;

/* Strategies of Section III-D..G.  IDENTITY copies (n < 2, k == 1, or an input
 * already in order under a profile that checks it).  REVERSE returns an input
 * found in reverse order reversed (§III-B's descending presorted edge case):
 * only an AUTO sort picks it, under a profile that returns presorted inputs
 * by a copy (GB300, MODEL, CUSTOM with sorted_identity), for an input with no
 * ascent and at least one descent -- strictly decreasing when it carries a
 * payload, so that the reversal is the stable order.  It cannot be forced. */
typedef enum {
    AHS_AUTO = 0, AHS_IDENTITY = 1, AHS_SMALL = 2, AHS_COUNTING = 3,
    AHS_RADIX = 4, AHS_GENERAL = 5, AHS_REVERSE = 6
} ahs_strategy;

/* Selector profiles.
 *  PAPER:    the FSM of Section III-A with n_t = 20, k_t = 1000, k_max = 10^6 and
 *            the entropy test H < 0.7 log2 k, evaluated as h = H / log2(nbins) < 0.7.
 *  LISTING6: the same thresholds without the entropy test (Listing 6).
 *  GB300:    the same chain with k_t = 65,536 (the largest range whose counting
 *            histogram is the feature histogram itself, the analogue of Eq. 2),
 *            n_t = the one-block sort capacity, and "already in order" -> IDENTITY.
 *  MODEL:    Section III-H, Table IV.  n < 1000: the static thresholds
 *            n <= 20 -> SMALL and k <= 500 -> COUNTING, then the GB300 rules;
 *            n >= 1000: k == 1 or an input in order -> IDENTITY, otherwise a tree
 *            ensemble evaluated on (log2 n, log2 k, h, key bytes, has payload),
 *            COUNTING only for k <= 65,536 and SMALL only up to the GB300 n_t
 *            (else GENERAL).  Without a loaded table every n takes the small-n
 *            branch.
 *  CUSTOM:   the thresholds given in ahs_config_t.thresholds.
 *  LEMMA32:  Section III-I (Lemma 3.2, Table V), the memory-aware choice for
 *            large ranges: PAPER's chain up to k_max = 10^6; above it COUNTING
 *            when k/n < 5 (high density) or when the number of distinct values
 *            k' is known (ahs_features_t.distinct, from ahs_entropy_exact) and
 *            k' <= 1000 (skewed, k' << k), RADIX when d < 1 + k/n with d from
 *            Eq. 4, else GENERAL.  ahs_select returns the paper's pick; an
 *            AUTO sort runs a COUNTING pick with k > 65,536 on the radix path
 *            (this library's counting sort reads the <= 2^16-bin histogram). */
typedef enum {
    AHS_SEL_PAPER = 0, AHS_SEL_LISTING6 = 1, AHS_SEL_GB300 = 2, AHS_SEL_MODEL = 3,
    AHS_SEL_CUSTOM = 4, AHS_SEL_LEMMA32 = 5
} ahs_select_mode;

/* The state vector of Section III-A with the histogram binning it was taken on.
 * min_bits / max_bits are the smallest / largest key's own bit pattern,
 * zero-extended to 64 bits.  span = max - min as an integer (k = span + 1).
 * The histogram has nbins = (span >> hist_shift) + 1 <= 65,536 bins of
 * (key - min) >> hist_shift, hist_shift = max(0, bitlen(span) - 16); for
 * k <= 65,536 the bins are the key values.  entropy_bits = -sum p log2 p over
 * non-empty bins (fp64), entropy_norm = entropy_bits / log2(nbins) (0 if
 * nbins == 1).  descents = #{i : key[i] > key[i+1]} (0: already in order),
 * ascents = #{i : key[i] < key[i+1]} (0: in reverse order).
 * distinct = k', the number of distinct values, when known (ahs_entropy_exact
 * measures it; the feature pass leaves it 0 = unknown). */
typedef struct {
    uint64_t n;
    uint64_t min_bits;
    uint64_t max_bits;
    uint64_t span;
    uint32_t hist_shift;
    uint32_t nbins;
    double entropy_bits;
    double entropy_norm;
    uint64_t descents;
    uint64_t distinct;
    uint64_t ascents;
} ahs_features_t;

/* FSM thresholds (Section III-A, Table II).  Comparisons follow the text:
 * n <= n_t, k <= k_t, k > k_max, h < h_max. */
typedef struct {
    uint64_t n_t;
    uint64_t k_t;
    uint64_t k_max;
    double h_max;
    int32_t use_entropy;
    int32_t sorted_identity;
} ahs_thresholds_t;

typedef struct {
    int32_t device;              /* CUDA device ordinal; -1: host-only context (selection only) */
    ahs_select_mode select_mode; /* used by ahs_sort / ahs_sort_batch with AHS_AUTO */
    ahs_thresholds_t thresholds; /* for AHS_SEL_CUSTOM */
    const char* model_path;      /* tree table for AHS_SEL_MODEL (NULL: none loaded) */
    uint64_t workspace_limit;    /* bytes of device workspace the ctx may hold, 0 = no limit */
    int32_t timing;              /* 1: record per-phase device times into info structs */
    uint32_t debug_flags;        /* AHS_DEBUG_* test hooks, 0 in normal use */
    const char* tuning_path;     /* tuned-shape table (ahs_load_tuning); NULL: compiled defaults */
} ahs_config_t;

/* Test hook: in every radix pass, tile 1 does not publish its counts, so the
 * later tiles' bounded look-back waits run out (about a second) and the call
 * returns AHS_ERR_DEVICE_TIMEOUT with the context still usable. */
#define AHS_DEBUG_STALL_ONE_TILE 1u
/* Test hook: the feature pass counts its histogram a second time in the
 * split layout, the path it takes when a packed 16-bit counter wraps. */
#define AHS_DEBUG_K2_SPLIT 2u

/* Filled by ahs_sort when non-NULL. */
typedef struct {
    ahs_strategy strategy;       /* the strategy that ran */
    int32_t features_valid;      /* 1 if features below were computed */
    /* With AHS_AUTO under a profile that returns presorted inputs by a copy
     * (sorted_identity: GB300, MODEL, or CUSTOM thresholds that set it), an
     * input found in order (descents == 0) or in reverse order (ascents == 0;
     * with a payload, descents == n - 1) gets no histogram pass: its
     * entropy_bits and entropy_norm are NaN. */
    ahs_features_t features;
    uint32_t passes;             /* radix digit passes run / sample-sort partition levels */
    uint32_t buckets;            /* final buckets sorted in shared memory (general path) */
    float ms_features;           /* device ms of the feature pass (timing = 1) */
    float ms_sort;               /* device ms of the strategy (timing = 1) */
    uint64_t workspace_bytes;    /* device workspace held by the ctx after the call */
} ahs_sort_info_t;

typedef struct {
    uint64_t n_keys;             /* total keys over all segments */
    uint32_t n_seg;
    uint32_t seg_per_strategy[6];/* segments per ahs_strategy value */
    uint64_t keys_per_strategy[6];
    float ms_features;
    float ms_select;             /* host time of the per-segment selection */
    float ms_sort;
} ahs_batch_info_t;

typedef struct ahs_ctx ahs_ctx;

/* ---------------------------------------------------------------- context */

/* Fill *cfg with defaults: device 0, GB300 profile, no model, no limit, no timing. */
void ahs_default_config(ahs_config_t* cfg);
/* Thresholds of a built-in profile (PAPER, LISTING6, GB300). */
ahs_status ahs_profile_thresholds(ahs_select_mode mode, ahs_thresholds_t* out);
/* Create a context on cfg->device (cfg may be NULL for defaults).  The ctx owns
 * its device workspace, which grows on demand and is freed by ahs_destroy. */
ahs_status ahs_create(ahs_ctx** out, const ahs_config_t* cfg);
void ahs_destroy(ahs_ctx* ctx);
const char* ahs_status_str(ahs_status s);
/* Text of the last CUDA error seen by this ctx ("" if none). */
const char* ahs_last_cuda_error(const ahs_ctx* ctx);
/* Load (or replace) the tuned-shape table of the context from a text file
 * written by the library's autotuner (NULL: back to the compiled defaults).
 * The table sets the largest digit width of the stable LSD radix passes
 * (Eq. 4: d = ceil(bitlen(k - 1) / r) passes of r <= 11 bits, chosen per key
 * width, payload and range by measured time) and the batched form's
 * one-block cutoff.  Format:
 *   ahs-tuning 1
 *   radix_bits <key bytes 4|8> <payload 0|1> <span bits 1..64> <digit bits 1..11>
 *   batch_small_cutoff <keys 0..8192>
 * AHS_ERR_NOT_FOUND if the file is missing or malformed (the table is then
 * unchanged). */
ahs_status ahs_load_tuning(ahs_ctx* ctx, const char* path);
/* The radix plan the context's table gives for a key range: pass count and
 * the digit width of the first pass (host only, pure). */
ahs_status ahs_tuned_radix_bits(const ahs_ctx* ctx, uint32_t key_bytes, int32_t has_payload,
                                uint64_t span, uint32_t* passes, uint32_t* digit_bits);
/* Load (or replace) the MODEL profile's tree table from a text file. */
ahs_status ahs_load_model(ahs_ctx* ctx, const char* path);

/* ---------------------------------------------------------------- tracing */

/* One traced kernel launch: the kernel's name (static string), the keys it
 * processed (0 where not meaningful), its device time from CUDA events
 * recorded around it on the launching stream, and when it started, in ms
 * after the start of the first launch of the same collect (the gaps between
 * launches are host work and transfers). */
typedef struct {
    const char* kernel;
    uint64_t items;
    float ms;
    float start_ms;
} ahs_trace_entry_t;

/* Turn per-launch tracing of this ctx's calls on (1) or off (0). */
ahs_status ahs_trace_enable(ahs_ctx* ctx, int32_t on);
/* Wait for and return the launches traced since the last collect (at most
 * cap entries are written; *count receives how many there were), then clear. */
ahs_status ahs_trace_collect(ahs_ctx* ctx, ahs_trace_entry_t* out, uint32_t cap, uint32_t* count);

/* ------------------------------------------------ Section III-A: features */

/* Compute the state vector of d_keys[0..n) on the device (three kernels: a
 * min/max/descent reduction, the <= 2^16-bin histogram, the fp64 entropy
 * reduction) and copy it to *h_out.  Synchronises `stream`. */
ahs_status ahs_features(ahs_ctx* ctx, const void* d_keys, uint64_t n, ahs_key_type type,
                        void* stream, ahs_features_t* h_out);

/* Feature extraction that allocates nothing.  The paper has no counterpart.
 * It serves callers that cannot call cudaMalloc when they need the state
 * vector: code whose device memory is all reserved up front by another
 * allocator or pool (a framework's caching allocator holding the whole HBM),
 * and latency-bound paths that cannot afford the device-wide synchronisation
 * of cudaMalloc / cudaFree.  It runs the same kernels as ahs_features and
 * returns the same result, with no ahs_ctx.  Its scratch is one fixed 48 MiB
 * device array inside the library, held by every GPU that loads the library
 * until the process exits.
 *  - d_keys: device keys on the current device; n <= AHS_NOALLOC_MAX_KEYS.
 *  - The first call on a device (with that device current) resolves the
 *    array's device address for that device; a failed attempt is retried by
 *    the next call.
 *  - All calls share the one array, which keeps the previous call's contents
 *    (each call clears what must start at zero): calls that overlap on the GPU
 *    (other streams, other threads) race and must not be issued.
 *  - Synchronises `stream`; writes *h_out on success.
 * Errors: AHS_ERR_DTYPE for an unknown key type; AHS_ERR_INVALID_ARG for a
 * null h_out or null keys with n > 0; AHS_ERR_RANGE when n exceeds
 * AHS_NOALLOC_MAX_KEYS or when the device has more SMs than the fixed array
 * was sized for (more than about 189); AHS_ERR_CUDA for a failed CUDA call. */
#define AHS_NOALLOC_MAX_KEYS 4294967295ull
ahs_status ahs_features_noalloc(const void* d_keys, uint64_t n, ahs_key_type type, void* stream,
                                ahs_features_t* h_out);

/* Exact per-value entropy (Section III-A: H = -sum over the distinct values v
 * of p_v log2 p_v, p_v = count(v) / n) and the number of distinct values k',
 * measured on the device: a copy of d_keys is sorted by this library (AUTO
 * under the context's profile) into a context-owned side buffer, then the
 * runs of equal keys are measured.  For k <= 65,536 it equals the feature
 * pass's entropy_bits.  n <= 2^32 - 1 (AHS_ERR_RANGE above).  Synchronises
 * `stream`; writes *h_entropy and *h_distinct. */
ahs_status ahs_entropy_exact(ahs_ctx* ctx, const void* d_keys, uint64_t n, ahs_key_type type,
                             void* stream, double* h_entropy, uint64_t* h_distinct);

/* ------------------------------------------- Section III-A / III-H: select */

/* Pure host function: the FSM with explicit thresholds. */
ahs_status ahs_select_fsm(const ahs_features_t* f, const ahs_thresholds_t* t,
                          ahs_strategy* out);
/* Select with a profile (MODEL uses the ctx's loaded tree table; key_bytes and
 * has_payload are model inputs and are ignored by the FSM profiles).  Returns
 * the profile's pick; ahs_sort with AHS_AUTO may differ from it by returning
 * a reversed input by AHS_REVERSE and by running a COUNTING pick over more
 * than 2^16 values on the radix path. */
ahs_status ahs_select(const ahs_ctx* ctx, const ahs_features_t* f, ahs_select_mode mode,
                      uint32_t key_bytes, int32_t has_payload, ahs_strategy* out);

/* ------------------------------------------------------------ the sorts */

/* Sort n keys (and their uint32 payload, stably) from d_keys_in into d_keys_out.
 * d_keys_out may equal d_keys_in (in place); likewise d_vals_out / d_vals_in.
 * d_vals_in == NULL means keys only (d_vals_out is then ignored).
 * force == AHS_AUTO: features -> select (ctx's select_mode) -> strategy; the
 * feature readback synchronises `stream` once.  A forced strategy skips the
 * selector; AHS_COUNTING requires k <= 65,536 (AHS_ERR_RANGE otherwise) and
 * AHS_SMALL requires n <= ahs_small_capacity(type, payload).
 * Output: keys in non-decreasing order; payload in the unique stable order.
 * info may be NULL. */
ahs_status ahs_sort(ahs_ctx* ctx, const void* d_keys_in, void* d_keys_out,
                    const uint32_t* d_vals_in, uint32_t* d_vals_out,
                    uint64_t n, ahs_key_type type, ahs_strategy force,
                    void* stream, ahs_sort_info_t* info);

/* One array in host memory for ahs_sort_host: keys (and optionally a uint32
 * payload) in, sorted keys (and payload) out; outputs may equal inputs. */
typedef struct {
    const void* h_keys_in;
    void* h_keys_out;
    const uint32_t* h_vals_in;   /* NULL for every array, or for none */
    uint32_t* h_vals_out;
    uint64_t n;
} ahs_host_array_t;

/* Sort `count` arrays that live in host memory, each as ahs_sort would (force,
 * the context's profile), end to end: the library copies array i + 1 to the
 * device and array i - 1 back to the host while it sorts array i (three
 * streams and two device buffer pairs owned by the context, kept between
 * calls so that consecutive calls overlap too).  Page-locked host buffers
 * (cudaHostAlloc) let the copies run asynchronously; pageable ones work but
 * do not overlap.  The work starts after the work queued on `stream` so far.
 * wait != 0: returns once every output is in host memory.  wait == 0: returns
 * once everything is queued; ahs_wait_host(ctx, stream) then makes `stream`
 * wait for it (synchronise that stream before reading the outputs).
 * strategies (nullable): receives the strategy each array took.  The host
 * buffers must stay valid until then.  Errors as ahs_sort. */
ahs_status ahs_sort_host(ahs_ctx* ctx, const ahs_host_array_t* arrays, uint32_t count,
                         ahs_key_type type, ahs_strategy force, void* stream, int32_t wait,
                         ahs_strategy* strategies);
/* Make `stream` wait (on the device) for every ahs_sort_host call so far. */
ahs_status ahs_wait_host(ahs_ctx* ctx, void* stream);

/* Largest n the one-block shared-memory sort (AHS_SMALL) takes. */
uint64_t ahs_small_capacity(ahs_key_type type, int32_t has_payload);

/* Sort n_seg independent segments [off[i], off[i+1]) of one key buffer, each
 * with its own features and strategy, using one launch per strategy class.
 * h_seg_offsets: host array of n_seg + 1 non-decreasing offsets (off[0] may be
 * > 0; keys outside [off[0], off[n_seg]) are not touched).  Out-of-place only
 * (d_keys_out != d_keys_in).  Payload as in ahs_sort.  Synchronises `stream`. */
ahs_status ahs_sort_batch(ahs_ctx* ctx, const void* d_keys_in, void* d_keys_out,
                          const uint32_t* d_vals_in, uint32_t* d_vals_out,
                          const uint64_t* h_seg_offsets, uint32_t n_seg,
                          ahs_key_type type, void* stream, ahs_batch_info_t* info);

/* ahs_sort_batch with the n_seg + 1 offsets in device memory (d_seg_offsets,
 * for batches whose layout is produced on the device).  The offsets are read
 * back behind the work already queued on `stream`, then the call proceeds as
 * ahs_sort_batch (same rules and errors).  Synchronises `stream`. */
ahs_status ahs_sort_batch_dev(ahs_ctx* ctx, const void* d_keys_in, void* d_keys_out,
                              const uint32_t* d_vals_in, uint32_t* d_vals_out,
                              const uint64_t* d_seg_offsets, uint32_t n_seg,
                              ahs_key_type type, void* stream, ahs_batch_info_t* info);

/* -------------------------------------------------------------- serving */

typedef struct {
    uint64_t budget_bytes;       /* HBM the in-flight requests may reserve */
    uint32_t max_inflight;       /* requests on the GPU at once */
    uint32_t tick_us;            /* scheduler period when idle */
} ahs_serve_config_t;

/* A served request: n keys of `type`, optionally with a uint32 payload that
 * is sorted stably with them.  Either the caller's device keys (d_keys_in,
 * valid until the request completes) or, with AHS_REQ_GENERATE, keys that
 * the library writes into d_keys_out on the device from (gen_seed, gen_id,
 * gen_kind) -- uint32 keys only, no payload -- before sorting them in place:
 *   gen_kind 0: uniform in [0, 4096);  1: Zipf(1.1) over 1,024 distinct
 *   values;  2: uniform 32-bit;  3: sorted uniform 32-bit with 1% of the
 *   positions replaced by uniform draws (the seeded generators of the
 *   library's workload module, streams 2^40 + 4 gen_id + part). */
#define AHS_REQ_GENERATE 1u
typedef struct {
    const void* d_keys_in;       /* device keys (unused with AHS_REQ_GENERATE) */
    void* d_keys_out;            /* device output (may equal d_keys_in) */
    uint64_t n;
    ahs_key_type type;
    uint32_t flags;              /* AHS_REQ_* */
    const uint32_t* d_vals_in;   /* optional payload (NULL: keys only) */
    uint32_t* d_vals_out;        /* payload output (may equal d_vals_in) */
    uint64_t gen_seed;
    uint64_t gen_id;
    uint32_t gen_kind;
    uint32_t reserved;
} ahs_request_t;

typedef struct {
    ahs_status status;           /* AHS_OK once done */
    ahs_strategy strategy;
    double latency_ms;           /* submit -> completion observed on the host */
    double queue_ms;             /* submit -> admission */
} ahs_result_t;

typedef struct {
    uint64_t completed;
    uint64_t keys;
    double p50_ms, p99_ms;       /* latency percentiles over completed requests */
    uint64_t peak_reserved_bytes;
    uint64_t batches;            /* batched launches issued */
} ahs_serve_stats_t;

/* Start the scheduler thread of a serving loop on this ctx (one per ctx). */
ahs_status ahs_serve_start(ahs_ctx* ctx, const ahs_serve_config_t* cfg);
/* Enqueue a request; *ticket identifies it.  AHS_ERR_BUDGET if its workspace
 * can never fit budget_bytes.  Thread-safe. */
ahs_status ahs_serve_submit(ahs_ctx* ctx, const ahs_request_t* req, uint64_t* ticket);
/* Wait up to timeout_ms (0: just look) for a ticket.  AHS_ERR_AGAIN if not
 * done; on completion fills *out once and forgets the ticket.  Thread-safe. */
ahs_status ahs_serve_poll(ahs_ctx* ctx, uint64_t ticket, int32_t timeout_ms, ahs_result_t* out);
ahs_status ahs_serve_stats(ahs_ctx* ctx, ahs_serve_stats_t* out);
/* Drain in-flight requests and stop the scheduler. */
ahs_status ahs_serve_stop(ahs_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* AHS_H */
