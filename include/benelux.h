/*
 * benelux.h -- C ABI of libbenelux, a GB300 (sm_103a) search for Benelux pairs.
 *
 * Method: Hercher, "On one of Erdos' Problems -- An Efficient Search for
 * Benelux Pairs" (arXiv 2506.01099).
 *
 *   rad(x)       product of the distinct primes dividing x; rad(1) = 1 (Sec. 2.1)
 *   first kind   1 <= m < n with rad(m) = rad(n) and rad(m+1) = rad(n+1) (Sec. 1)
 *   second kind  1 <= m < n with rad(m) = rad(n+1) and rad(m+1) = rad(n) (Sec. 1)
 *
 * A search over an n-range [lo, hi) reports every pair (m, n) of the requested
 * kinds with lo <= n < hi and any 1 <= m < n: the contract of Algorithm 3
 * (Sec. 2.2), which reports the pairs whose larger member lies in the chunk.
 * Pairs come back sorted by (n, m, kind).
 *
 * Conventions for every call:
 *  - Return value: BNX_OK (0) or one of the BNX_E_* codes below; no C++
 *    exception crosses this boundary.  bnx_strerror() names a code, and
 *    bnx_last_error() gives the message of the last failure on this thread.
 *  - `kinds` is a bit mask: 1 = first kind, 2 = second kind, 4 = three-term
 *    pairs (first-kind pairs with also rad(m+2) = rad(n+2): Erdos's original
 *    question quoted in Sec. 1; reported with kind 4).  bnx_search_hash takes
 *    1, 2 or 3.
 *  - Ranges: 1 <= lo < hi <= max_hi, where max_hi is fixed at bnx_create and is
 *    at most BNX_MAX_HI = 2^42 (so that 2n and every intermediate fit in 64 bits).
 *  - Output buffers are owned by the caller.  The library owns its device
 *    tables and workspace (allocated with cudaMalloc, freed by bnx_destroy).
 *  - When a pair buffer is too small the call returns BNX_E_TRUNCATED, writes
 *    the first `cap` pairs and still stores the exact count in *n_out.
 *  - A context is bound to one device and one CUDA stream; calls on one context
 *    must not run concurrently.  Different contexts are independent.
 *  - Synchronous calls (bnx_search, bnx_search_hash, bnx_batch) return after the
 *    device work is complete.  bnx_rad_segment is asynchronous on the stream.
 */
#ifndef BENELUX_H
#define BENELUX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BNX_OK 0
#define BNX_E_ARG 1        /* an argument is out of range or a pointer is NULL */
#define BNX_E_TRUNCATED 2  /* the output buffer was too small; *n_out is exact */
#define BNX_E_NOMEM 3      /* a device or host allocation failed, or admission refused */
#define BNX_E_CUDA 4       /* a CUDA runtime call or kernel launch failed */
#define BNX_E_TIMEOUT 5    /* a bounded device or host wait gave up */
#define BNX_E_BUSY 6       /* a served request is not finished yet */
#define BNX_E_STATE 7      /* the call does not fit the context's state */
#define BNX_E_OVERFLOW 8   /* a device-side capacity was exceeded */
#define BNX_E_CANCELLED 9  /* a served request was cancelled before it finished */

#define BNX_MAX_HI ((uint64_t)1 << 42)

typedef struct bnx_ctx bnx_ctx;

/* One reported pair.  kind is 1, 2 or 4 (three-term). */
typedef struct {
    uint64_t m, n;
    uint32_t kind;
    uint32_t iv; /* index of the interval (bnx_batch) or 0 */
} bnx_pair;

/* One n-range [lo, hi) with its kind mask and a caller tag. */
typedef struct {
    uint64_t lo, hi;
    uint32_t kinds;
    uint32_t id;
} bnx_interval;

/* Tunable launch parameters (all optional in the JSON given to bnx_create). */
typedef struct {
    uint32_t tile_log2;    /* shared-memory tile: 2^tile_log2 integers (10..16; the exact
                              tile uses at most 2^14 and walks a longer one in pieces) */
    uint32_t seg_tiles;    /* tiles per queue segment (1..64) */
    uint32_t threads;      /* threads per CTA (256, 512 or 1024) */
    uint32_t ctas_per_sm;  /* resident CTAs per SM for the persistent grid (0 = occupancy limit) */
    uint32_t small_q_log2; /* prime powers q <= 2^small_q_log2 are struck in shared
                              memory, larger ones come from the HBM buckets (8..16) */
    uint32_t tile_kind;    /* searches: log-domain tile of 0 = u32, 2 = u16 or 3 = u8 values
                              (each with exact re-check of candidates), 1 = exact u64
                              square-part tile */
} bnx_tune;

/* Per-call counters of the last search on a context. */
typedef struct {
    uint64_t integers;     /* n values searched */
    uint64_t segments;     /* queue segments processed */
    uint64_t bucket_hits;  /* large prime-power hits written to the buckets */
    uint64_t survivors1;   /* n passing the first-kind necessary condition */
    uint64_t survivors2;   /* n passing the second-kind necessary condition */
    uint64_t candidates;   /* candidate m values verified */
    uint64_t pairs;        /* pairs found */
    uint64_t hash_keys;    /* keys inserted (bnx_search_hash) */
    float ms_total;        /* device time of the whole call (CUDA events) */
    float ms_sieve;        /* device time of the sieve kernel launches */
    uint32_t sieve_launches;
    uint32_t pad;
} bnx_stats;

/* ------------------------------------------------------------------------ */
/* Context                                                                    */
/* ------------------------------------------------------------------------ */

/* Create a context on `device` for ranges up to max_hi (<= BNX_MAX_HI).  Builds
 * the device-resident tables of Sec. 3.1 ("the list of primes ... sent to the
 * GPU" once): every prime p <= sqrt(max_hi) by a device sieve, the prime powers
 * p^k (k >= 2) <= max_hi, and per-entry constants.  `tune_json` is NULL or a
 * JSON object with any of the bnx_tune field names; missing fields take the
 * built-in defaults.  `stream` is a cudaStream_t to run on, or NULL for a new
 * stream owned by the context.  Errors: BNX_E_ARG, BNX_E_NOMEM, BNX_E_CUDA. */
int bnx_create(bnx_ctx **out, int device, uint64_t max_hi, const char *tune_json, void *stream);

/* Free every device and host resource of the context (NULL is accepted). */
void bnx_destroy(bnx_ctx *ctx);

/* Parse a tuning JSON object (the form bnx_create takes and bnx_autotune
 * writes) into *out: the built-in defaults, overridden by the object's fields.
 * The object is flat; its keys are bnx_tune's field names with non-negative
 * integer values, plus "ms" (any number, ignored).  Unknown or repeated keys,
 * non-integers, values beyond 32 bits, values outside the ranges bnx_tune
 * states, and text after the object give BNX_E_ARG (and leave *out as it
 * was).  Host code only; bnx_create applies the same reader. */
int bnx_tune_parse(const char *json, bnx_tune *out);

/* Read or replace the tuning of a context (replacing frees cached graphs). */
int bnx_get_tune(const bnx_ctx *ctx, bnx_tune *out);
int bnx_set_tune(bnx_ctx *ctx, const bnx_tune *tune);

/* Counters of the last completed search on this context. */
int bnx_get_stats(const bnx_ctx *ctx, bnx_stats *out);

/* Number of primes <= sqrt(max_hi) held on the device. */
int bnx_prime_count(const bnx_ctx *ctx, uint64_t *out);

/* ------------------------------------------------------------------------ */
/* Segment-level calls                                                         */
/* ------------------------------------------------------------------------ */

/* Radicals of x in [lo, lo+len): rad_out[i] = rad(lo+i) and, when sq_out is not
 * NULL, sq_out[i] = (lo+i) / rad(lo+i), the product of p^(e-1) over p^e || x.
 * This is the output of Algorithm 1 (Sec. 2.1), computed by the same
 * shared-memory tile sieve as the search.  rad_out and sq_out (uint64_t, len
 * elements, 8-byte aligned) are both DEVICE pointers or both HOST pointers:
 *  - device buffers: the call is asynchronous on `stream` (NULL: the
 *    context's stream);
 *  - host buffers (pageable or pinned): the values are sieved into a device
 *    staging buffer owned by the context (kept up to 256 MiB, freed after the
 *    call above that), copied back on `stream`, and the call returns once they
 *    are written.
 * 1 <= lo, lo + len <= max_hi, 1 <= len <= 2^31.
 * Errors: BNX_E_ARG, BNX_E_NOMEM, BNX_E_CUDA. */
int bnx_rad_segment(bnx_ctx *ctx, uint64_t lo, uint64_t len, uint64_t *rad_out, uint64_t *sq_out, void *stream);

/* Segment-level search: all pairs (m, n) of the requested kinds with
 * lo <= n < lo + len and any m < n -- the output Algorithm 3 (Sec. 2.2) gives
 * for one chunk C_i, for a caller that drives its own loop over segments (the
 * paper's host passes only the chunk number down, Sec. 3.1).  The same staged
 * pipeline as bnx_search (sieve, per-kind CRT conditions, compaction,
 * verification) over the one segment; a segment's pairs do not depend on any
 * other segment, so consecutive segments concatenate to bnx_search's result.
 * `out` is a HOST buffer of `cap` pairs sorted by (n, m, kind).  Blocking.
 * 1 <= len < 2^32, 1 <= lo, lo + len <= max_hi.
 * Errors: BNX_E_ARG, BNX_E_TRUNCATED, BNX_E_NOMEM, BNX_E_CUDA, BNX_E_OVERFLOW. */
int bnx_search_segment(bnx_ctx *ctx, uint64_t lo, uint32_t len, uint32_t kinds, bnx_pair *out, size_t cap,
                       size_t *n_out);

/* Checkpointed search: all pairs with lo <= n < hi of the given kinds, as
 * bnx_search finds them, run as consecutive chunks of `chunk` integers.  After
 * each chunk the progress -- the search (lo, hi, kinds), the next n to search
 * and the pairs found so far -- is written to the file `path` (a new file
 * renamed over the old one, so the file always holds a finished chunk).  A call
 * that finds a checkpoint of the same search in `path` resumes after its last
 * chunk; a checkpoint of another search gives BNX_E_STATE, an unreadable one
 * BNX_E_ARG.  The paper's long search (Sec. 3.1) keeps only its chunk number;
 * this keeps the pairs too, so a resumed search returns them all.
 *  - max_chunks: at most that many chunks this call (BNX_CKPT_ALL: to hi; 0:
 *    none, only the saved pairs are returned); a search not finished after them
 *    returns BNX_E_BUSY (call again to go on), with the pairs so far in `out`.
 *  - *next (may be NULL): the next n to search (hi once finished).
 *  - out, cap, n_out: as bnx_search (HOST buffer, sorted by (n, m, kind)); on
 *    BNX_E_TRUNCATED the progress is saved, and a call with max_chunks = 0 and a
 *    larger buffer returns the pairs without searching.
 * A finished search leaves its checkpoint (next = hi), so calling again returns
 * the pairs without searching.  Blocking.  Errors: BNX_E_ARG, BNX_E_STATE,
 * BNX_E_BUSY, BNX_E_TRUNCATED, BNX_E_NOMEM, BNX_E_CUDA, BNX_E_OVERFLOW. */
#define BNX_CKPT_ALL UINT64_MAX
int bnx_search_checkpointed(bnx_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t kinds, const char *path,
                            uint64_t chunk, uint64_t max_chunks, bnx_pair *out, size_t cap, size_t *n_out,
                            uint64_t *next);

/* Radicals of [lo, lo+len) without allocating any device memory -- for
 * callers that cannot call cudaMalloc (their device memory is owned by another
 * allocator or budget, or they run where allocation is not allowed).  The
 * paper has no counterpart to this entry point; it returns what
 * bnx_rad_segment returns, needs no context, and does all of its work in a
 * fixed scratch array of BNX_NOALLOC_SCRATCH_BYTES compiled into the library,
 * which every GPU that loads the library keeps until the process exits.
 *  - rad_out / sq_out: caller DEVICE buffers of len uint64_t (sq_out may be
 *    NULL); the work is queued on `stream` (NULL: the legacy default stream)
 *    on the current device.
 *  - Limits: 1 <= lo, 1 <= len <= BNX_NOALLOC_MAX_LEN, lo + len <= BNX_NOALLOC_MAX_HI;
 *    anything larger is rejected with BNX_E_ARG.
 *  - The first call on a device looks up the scratch's device address
 *    (cudaGetSymbolAddress); make that first call before any stream capture.
 *    The address is then kept per device ordinal for the life of the process,
 *    so it belongs to the device's primary context: do not use this entry
 *    point after cudaDeviceReset on that device, or with another CUDA context
 *    current on it.
 *  - Every call uses the same scratch: calls that may overlap on the GPU
 *    (different streams, or threads without ordering) race.  Each call
 *    re-initialises the scratch it reads, so back-to-back calls are independent.
 * Errors: BNX_E_ARG, BNX_E_CUDA. */
#define BNX_NOALLOC_MAX_LEN ((uint64_t)1 << 18)
#define BNX_NOALLOC_MAX_HI ((uint64_t)1 << 40)
#define BNX_NOALLOC_SCRATCH_BYTES 3145984u
int bnx_rad_segment_noalloc(uint64_t lo, uint64_t len, uint64_t *rad_out, uint64_t *sq_out, void *stream);

/* ------------------------------------------------------------------------ */
/* Log weights of the filter                                                  */
/* ------------------------------------------------------------------------ */

/* The log-domain tiles bound the odd square part s of rad's complement x/rad(x)
 * (Algorithm 1, Sec. 2.1, records the same prime-power hits) from above by a
 * sum of per-prime weights, and reject n when the bound cannot meet the
 * per-kind necessary condition.  That is exact only if every weight is at
 * least F log2 p, F the tile's units per bit.  bnx_log_weight(p, f) is the
 * smallest integer L with 2^L > p^(2^f) -- the bit length of p^(2^f) --
 * computed in integers by repeated squaring with upward rounding; it never
 * falls below the bit length and equals it unless a rounding tie intervenes.
 * Host code only (no GPU needed); 2 <= p < 2^32, f <= 16, else 0.  The u16 and
 * u32 tiles use it with F = 2^8 and 2^16. */
uint32_t bnx_log_weight(uint64_t p, uint32_t frac_log2);

/* The u8 tile's weight, in units of 4/5 bit (F = 5/4): ceil(bitlen(p^5) / 4),
 * with p^5 computed exactly in 128-bit integers.  bitlen(p^5) > 5 log2 p, so the
 * weight exceeds (5/4) log2 p.  At most 1.468 units per bit of p (p = 17), so a
 * u8 value stays below 2^6 and a pair sum below 2^7 for n < 2^42.  Host code
 * only; 2 <= p < 2^25, else 0. */
uint32_t bnx_log_weight54(uint64_t p);

/* For every prime p <= sqrt(max_hi) of the context's device table (ascending),
 * the weights the log tile `tile_kind` (0 = u32, 2 = u16, 3 = u8) adds, read
 * along the kernels' own code paths on the device: out[4i .. 4i+4) =
 * {p, in-tile strike weight, weight of a bucket hit through the shared-memory
 * cache, weight of a bucket hit read from global memory}, in units of 2^-16,
 * 2^-8 or 4/5 bit.  `out` is a HOST buffer of 4 * cap uint32_t; *n_out is the
 * number of primes.  Blocking.  Errors: BNX_E_ARG, BNX_E_TRUNCATED, BNX_E_CUDA. */
int bnx_log_weights(bnx_ctx *ctx, uint32_t tile_kind, uint32_t *out, size_t cap, size_t *n_out);

/* rad(x[i]) == rad(y[i]) for n pairs, on the current device, by the gcd strips
 * the verification kernel applies to a candidate (the same device function:
 * strip from x every common factor with y until 1 remains, and the same the
 * other way).  This is the test behind Erdos's three-term question (Sec. 1):
 * a first-kind pair (m, n) is also a three-term pair when rad(m+2) = rad(n+2).
 * x, y are HOST arrays of n values >= 1; out is a HOST array of n bytes
 * (1: equal radicals, 0: not); n <= 2^24.  Device scratch is allocated and
 * freed inside the call; blocking.  Errors: BNX_E_ARG, BNX_E_NOMEM, BNX_E_CUDA. */
int bnx_same_rad(const uint64_t *x, const uint64_t *y, size_t n, uint8_t *out);

/* ------------------------------------------------------------------------ */
/* Searches                                                                    */
/* ------------------------------------------------------------------------ */

/* Plain path: all pairs with lo <= n < hi.  The range is cut into queue
 * segments; per segment the tile sieve (Algorithm 1 restated per tile), the key
 * (rad n, rad n+1) of Sec. 2.1, the exact per-kind necessary conditions forced
 * by the Chinese remainder theorem (first kind rad(n)rad(n+1) | n - m, second
 * kind rad(n)rad(n+1) | m + n + 1), warp-ballot compaction of survivors, and
 * candidate verification.  `out` is a HOST buffer of `cap` pairs.  Blocking.
 * Errors: BNX_E_ARG, BNX_E_TRUNCATED, BNX_E_NOMEM, BNX_E_CUDA, BNX_E_OVERFLOW. */
int bnx_search(bnx_ctx *ctx, uint64_t lo, uint64_t hi, uint32_t kinds, bnx_pair *out, size_t cap, size_t *n_out);

/* Full-range search by collision detection, as in Algorithms 2 and 3: all
 * pairs with m < n < S.  Every x < S whose key (rad x, rad x+1) can belong to a
 * pair (rad(x)rad(x+1) <= 2S) is inserted into a device open-addressing hash
 * table keyed by the 2-set; every two integers with equal keys form a pair, of
 * the first kind when rad(m) = rad(n) (Algorithm 2's rule).  2 <= S <= 2^40.
 * `out` is a HOST buffer.  Blocking.  Errors as bnx_search. */
int bnx_search_hash(bnx_ctx *ctx, uint64_t S, uint32_t kinds, bnx_pair *out, size_t cap, size_t *n_out);

/* Algorithm 3 (Sec. 2.2) as the paper runs it, kept as a measured baseline:
 * all pairs with m < n < S by chunks of 2^chunk_log2 integers.  For each chunk
 * C_i every n's key {rad n, rad n+1} goes into an open-addressing table of
 * 4 * 2^chunk_log2 slots (collisions inside C_i give pairs), then every earlier
 * chunk C_j is sieved again and probed (collisions give the pairs m in C_j,
 * n in C_i): (S / 2^chunk_log2)^2 / 2 chunk sieves.  2 <= S <= 2^32 (keys
 * are exact 64-bit words), S < max_hi, 10 <= chunk_log2 <= 28, kinds 1..3.
 * The table and radical buffers are allocated for the call and freed after
 * it.  `out` is a HOST buffer; blocking.  Errors as bnx_search. */
int bnx_search_chunked(bnx_ctx *ctx, uint64_t S, uint32_t chunk_log2, uint32_t kinds, bnx_pair *out, size_t cap,
                       size_t *n_out);

/* Algorithm 2 (Sec. 2.1) on the device: all pairs with m < n < S by sorting.
 * The radicals of [1, S] are sieved, every n < S gets the exact key
 * {rad n, rad n+1} = max << 32 | min, relabelled by a bijective 64-bit mix h,
 * the (h, n) records are sorted by the top 32 bits of h (a stable 4-pass
 * least-significant-digit radix sort), and every run of equal prefixes gives
 * all its pairs m < n with equal h, i.e. equal 2-sets (not only neighbours, so
 * runs of three or more lose nothing), of the first kind when rad(m) = rad(n).
 * 3 <= S <= 2^32,
 * S < max_hi, kinds 1..3.  About 32 S bytes of device memory (radicals and two
 * key/value buffers) are allocated for the call and freed after it: 137 GB at
 * S = 2^32.  `out` is a HOST buffer; blocking.  Errors as bnx_search,
 * BNX_E_NOMEM when the buffers do not fit, and BNX_E_TIMEOUT if a tile of the
 * sort waited too long for the counts of the tiles before it (a bounded wait
 * that is not expected to run out). */
int bnx_search_sorted(bnx_ctx *ctx, uint64_t S, uint32_t kinds, bnx_pair *out, size_t cap, size_t *n_out);

/* Test hook for bnx_search_sorted's bounded wait: the next bnx_search_sorted
 * call on this context has the first sort tile of its first pass keep its
 * digit counts to itself, and every tile gives up waiting for them after
 * spin_limit polls (1 .. 2^22), so the call returns BNX_E_TIMEOUT with no pair
 * written (when the sort has at least two tiles, S > 7169).  The hook arms that one call only; the
 * call after it runs normally.  Every index the sort writes stays in bounds
 * and every wait ends; nothing here can stall the device.  Errors: BNX_E_ARG. */
int bnx_arm_lookback_timeout(bnx_ctx *ctx, uint32_t spin_limit);

/* Batched path: k intervals in one pipeline -- large-prime bucket fill, one
 * persistent sieve launch pulling segments from a device queue, verification
 * and a device sort -- replayed from a cached CUDA graph when the batch shape
 * repeats.  `iv`, `out` and `offsets` are HOST buffers.  On success out holds
 * the pairs sorted by (interval index, n, m, kind) with bnx_pair.iv set, and
 * offsets[i] .. offsets[i+1] delimit interval i's pairs (offsets has k+1
 * entries; may be NULL).  Errors as bnx_search. */
int bnx_batch(bnx_ctx *ctx, const bnx_interval *iv, size_t k, bnx_pair *out, size_t cap, size_t *n_out,
              uint64_t *offsets);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of interval requests                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t max_active;      /* requests on the device at once (slots, 1 .. 2^24) */
    uint32_t pad;
    uint64_t slice;           /* an iteration runs as many integers as an equal share eq
                                 of slice * max_active (at least slice per request)
                                 would: a request with at most eq left finishes, every
                                 other one gets slice, and the rest go to the oldest
                                 requests first (any value >= 1) */
    uint64_t mem_budget;      /* bytes of device workspace the loop may hold (0: 90% of
                                 the HBM free at start); the context's prime tables are
                                 not counted */
} bnx_server_cfg;

/* Counters of a serving loop (the current one, or the last after a stop). */
typedef struct {
    uint64_t submitted;      /* requests queued */
    uint64_t completed;      /* requests finished, successfully or not */
    uint64_t iterations;     /* batched pipeline runs */
    uint64_t deferred;       /* requests that waited for memory while a slot was free */
    uint64_t rejected;       /* requests whose first slice exceeds the budget even alone:
                                they finish at once with BNX_E_NOMEM */
    uint64_t budget_bytes;   /* the loop's workspace budget */
    uint64_t ws_peak_bytes;  /* largest workspace held after an iteration (<= budget_bytes) */
    uint64_t cancelled;      /* requests cancelled before they finished */
} bnx_server_stats;

/* Start the serving loop on a background host thread.  Each iteration
 *  - admits waiting requests in arrival order while a slot is free and an
 *    iteration giving every admitted request `slice` integers fits the budget
 *    (otherwise the request waits for memory);
 *  - takes the next slice of every active request (the requests that fit their
 *    equal share finish; the others get `slice`, and the rest of the iteration
 *    goes to the oldest first; the extra is cut, then the per-request slice down
 *    to one queue segment, until the iteration's workspace fits the budget) and
 *    runs all of them as one batched pipeline, the workspace sized under the
 *    budget.
 * So the budget bounds the device memory the loop holds.
 * Errors: BNX_E_ARG, BNX_E_STATE (already running), BNX_E_NOMEM, BNX_E_CUDA. */
int bnx_server_start(bnx_ctx *ctx, const bnx_server_cfg *cfg);

/* Counters of the serving loop (readable while it runs and after it stops). */
int bnx_server_get_stats(bnx_ctx *ctx, bnx_server_stats *out);

/* Device workspace, in bytes, that one batched run over these k intervals
 * needs (bnx_batch sizes its workspace to at least this; the serving loop's
 * admission uses the same figure).  `iv` is a HOST array.  Not while the
 * serving loop runs.  Errors: BNX_E_ARG, BNX_E_STATE. */
int bnx_workspace_bytes(bnx_ctx *ctx, const bnx_interval *iv, size_t k, uint64_t *bytes);

/* Queue a request; *ticket identifies it.  Never blocks on the device. */
int bnx_server_submit(bnx_ctx *ctx, const bnx_interval *iv, uint64_t *ticket);

/* Cancel a request.  One still waiting for a slot is dropped at once; one on the
 * device finishes the slice it is running and is retired at the end of that
 * iteration, its pairs discarded.  Either way it counts as completed and
 * cancelled, and bnx_server_poll then returns BNX_E_CANCELLED (and releases the
 * ticket).  A request that already finished is left as it is.  Never blocks on
 * the device.  Errors: BNX_E_ARG (unknown ticket), BNX_E_STATE (not serving). */
int bnx_server_cancel(bnx_ctx *ctx, uint64_t ticket);

/* BNX_E_BUSY while the request runs; BNX_OK once done, with its pairs copied to
 * the host buffer `out` (sorted by (n, m, kind)) and latency_s = completion time
 * minus submit time.  A finished request is released by the first successful
 * poll.  BNX_E_ARG for an unknown ticket. */
int bnx_server_poll(bnx_ctx *ctx, uint64_t ticket, bnx_pair *out, size_t cap, size_t *n_out, double *latency_s);

/* Stop the loop after the current iteration; unfinished requests are dropped. */
int bnx_server_stop(bnx_ctx *ctx);

/* ------------------------------------------------------------------------ */
/* Autotuning                                                                 */
/* ------------------------------------------------------------------------ */

/* Time candidate tunings (tile length, tiles per segment, threads, CTAs per SM,
 * shared-memory prime-power limit) on the batched path over `k` sample
 * intervals, keep the fastest in the context, and write it as JSON to
 * `json_out` (size `json_cap`, may be NULL).  Errors: BNX_E_ARG, BNX_E_CUDA. */
int bnx_autotune(bnx_ctx *ctx, const bnx_interval *iv, size_t k, int rounds, char *json_out, size_t json_cap);

/* ------------------------------------------------------------------------ */
/* Errors                                                                      */
/* ------------------------------------------------------------------------ */

const char *bnx_strerror(int code);
const char *bnx_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* BENELUX_H */
