// Host side of libbenelux: contexts, device tables, workspace, the pipeline
// (captured once as a CUDA graph and replayed), and the C ABI entry points
// declared in include/benelux.h.
#include <algorithm>
#include <unistd.h>
#include <cerrno>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "benelux.h"
#include "bnx_ctx.cuh"

namespace bnx {

thread_local std::string g_last_error;

int fail(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

int grow(DevBuf &b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return BNX_OK;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
    if (cudaMalloc(&b.p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(BNX_E_NOMEM, "cudaMalloc of %zu bytes failed", bytes);
    }
    b.bytes = bytes;
    return BNX_OK;
}

void release(DevBuf &b) {
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
}

static uint64_t isqrt64(uint64_t x) {
    uint64_t r = (uint64_t)std::sqrt((double)x);
    while (r * r > x) r--;
    while ((r + 1) * (r + 1) <= x) r++;
    return r;
}

// ----------------------------------------------------------------- tune ----
static void tune_defaults(bnx_tune *t) {
    t->tile_log2 = 15;
    t->seg_tiles = 16;
    t->threads = 256;
    t->ctas_per_sm = 0;
    t->small_q_log2 = 16;
    t->tile_kind = kTileLog8;
}

static int tune_check(const bnx_tune *t) {
    if (t->tile_log2 < 10 || t->tile_log2 > 16) return fail(BNX_E_ARG, "tile_log2 must be in [10, 16]");
    if (t->seg_tiles < 1 || t->seg_tiles > 64 || (t->seg_tiles & (t->seg_tiles - 1)))
        return fail(BNX_E_ARG, "seg_tiles must be a power of two in [1, 64]");
    if (t->threads != 128 && t->threads != 256 && t->threads != 512 && t->threads != 1024)
        return fail(BNX_E_ARG, "threads must be 128, 256, 512 or 1024");
    if (t->small_q_log2 < 8 || t->small_q_log2 > 16) return fail(BNX_E_ARG, "small_q_log2 must be in [8, 16]");
    if (t->tile_kind > 3) return fail(BNX_E_ARG, "tile_kind must be 0, 1, 2 or 3");
    if (t->ctas_per_sm > 32) return fail(BNX_E_ARG, "ctas_per_sm must be <= 32");
    return BNX_OK;
}

// Reader for a flat JSON object whose values are non-negative integers: the
// bnx_tune field names, plus "ms" (a number, ignored), which bnx_autotune writes
// beside them.  Unknown or repeated keys, values that are not integers or do not
// fit 32 bits, and anything after the closing brace are errors; fields that are
// absent keep their value in *t.
static int parse_tune_json(const char *s, bnx_tune *t) {
    struct F {
        const char *name;
        uint32_t *dst;
    } fields[] = {{"tile_log2", &t->tile_log2},
                  {"seg_tiles", &t->seg_tiles},
                  {"threads", &t->threads},
                  {"ctas_per_sm", &t->ctas_per_sm},
                  {"small_q_log2", &t->small_q_log2},
                  {"tile_kind", &t->tile_kind},
                  {"ms", nullptr}};
    constexpr int nf = sizeof fields / sizeof fields[0];
    bool seen[nf] = {};
    auto ws = [](const char *&p) {
        while (*p == ' ' || *p == '\t' || *p == '\n' || *p == '\r') p++;
    };
    const char *p = s;
    ws(p);
    if (*p++ != '{') return fail(BNX_E_ARG, "tune JSON: expected '{'");
    ws(p);
    if (*p == '}') {
        p++;
    } else {
        for (;;) {
            ws(p);
            if (*p++ != '"') return fail(BNX_E_ARG, "tune JSON: expected a quoted key");
            const char *k0 = p;
            while (*p && *p != '"') p++;
            if (*p != '"') return fail(BNX_E_ARG, "tune JSON: unterminated key");
            const std::string key(k0, (size_t)(p - k0));
            p++;
            int f = -1;
            for (int i = 0; i < nf; i++)
                if (key == fields[i].name) f = i;
            if (f < 0) return fail(BNX_E_ARG, "tune JSON: unknown field \"%s\"", key.c_str());
            if (seen[f]) return fail(BNX_E_ARG, "tune JSON: field \"%s\" given twice", key.c_str());
            seen[f] = true;
            ws(p);
            if (*p++ != ':') return fail(BNX_E_ARG, "tune JSON: expected ':' after \"%s\"", key.c_str());
            ws(p);
            if (*p < '0' || *p > '9') return fail(BNX_E_ARG, "tune JSON: %s is not a non-negative number", key.c_str());
            uint64_t v = 0;
            while (*p >= '0' && *p <= '9') {
                v = v * 10 + (uint64_t)(*p++ - '0');
                if (v > 0xffffffffull) return fail(BNX_E_ARG, "tune JSON: %s does not fit 32 bits", key.c_str());
            }
            if (fields[f].dst) {
                if (*p == '.' || *p == 'e' || *p == 'E')
                    return fail(BNX_E_ARG, "tune JSON: %s is not an integer", key.c_str());
                *fields[f].dst = (uint32_t)v;
            } else {  // "ms": the fraction and exponent of a JSON number
                if (*p == '.') {
                    p++;
                    while (*p >= '0' && *p <= '9') p++;
                }
                if (*p == 'e' || *p == 'E') {
                    p++;
                    if (*p == '+' || *p == '-') p++;
                    while (*p >= '0' && *p <= '9') p++;
                }
            }
            ws(p);
            if (*p == ',') {
                p++;
                continue;
            }
            if (*p == '}') {
                p++;
                break;
            }
            return fail(BNX_E_ARG, "tune JSON: expected ',' or '}' after \"%s\"", key.c_str());
        }
    }
    ws(p);
    if (*p) return fail(BNX_E_ARG, "tune JSON: text after the closing brace");
    return tune_check(t);
}

// ---------------------------------------------------------- tables --------
int build_pp_tables(bnx_ctx *c) {
    const uint32_t q_small = 1u << c->tune.small_q_log2;
    uint64_t lpp_cap = 2;
    while (lpp_cap < (uint64_t)c->np + 65536) lpp_cap <<= 1;  // a power of two: the table is bitonic-sorted
    int rc;
    if ((rc = grow(c->spp, sizeof(SmallPP) * kMaxSpp))) return rc;
    if ((rc = grow(c->lpp, sizeof(LargePP) * lpp_cap))) return rc;
    if ((rc = grow(c->tmp_counts, sizeof(uint32_t) * (4 + 4 * ((size_t)c->np + 1))))) return rc;
    uint32_t *cnt = (uint32_t *)c->tmp_counts.p;
    launch_build_pp((uint32_t *)c->primes.p, c->np, c->max_hi, q_small, (SmallPP *)c->spp.p, cnt,
                    (LargePP *)c->lpp.p, cnt + 1, lpp_cap, cnt + 4, c->stream);
    CUDA_TRY(cudaGetLastError());
    uint32_t h[2];
    CUDA_TRY(cudaMemcpyAsync(h, cnt, sizeof h, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if (h[0] > (uint32_t)kMaxSpp)
        return fail(BNX_E_ARG, "%u in-tile prime powers exceed the limit %d: lower small_q_log2", h[0], kMaxSpp);
    if (h[1] > lpp_cap) return fail(BNX_E_NOMEM, "large prime-power table overflow");
    c->n_spp = h[0];
    c->n_lpp = h[1];
    {
        uint32_t n2 = 2;
        while (n2 < c->n_lpp) n2 <<= 1;
        launch_sort_lpp((LargePP *)c->lpp.p, c->n_lpp, n2, c->stream);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaStreamSynchronize(c->stream));  // the copies below run on the default stream
    }
    std::vector<SmallPP> hs(c->n_spp);
    if (c->n_spp) CUDA_TRY(cudaMemcpy(hs.data(), c->spp.p, sizeof(SmallPP) * c->n_spp, cudaMemcpyDeviceToHost));
    c->h_spp_q.resize(c->n_spp);
    for (uint32_t i = 0; i < c->n_spp; i++) c->h_spp_q[i] = hs[i].q;
    // host copy of the large q values, sorted, for the bucket capacity bound
    std::vector<LargePP> tmp(c->n_lpp);
    if (c->n_lpp)
        CUDA_TRY(cudaMemcpy(tmp.data(), c->lpp.p, sizeof(LargePP) * c->n_lpp, cudaMemcpyDeviceToHost));
    c->lq.resize(c->n_lpp);
    for (uint32_t i = 0; i < c->n_lpp; i++) c->lq[i] = tmp[i].q;
    std::sort(c->lq.begin(), c->lq.end());
    c->lq_inv.assign(c->n_lpp + 1, 0.0);
    for (uint32_t i = 0; i < c->n_lpp; i++) c->lq_inv[i + 1] = c->lq_inv[i] + 1.0 / (double)c->lq[i];
    return BNX_OK;
}

static int build_tables(bnx_ctx *c) {
    const uint64_t lim = std::max<uint64_t>(isqrt64(c->max_hi), 16);
    DevBuf comp;
    int rc;
    if ((rc = grow(comp, lim + 1))) return rc;
    CUDA_TRY(cudaMemsetAsync(comp.p, 0, lim + 1, c->stream));
    launch_prime_sieve((uint8_t *)comp.p, lim, c->stream);
    const uint32_t nb = flags_blocks(lim + 1);
    DevBuf sums;
    if ((rc = grow(sums, sizeof(uint32_t) * (nb + 1)))) {
        release(comp);
        return rc;
    }
    launch_scan_u8_count((uint8_t *)comp.p, lim + 1, (uint32_t *)sums.p, nb, c->stream);
    uint32_t np = 0;
    CUDA_TRY(cudaMemcpyAsync(&np, (uint32_t *)sums.p + nb, sizeof np, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    if ((rc = grow(c->primes, sizeof(uint32_t) * (np + 1)))) {
        release(comp);
        release(sums);
        return rc;
    }
    launch_compact_primes((uint8_t *)comp.p, lim, (uint32_t *)sums.p, (uint32_t *)c->primes.p, nb, c->stream);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(c->stream));
    release(comp);
    release(sums);
    c->np = np;
    return build_pp_tables(c);
}

// ------------------------------------------------------------ planning ----
uint64_t bucket_bound(const bnx_ctx *c, uint64_t lo, uint64_t hi, uint64_t nseg) {
    // hits of the large prime powers q <= hi among the W = hi - lo + 1 sieved
    // values: sum floor(W/q) + 1 over q <= hi, plus the re-listing of a boundary
    // value as the previous segment's halo (at most log_3(hi) < 28 prime powers
    // divide it)
    const uint64_t W = hi - lo + 1;
    const size_t nq = std::upper_bound(c->lq.begin(), c->lq.end(), hi) - c->lq.begin();
    const double h = c->lq_inv[nq];
    return (uint64_t)std::ceil((double)W * h * (1.0 + 1e-9)) + nq + 28 * nseg + 16;
}

int plan_host(bnx_ctx *c, const IvDev *iv, size_t k, PlanTotals *t) {
    const uint32_t seg_log2 = c->seg_log2(), chunk_log2 = c->chunk_log2();
    t->segs = t->chunks = t->buckets = t->integers = 0;
    for (size_t i = 0; i < k; i++) {
        const uint64_t len = iv[i].hi - iv[i].lo;
        const uint64_t ns = (len + (1ull << seg_log2) - 1) >> seg_log2;
        t->segs += ns;
        t->chunks += (len + 1 + (1ull << chunk_log2) - 1) >> chunk_log2;
        t->buckets += bucket_bound(c, iv[i].lo, iv[i].hi, ns);
        t->integers += len;
    }
    return BNX_OK;
}

// The workspace buffers of one pipeline run and the bytes each needs for a run
// with plan totals t over k intervals.
static int ws_needs(bnx_ctx *c, const PlanTotals &t, size_t k, DevBuf **buf, size_t *bytes) {
    int n = 0;
    auto add = [&](DevBuf &b, size_t v) {
        buf[n] = &b;
        bytes[n++] = v;
    };
    add(c->ivs, sizeof(IvDev) * (k + 1));
    add(c->offsets, sizeof(uint64_t) * (k + 2));
    add(c->bcnt, sizeof(uint32_t) * (t.segs + 1));
    add(c->seg_iv, sizeof(uint32_t) * (t.segs + 1));
    add(c->boff, sizeof(unsigned long long) * (t.segs + 2));
    add(c->scan_tmp, sizeof(unsigned long long) * (t.segs / 4096 + 2));
    add(c->bent, sizeof(uint2) * (t.buckets + 1));
    add(c->cand, sizeof(Cand) * c->cand_want);
    add(c->surv, sizeof(Survivor) * c->surv_want);
    add(c->pairs, sizeof(PairDev) * c->pair_want);
    add(c->pairs_sorted, sizeof(PairDev) * c->pair_want);
    return n;
}
constexpr int kWsBufs = 11;

uint64_t ws_need_bytes(bnx_ctx *c, const PlanTotals &t, size_t k) {
    DevBuf *b[kWsBufs];
    size_t v[kWsBufs];
    const int n = ws_needs(c, t, k, b, v);
    uint64_t sum = 0;
    for (int i = 0; i < n; i++) sum += v[i];
    return sum;
}

uint64_t ws_footprint(bnx_ctx *c) {
    const PlanTotals t0{0, 0, 0, 0};
    DevBuf *b[kWsBufs];
    size_t v[kWsBufs];
    const int n = ws_needs(c, t0, 0, b, v);
    uint64_t sum = 0;
    for (int i = 0; i < n; i++) sum += b[i]->bytes;
    return sum;
}

// Grow the workspace to fit a run.  A grown buffer gets a quarter more than it
// needs, so that batches that grow slowly do not reallocate every time.  With a
// budget (bytes, 0 = none) the workspace never exceeds it: when the usual growth
// would, every buffer is sized to exactly what the run needs (larger leftovers
// of earlier runs are freed first), and a run that needs more than the budget
// fails with BNX_E_NOMEM before anything is allocated.
int ensure_ws(bnx_ctx *c, const PlanTotals &t, size_t k, uint64_t budget) {
    DevBuf *b[kWsBufs];
    size_t v[kWsBufs];
    const int n = ws_needs(c, t, k, b, v);
    uint64_t grown = 0, exact = 0;
    for (int i = 0; i < n; i++) {
        grown += b[i]->bytes >= v[i] ? b[i]->bytes : v[i] + v[i] / 4;
        exact += v[i];
    }
    const bool tight = budget && grown > budget;
    if (tight && exact > budget)
        return fail(BNX_E_NOMEM, "the run needs %llu bytes of workspace, the budget is %llu",
                    (unsigned long long)exact, (unsigned long long)budget);
    bool changed = false;
    int rc;
    for (int i = 0; i < n; i++)
        if (tight && b[i]->bytes > v[i]) {
            release(*b[i]);
            changed = true;
        }
    for (int i = 0; i < n; i++) {
        if (b[i]->bytes >= v[i]) continue;
        changed = true;
        if ((rc = grow(*b[i], tight ? v[i] : v[i] + v[i] / 4))) return rc;
    }
    if (changed) c->invalidate_graphs();
    return ensure_staging(c, k);
}

// Pinned host staging for the intervals of a run of k intervals.
int ensure_staging(bnx_ctx *c, size_t k) {
    if (k + 1 <= c->h_ivs_cap) return BNX_OK;
    if (c->h_ivs) cudaFreeHost(c->h_ivs);
    c->h_ivs = nullptr;
    c->h_ivs_cap = 0;
    if (cudaMallocHost(&c->h_ivs, sizeof(IvDev) * (k + 1) * 2) != cudaSuccess) {
        cudaGetLastError();
        return fail(BNX_E_NOMEM, "pinned host allocation failed");
    }
    c->h_ivs_cap = (k + 1) * 2;
    return BNX_OK;
}

Plan make_plan(const bnx_ctx *c) {
    Plan P;
    memset(&P, 0, sizeof P);
    P.ivs = (const IvDev *)c->ivs.p;
    P.n_iv = (const uint32_t *)c->n_iv.p;
    P.spp = (const SmallPP *)c->spp.p;
    P.n_spp = c->n_spp;
    P.n_sched = c->n_sched();
    {
        uint32_t r = 1u << (c->tune.small_q_log2 / 2);
        while ((uint64_t)(r + 1) * (r + 1) <= (1ull << c->tune.small_q_log2)) r++;
        P.sqrt_q = r;
    }
    P.lpp = (const LargePP *)c->lpp.p;
    P.n_lpp = c->n_lpp;
    P.tile_log2 = c->tune.tile_log2;
    P.seg_log2 = c->seg_log2();
    P.chunk_log2 = c->chunk_log2();
    {
        // walked by a whole warp: prime powers with at least 32 multiples per chunk (one
        // full warp round), up to 2^20 (above that one thread per q measured faster)
        const uint64_t qd = std::min<uint64_t>(1ull << (P.chunk_log2 - 5), 1ull << 20);
        P.n_lpp_dense = (uint32_t)(std::upper_bound(c->lq.begin(), c->lq.end(), qd) - c->lq.begin());
    }
    P.bcnt = (uint32_t *)c->bcnt.p;
    P.seg_iv = (uint32_t *)c->seg_iv.p;
    P.boff = (unsigned long long *)c->boff.p;
    P.bent = (uint2 *)c->bent.p;
    {
        const uint64_t a = std::min(c->bcnt.bytes, c->seg_iv.bytes) / sizeof(uint32_t),
                       b = c->boff.bytes / sizeof(unsigned long long);
        P.seg_cap = std::min(a > 0 ? a - 1 : 0, b > 1 ? b - 2 : 0);
    }
    P.bucket_cap = c->bent.bytes / sizeof(uint2);
    P.ctr = (Counters *)c->ctr.p;
    P.surv = (Survivor *)c->surv.p;
    P.surv_cap = c->surv.bytes / sizeof(Survivor);
    P.cand = (Cand *)c->cand.p;
    P.cand_cap = c->cand.bytes / sizeof(Cand);
    P.pairs = (PairDev *)c->pairs.p;
    P.pairs_sorted = (PairDev *)c->pairs_sorted.p;
    P.pair_cap = c->pairs.bytes / sizeof(PairDev);
    P.iv_offsets = (uint64_t *)c->offsets.p;
    P.rad_out = c->rad_out;
    P.sq_out = c->sq_out;
    P.rad_lo = c->rad_lo;
    P.rad_len = c->rad_len;
    P.hash_S = c->hash_S;
    P.hkeys = (unsigned long long *)c->hkeys.p;
    P.hheads = (uint32_t *)c->hheads.p;
    P.hnext = (uint32_t *)c->hnext.p;
    P.hslot = (uint32_t *)c->hslot.p;
    P.hash_mask = c->hash_mask;
    return P;
}

// Launch shape of the persistent sieve for the current tuning (queried outside
// any stream capture and cached until the tuning changes).
static bool use_log_tile(const bnx_ctx *c, int mode) { return mode != kModeRad && c->tune.tile_kind != kTileExact; }

// The exact u64 tile (searches) and the u32 radical tile fit shared memory up to
// 2^14 values; a longer tuned tile is processed as several tiles of the same
// queue segment.
static uint32_t tile_log2_for(const bnx_ctx *c, int mode) {
    return use_log_tile(c, mode) ? c->tune.tile_log2 : std::min<uint32_t>(c->tune.tile_log2, 14u);
}
// bytes per value of the log-domain tile
static int log_vb(const bnx_ctx *c) {
    return c->tune.tile_kind == kTileLog8 ? 1 : c->tune.tile_kind == kTileLog16 ? 2 : 4;
}

int sieve_config(bnx_ctx *c, int mode, int *grid, int *threads, size_t *smem) {
    const bool lg = use_log_tile(c, mode);
    const int vb = lg ? log_vb(c) : 8;
    SieveCfg &sc = c->sieve_cfg[mode * 4 + (lg ? (vb == 4 ? 1 : vb == 2 ? 2 : 3) : 0)];
    const uint32_t tlog = tile_log2_for(c, mode);
    const uint32_t nsched = sched_length(tlog, c->h_spp_q.data(), c->n_spp);
    const size_t want_smem = lg                ? sieve_log_smem_bytes(tlog, c->n_spp, nsched, vb)
                             : mode == kModeRad ? rad_smem_bytes(tlog, c->n_spp, nsched)
                                                : sieve_smem_bytes(tlog, c->n_spp, nsched);
    if (!sc.valid || sc.tile_log2 != tlog || sc.threads != c->tune.threads ||
        sc.ctas != c->tune.ctas_per_sm || sc.smem != want_smem) {
        if (c->capturing) return fail(BNX_E_STATE, "sieve launch shape unknown during capture");
        const int thr = (int)c->tune.threads;
        const size_t smem_b = want_smem;
        int occ = 0;
        int e = lg                ? sieve_log_occupancy(mode, thr, vb, smem_b, &occ)
                : mode == kModeRad ? rad_occupancy(thr, smem_b, &occ)
                                   : sieve_occupancy(mode, thr, smem_b, &occ);
        if (e != 0) return fail(BNX_E_CUDA, "sieve occupancy query failed: %s", cudaGetErrorString((cudaError_t)e));
        if (occ < 1) return fail(BNX_E_ARG, "sieve kernel does not fit an SM with this tuning");
        const int per = c->tune.ctas_per_sm ? std::min<int>((int)c->tune.ctas_per_sm, occ) : occ;
        sc.grid = c->n_sm * per;
        sc.threads = c->tune.threads;
        sc.smem = smem_b;
        sc.tile_log2 = tlog;
        sc.ctas = c->tune.ctas_per_sm;
        sc.occ = occ;
        sc.valid = true;
    }
    *grid = sc.grid;
    *threads = (int)sc.threads;
    *smem = sc.smem;
    return BNX_OK;
}

// Launch the whole pipeline on stream s (directly or under capture).
int record_pipeline(bnx_ctx *c, int mode, cudaStream_t s, bool timing) {
    Plan P = make_plan(c);
    P.tile_log2 = tile_log2_for(c, mode);
    P.n_sched = sched_length(P.tile_log2, c->h_spp_q.data(), c->n_spp);
    int sgrid, sthreads;
    size_t ssmem;
    int rc = sieve_config(c, mode, &sgrid, &sthreads, &ssmem);
    if (rc) return rc;
    const int bgrid = c->n_sm * 8;
    CUDA_TRY(cudaMemsetAsync(c->ctr.p, 0, sizeof(Counters), s));
    launch_plan(P, (uint32_t *)c->n_iv.p, (IvDev *)c->ivs.p, 0, s);
    CUDA_TRY(cudaMemsetAsync(c->bcnt.p, 0, c->bcnt.bytes, s));
    launch_bucket(P, false, bgrid, s);
    launch_exclusive_scan_u32(P.bcnt, P.boff, &P.ctr->total_segs, P.seg_cap, (unsigned long long *)c->scan_tmp.p,
                              (uint32_t)(c->scan_tmp.bytes / 8), s);
    CUDA_TRY(cudaMemsetAsync(c->bcnt.p, 0, c->bcnt.bytes, s));
    launch_bucket(P, true, bgrid, s);
    if (timing) CUDA_TRY(cudaEventRecordWithFlags(c->ev_s0, s, c->capturing ? cudaEventRecordExternal : 0));
    if (use_log_tile(c, mode)) launch_sieve_log(P, mode, log_vb(c), sgrid, sthreads, ssmem, s);
    else if (mode == kModeRad) launch_rad(P, sgrid, sthreads, ssmem, s);
    else launch_sieve(P, mode, sgrid, sthreads, ssmem, s);
    if (timing) CUDA_TRY(cudaEventRecordWithFlags(c->ev_s1, s, c->capturing ? cudaEventRecordExternal : 0));
    if (use_log_tile(c, mode)) launch_cand(P, mode, c->n_sm * 2, s);
    if (mode == kModeSearch) {
        launch_verify(P, c->n_sm * 4, s);
        launch_sort(P, c->n_sm * 2, s);
        launch_offsets(P, c->n_sm, s);
    }
    if (mode != kModeRad)
        CUDA_TRY(cudaMemcpyAsync(c->h_ctr, c->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaGetLastError());
    return BNX_OK;
}

// Run the search pipeline for the intervals already in c->h_ivs[0..k), waiting
// for completion; the counters land in c->h_ctr.
int run_search(bnx_ctx *c, size_t k, bool use_graph) {
    cudaStream_t s = c->stream;
    CUDA_TRY(cudaMemcpyAsync(c->ivs.p, c->h_ivs, sizeof(IvDev) * k, cudaMemcpyHostToDevice, s));
    c->h_nk = (uint32_t)k;
    CUDA_TRY(cudaMemcpyAsync(c->n_iv.p, &c->h_nk, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaEventRecord(c->ev0, s));
    if (use_graph) {
        const uint32_t slot = c->seg_log2() - c->tune.tile_log2;  // < kGraphSlots: segments hold 1 .. 64 tiles
        cudaGraphExec_t &gexec = c->gexec[slot];
        if (!c->graph_ok[slot]) {
            if (gexec) cudaGraphExecDestroy(gexec);
            gexec = nullptr;
            cudaGraph_t g;
            int sg, st;
            size_t ss;
            int rc0 = sieve_config(c, kModeSearch, &sg, &st, &ss);
            if (rc0) return rc0;
            CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            c->capturing = true;
            int rc = record_pipeline(c, kModeSearch, s, true);
            c->capturing = false;
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (rc) {
                if (e == cudaSuccess) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return fail(BNX_E_CUDA, "graph capture failed: %s", cudaGetErrorString(e));
            e = cudaGraphInstantiate(&gexec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return fail(BNX_E_CUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
            c->graph_ok[slot] = true;
        }
        CUDA_TRY(cudaGraphLaunch(gexec, s));
    } else {
        int rc = record_pipeline(c, kModeSearch, s, true);
        if (rc) return rc;
    }
    CUDA_TRY(cudaEventRecord(c->ev1, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    return BNX_OK;
}

// Check the counters of a finished search; grow and ask for a rerun when a
// device-side capacity was exceeded.  Returns BNX_OK, or BNX_E_OVERFLOW with
// *rerun set when the run should be repeated.
int check_counters(bnx_ctx *c, bool *rerun) {
    *rerun = false;
    const Counters &h = *c->h_ctr;
    if (h.err & (kErrSurvOverflow | kErrPairOverflow | kErrCandOverflow)) {
        if (h.n_surv > c->surv.bytes / sizeof(Survivor)) c->surv_want = (size_t)(h.n_surv + h.n_surv / 2 + 1024);
        if (h.n_cand > c->cand.bytes / sizeof(Cand)) c->cand_want = (size_t)(h.n_cand + h.n_cand / 2 + 1024);
        if (h.n_pairs > c->pairs.bytes / sizeof(PairDev)) c->pair_want = (size_t)(h.n_pairs + h.n_pairs / 2 + 1024);
        *rerun = true;
        return BNX_E_OVERFLOW;
    }
    if (h.err & kErrBounds) return fail(BNX_E_OVERFLOW, "a device index fell outside its buffer (flags 0x%x)", h.err);
    if (h.err) return fail(BNX_E_OVERFLOW, "device capacity exceeded (flags 0x%x)", h.err);
    return BNX_OK;
}

void fill_stats(bnx_ctx *c, uint64_t integers) {
    const Counters &h = *c->h_ctr;
    bnx_stats &st = c->stats;
    memset(&st, 0, sizeof st);
    st.integers = integers;
    st.segments = h.total_segs;
    st.bucket_hits = h.bucket_hits;
    st.survivors1 = h.surv1;
    st.survivors2 = h.surv2;
    st.candidates = h.candidates;
    st.pairs = h.n_pairs;
    st.hash_keys = h.hash_keys;
    float ms = 0;
    if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) st.ms_total = ms;
    if (cudaEventElapsedTime(&ms, c->ev_s0, c->ev_s1) == cudaSuccess) st.ms_sieve = ms;
    cudaGetLastError();
    st.sieve_launches = 1;
}

int validate_interval(const bnx_ctx *c, uint64_t lo, uint64_t hi, uint32_t kinds) {
    if (lo < 1 || hi <= lo) return fail(BNX_E_ARG, "need 1 <= lo < hi (lo=%llu hi=%llu)", (unsigned long long)lo,
                                        (unsigned long long)hi);
    if (hi > c->max_hi) return fail(BNX_E_ARG, "hi=%llu exceeds max_hi=%llu", (unsigned long long)hi,
                                    (unsigned long long)c->max_hi);
    if (kinds < 1 || kinds > 7) return fail(BNX_E_ARG, "kinds must be a mask of 1, 2 and 4");
    return BNX_OK;
}

// Search the intervals staged in c->h_ivs[0..k), retrying on capacity
// overflow; copies the sorted pairs (and per-interval offsets) to the host.
int search_staged(bnx_ctx *c, size_t k, bnx_pair *out, size_t cap, size_t *n_out, uint64_t *offsets,
                  uint64_t budget) {
    NvtxRange r_all("bnx.search");
    PlanTotals t;
    {
        NvtxRange r("bnx.plan");
        plan_host(c, c->h_ivs, k, &t);
    }
    for (int attempt = 0; attempt < 4; attempt++) {
        int rc;
        {
            NvtxRange r("bnx.workspace");
            rc = ensure_ws(c, t, k, budget);
        }
        if (rc) return rc;
        {
            NvtxRange r("bnx.pipeline");  // graph launch (or capture) and the wait for it
            rc = run_search(c, k, true);
        }
        if (rc) return rc;
        bool rerun = false;
        rc = check_counters(c, &rerun);
        if (rerun) continue;
        if (rc) return rc;
        fill_stats(c, t.integers);
        NvtxRange r_out("bnx.copy_out");
        const size_t np = (size_t)c->h_ctr->n_pairs;
        if (n_out) *n_out = np;
        const size_t ncopy = std::min(np, cap);
        if (ncopy) {
            if (!out) return fail(BNX_E_ARG, "out is NULL");
            CUDA_TRY(cudaMemcpy(out, c->pairs_sorted.p, sizeof(PairDev) * ncopy, cudaMemcpyDeviceToHost));
        }
        if (offsets) CUDA_TRY(cudaMemcpy(offsets, c->offsets.p, sizeof(uint64_t) * (k + 1), cudaMemcpyDeviceToHost));
        if (np > cap) return fail(BNX_E_TRUNCATED, "%zu pairs, buffer holds %zu", np, cap);
        return BNX_OK;
    }
    return fail(BNX_E_OVERFLOW, "device capacities kept overflowing");
}

}  // namespace bnx

using namespace bnx;

// ======================================================================== ABI

extern "C" {

const char *bnx_strerror(int code) {
    switch (code) {
        case BNX_OK: return "ok";
        case BNX_E_ARG: return "invalid argument";
        case BNX_E_TRUNCATED: return "output truncated";
        case BNX_E_NOMEM: return "out of memory";
        case BNX_E_CUDA: return "CUDA error";
        case BNX_E_TIMEOUT: return "timeout";
        case BNX_E_BUSY: return "busy";
        case BNX_E_STATE: return "invalid state";
        case BNX_E_OVERFLOW: return "device capacity exceeded";
        case BNX_E_CANCELLED: return "cancelled";
        default: return "unknown error";
    }
}

const char *bnx_last_error(void) { return g_last_error.c_str(); }

int bnx_tune_parse(const char *json, bnx_tune *out) {
    if (!json || !out) return fail(BNX_E_ARG, "NULL argument");
    bnx_tune t;
    tune_defaults(&t);
    const int rc = parse_tune_json(json, &t);
    if (rc == BNX_OK) *out = t;
    return rc;
}

static int bnx_create_impl(bnx_ctx **out, int device, uint64_t max_hi, const char *tune_json, void *stream) {
    if (!out) return fail(BNX_E_ARG, "out is NULL");
    *out = nullptr;
    if (max_hi < 4 || max_hi > BNX_MAX_HI) return fail(BNX_E_ARG, "max_hi must be in [4, 2^42]");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return fail(BNX_E_ARG, "no CUDA device %d", device);
    }
    bnx_ctx *c = new (std::nothrow) bnx_ctx();
    if (!c) return fail(BNX_E_NOMEM, "host allocation failed");
    c->device = device;
    c->max_hi = max_hi;
    tune_defaults(&c->tune);
    int rc = BNX_OK;
    if (tune_json && (rc = parse_tune_json(tune_json, &c->tune))) {
        delete c;
        return rc;
    }
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return fail(BNX_E_CUDA, "cudaSetDevice(%d) failed", device);
    }
    cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, device);
    if (stream) {
        c->stream = (cudaStream_t)stream;
        c->own_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete c;
            return fail(BNX_E_CUDA, "cudaStreamCreate failed");
        }
        c->own_stream = true;
    }
    if (cudaEventCreate(&c->ev0) || cudaEventCreate(&c->ev1) || cudaEventCreate(&c->ev_s0) ||
        cudaEventCreate(&c->ev_s1) || cudaMallocHost(&c->h_ctr, sizeof(Counters))) {
        cudaGetLastError();
        bnx_destroy(c);
        return fail(BNX_E_CUDA, "event or pinned allocation failed");
    }
    if ((rc = grow(c->ctr, sizeof(Counters))) || (rc = grow(c->n_iv, 16)) || (rc = build_tables(c))) {
        bnx_destroy(c);
        return rc;
    }
    *out = c;
    return BNX_OK;
}

int bnx_create(bnx_ctx **out, int device, uint64_t max_hi, const char *tune_json, void *stream) {
    return guarded([&] { return bnx_create_impl(out, device, max_hi, tune_json, stream); });
}

void bnx_destroy(bnx_ctx *c) {
    if (!c) return;
    bnx_server_stop(c);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (cudaGraphExec_t g : c->gexec)
        if (g) cudaGraphExecDestroy(g);
    for (DevBuf *b : c->all_bufs()) release(*b);
    if (c->h_ctr) cudaFreeHost(c->h_ctr);
    if (c->h_ivs) cudaFreeHost(c->h_ivs);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->ev_s0) cudaEventDestroy(c->ev_s0);
    if (c->ev_s1) cudaEventDestroy(c->ev_s1);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    cudaGetLastError();
    delete c;
}

int bnx_get_tune(const bnx_ctx *c, bnx_tune *out) {
    if (!c || !out) return fail(BNX_E_ARG, "NULL argument");
    *out = c->tune;
    return BNX_OK;
}

int bnx_set_tune(bnx_ctx *c, const bnx_tune *t) {
    if (!c || !t) return fail(BNX_E_ARG, "NULL argument");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    int rc = tune_check(t);
    if (rc) return rc;
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    const bool q_changed = t->small_q_log2 != c->tune.small_q_log2;
    const bnx_tune old = c->tune;
    c->tune = *t;
    if (q_changed && (rc = build_pp_tables(c))) {
        c->tune = old;
        build_pp_tables(c);
        return rc;
    }
    c->invalidate_graphs();
    return BNX_OK;
}

int bnx_get_stats(const bnx_ctx *c, bnx_stats *out) {
    if (!c || !out) return fail(BNX_E_ARG, "NULL argument");
    *out = c->stats;
    return BNX_OK;
}

int bnx_prime_count(const bnx_ctx *c, uint64_t *out) {
    if (!c || !out) return fail(BNX_E_ARG, "NULL argument");
    *out = c->np;
    return BNX_OK;
}

// Whether a caller's buffer is host memory that the kernels cannot write (pageable,
// or pinned: both are staged through device memory and copied).
static int host_buffer(const void *p, bool *host) {
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BNX_E_CUDA, "cudaPointerGetAttributes: %s", cudaGetErrorString(e));
    }
    *host = a.type == cudaMemoryTypeHost || a.type == cudaMemoryTypeUnregistered;
    return BNX_OK;
}

int bnx_rad_segment(bnx_ctx *c, uint64_t lo, uint64_t len, uint64_t *rad_out, uint64_t *sq_out, void *stream) {
    if (!c || !rad_out) return fail(BNX_E_ARG, "NULL argument");
    // (lo > max_hi - len, not lo + len > max_hi: the sum could wrap)
    if (lo < 1 || len < 1 || len > (1ull << 31) || len > c->max_hi || lo > c->max_hi - len)
        return fail(BNX_E_ARG, "need 1 <= lo, 1 <= len <= 2^31, lo + len <= max_hi");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    cudaStream_t s = stream ? (cudaStream_t)stream : c->stream;
    bool host = false, host_sq = false;
    int rc = host_buffer(rad_out, &host);
    if (rc == BNX_OK && sq_out) rc = host_buffer(sq_out, &host_sq);
    if (rc) return rc;
    if (sq_out && host != host_sq) return fail(BNX_E_ARG, "rad_out and sq_out must both be host or both device buffers");
    if (!host) return rad_segment_unlocked(c, lo, len, rad_out, sq_out, s);
    // host buffers: sieve into device staging, copy back, and wait
    const size_t bytes = sizeof(uint64_t) * len;
    if ((rc = grow(c->rad_stage, sq_out ? 2 * bytes : bytes))) return rc;
    uint64_t *d_rad = (uint64_t *)c->rad_stage.p, *d_sq = sq_out ? d_rad + len : nullptr;
    rc = rad_segment_unlocked(c, lo, len, d_rad, d_sq, s);
    if (rc == BNX_OK) {
        cudaError_t e = cudaMemcpyAsync(rad_out, d_rad, bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess && sq_out) e = cudaMemcpyAsync(sq_out, d_sq, bytes, cudaMemcpyDeviceToHost, s);
        // the run's error flags (a blocking call can report them)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(&c->h_ctr->err, &static_cast<Counters *>(c->ctr.p)->err, sizeof(c->h_ctr->err),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) {
            cudaGetLastError();
            rc = fail(BNX_E_CUDA, "copy of the radicals to the host: %s", cudaGetErrorString(e));
        } else if (c->h_ctr->err) {
            rc = fail(BNX_E_OVERFLOW, "the radical run flagged 0x%x (0x%x: an index outside its buffer)",
                      c->h_ctr->err, kErrBounds);
        }
    }
    if (c->rad_stage.bytes > ((size_t)1 << 28)) {  // a large staging buffer is not kept
        cudaStreamSynchronize(s);
        release(c->rad_stage);
    }
    return rc;
}

}  // extern "C"

namespace bnx {
// bnx_rad_segment's work, for callers that already hold the context.
int rad_segment_unlocked(bnx_ctx *c, uint64_t lo, uint64_t len, uint64_t *rad_out, uint64_t *sq_out,
                         cudaStream_t s) {
    IvDev iv;
    memset(&iv, 0, sizeof iv);
    iv.lo = lo;
    iv.hi = lo + len;
    iv.kinds = 3;
    PlanTotals t;
    plan_host(c, &iv, 1, &t);
    int rc = ensure_ws(c, t, 1);
    if (rc) return rc;
    CUDA_TRY(cudaStreamSynchronize(s));  // the staging buffers below are reused across calls
    c->h_ivs[0] = iv;
    c->h_nk = 1;
    CUDA_TRY(cudaMemcpyAsync(c->ivs.p, c->h_ivs, sizeof(IvDev), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(c->n_iv.p, &c->h_nk, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    c->rad_out = rad_out;
    c->sq_out = sq_out;
    c->rad_lo = lo;
    c->rad_len = len;
    rc = record_pipeline(c, kModeRad, s, false);
    c->rad_out = c->sq_out = nullptr;
    return rc;
}
}  // namespace bnx

extern "C" {

uint32_t bnx_log_weight(uint64_t p, uint32_t frac_log2) { return log_weight(p, frac_log2); }

uint32_t bnx_log_weight54(uint64_t p) { return log_weight54(p); }

int bnx_same_rad(const uint64_t *x, const uint64_t *y, size_t n, uint8_t *out) {
    if (n == 0) return BNX_OK;
    if (!x || !y || !out) return fail(BNX_E_ARG, "NULL argument");
    if (n > ((size_t)1 << 24)) return fail(BNX_E_ARG, "at most 2^24 pairs per call");
    for (size_t i = 0; i < n; i++)
        if (x[i] == 0 || y[i] == 0) return fail(BNX_E_ARG, "values must be >= 1 (pair %zu)", i);
    DevBuf b;
    int rc = grow(b, n * (2 * sizeof(uint64_t) + 1));
    if (rc) return rc;
    uint64_t *dx = (uint64_t *)b.p, *dy = dx + n;
    uint8_t *dout = (uint8_t *)(dy + n);
    cudaError_t e = cudaMemcpy(dx, x, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(dy, y, n * sizeof(uint64_t), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        launch_same_rad(dx, dy, n, dout, nullptr);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpy(out, dout, n, cudaMemcpyDeviceToHost);
    release(b);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BNX_E_CUDA, "same_rad: %s", cudaGetErrorString(e));
    }
    return BNX_OK;
}

int bnx_log_weights(bnx_ctx *c, uint32_t tile_kind, uint32_t *out, size_t cap, size_t *n_out) {
    if (!c || !n_out) return fail(BNX_E_ARG, "NULL argument");
    if (tile_kind != kTileLog32 && tile_kind != kTileLog16 && tile_kind != kTileLog8)
        return fail(BNX_E_ARG, "tile_kind must be 0, 2 or 3 (a log-domain tile)");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    *n_out = c->np;
    const size_t ncopy = std::min<size_t>(c->np, cap);
    if (ncopy == 0) return c->np > cap ? fail(BNX_E_TRUNCATED, "%u primes, buffer holds %zu", c->np, cap) : BNX_OK;
    if (!out) return fail(BNX_E_ARG, "out is NULL");
    DevBuf w;
    int rc = grow(w, sizeof(uint32_t) * 4 * (size_t)c->np);
    if (rc) return rc;
    const int vb = tile_kind == kTileLog8 ? 1 : tile_kind == kTileLog16 ? 2 : 4;
    launch_log_weights((const uint32_t *)c->primes.p, c->np, vb, (uint32_t *)w.p, c->stream);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, w.p, sizeof(uint32_t) * 4 * ncopy, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    release(w);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(BNX_E_CUDA, "log weights: %s", cudaGetErrorString(e));
    }
    return c->np > cap ? fail(BNX_E_TRUNCATED, "%u primes, buffer holds %zu", c->np, cap) : BNX_OK;
}

}  // extern "C"

// Queue-segment length (log2) for a run over one interval of len integers: the tuned
// length, or shorter (down to one tile) when the interval would otherwise give fewer
// than about two segments per CTA of the persistent grid -- a short search then still
// spreads over many CTAs instead of running on a few.
static uint32_t single_seg_log2(bnx_ctx *c, uint64_t len) {
    const uint32_t tuned = c->seg_log2_tuned();
    int grid = 0, threads = 0;
    size_t smem = 0;
    if (sieve_config(c, kModeSearch, &grid, &threads, &smem) != BNX_OK || grid <= 0) {
        g_last_error.clear();
        return tuned;  // the run itself reports the problem
    }
    uint32_t s = c->tune.tile_log2;
    while (s < tuned && ((uint64_t)4 << s) * (uint64_t)grid <= len) s++;
    return s;
}

// One n-range through the staged pipeline (bnx_search and bnx_search_segment).
static int search_one(bnx_ctx *c, uint64_t lo, uint64_t hi, uint32_t kinds, bnx_pair *out, size_t cap,
                      size_t *n_out) {
    int rc = validate_interval(c, lo, hi, kinds);
    if (rc) return rc;
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    struct SegGuard {  // the run's segment length, back to the tuned one on every return
        bnx_ctx *c;
        ~SegGuard() { c->seg_log2_run = 0; }
    } seg_guard{c};
    c->seg_log2_run = single_seg_log2(c, hi - lo);
    PlanTotals t;
    IvDev iv;
    memset(&iv, 0, sizeof iv);
    iv.lo = lo;
    iv.hi = hi;
    iv.kinds = kinds;
    plan_host(c, &iv, 1, &t);
    if ((rc = ensure_ws(c, t, 1))) return rc;
    c->h_ivs[0] = iv;
    return search_staged(c, 1, out, cap, n_out, nullptr);
}

extern "C" {

int bnx_search(bnx_ctx *c, uint64_t lo, uint64_t hi, uint32_t kinds, bnx_pair *out, size_t cap, size_t *n_out) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    return search_one(c, lo, hi, kinds, out, cap, n_out);
}

int bnx_search_segment(bnx_ctx *c, uint64_t lo, uint32_t len, uint32_t kinds, bnx_pair *out, size_t cap,
                       size_t *n_out) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    // (lo > max_hi - len, not lo + len > max_hi: the sum could wrap)
    if (len < 1 || lo < 1 || len > c->max_hi || lo > c->max_hi - len)
        return fail(BNX_E_ARG, "need len >= 1, lo >= 1 and lo + len <= max_hi");
    return search_one(c, lo, lo + len, kinds, out, cap, n_out);
}

// Checkpoint file of bnx_search_checkpointed: this header, then `npairs` bnx_pair
// records (host byte order).
struct CkptHeader {
    char magic[8];  // "BNXCKPT1"
    uint64_t lo, hi;
    uint32_t kinds, pad;
    uint64_t next, npairs;
};
static const char kCkptMagic[8] = {'B', 'N', 'X', 'C', 'K', 'P', 'T', '1'};

// BNX_OK with *found = false when the file does not exist
static int read_checkpoint(const char *path, CkptHeader *h, std::vector<bnx_pair> &pairs, bool *found) {
    *found = false;
    FILE *f = fopen(path, "rb");
    if (!f) {
        if (errno == ENOENT) return BNX_OK;
        return fail(BNX_E_ARG, "cannot open checkpoint %s", path);
    }
    int rc = BNX_OK;
    long size = -1;  // the file's length, checked against its header before anything is allocated
    if (fseek(f, 0, SEEK_END) == 0) size = ftell(f);
    rewind(f);
    if (size < (long)sizeof *h || fread(h, sizeof *h, 1, f) != 1 || memcmp(h->magic, kCkptMagic, 8) != 0 ||
        h->next < h->lo || h->next > h->hi) {
        rc = fail(BNX_E_ARG, "%s is not a checkpoint of this library", path);
    } else if (h->npairs != ((uint64_t)size - sizeof *h) / sizeof(bnx_pair) ||
               ((uint64_t)size - sizeof *h) % sizeof(bnx_pair) != 0) {
        rc = fail(BNX_E_ARG, "checkpoint %s: %llu pairs in the header, %ld bytes in the file", path,
                  (unsigned long long)h->npairs, size);
    } else {
        pairs.resize(h->npairs);  // the size matches the file (an allocation failure is caught outside)
        if (h->npairs && fread(pairs.data(), sizeof(bnx_pair), h->npairs, f) != h->npairs)
            rc = fail(BNX_E_ARG, "checkpoint %s is truncated", path);
    }
    fclose(f);
    if (rc == BNX_OK) *found = true;
    return rc;
}

// write to path.tmp, flush it to the disk, then rename it over path
static int write_checkpoint(const char *path, const CkptHeader &h, const std::vector<bnx_pair> &pairs) {
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "wb");
    if (!f) return fail(BNX_E_ARG, "cannot write checkpoint %s", tmp.c_str());
    bool ok = fwrite(&h, sizeof h, 1, f) == 1;
    if (ok && !pairs.empty()) ok = fwrite(pairs.data(), sizeof(bnx_pair), pairs.size(), f) == pairs.size();
    ok = ok && fflush(f) == 0 && fsync(fileno(f)) == 0;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return fail(BNX_E_ARG, "cannot write checkpoint %s", path);
    }
    return BNX_OK;
}

static int search_checkpointed(bnx_ctx *c, uint64_t lo, uint64_t hi, uint32_t kinds, const char *path, uint64_t chunk,
                               uint64_t max_chunks, bnx_pair *out, size_t cap, size_t *n_out, uint64_t *next) {
    if (!c || !path) return fail(BNX_E_ARG, "NULL argument");
    if (chunk < 1) return fail(BNX_E_ARG, "chunk must be >= 1");
    int rc = validate_interval(c, lo, hi, kinds);
    if (rc) return rc;
    CkptHeader h;
    std::vector<bnx_pair> pairs;
    bool found = false;
    if ((rc = read_checkpoint(path, &h, pairs, &found))) return rc;
    if (found && (h.lo != lo || h.hi != hi || h.kinds != kinds))
        return fail(BNX_E_STATE, "%s holds another search: [%llu, %llu) kinds %u", path, (unsigned long long)h.lo,
                    (unsigned long long)h.hi, h.kinds);
    if (!found) {
        memset(&h, 0, sizeof h);
        memcpy(h.magic, kCkptMagic, 8);
        h.lo = lo;
        h.hi = hi;
        h.kinds = kinds;
        h.next = lo;
    }
    std::vector<bnx_pair> part(64);
    for (uint64_t done = 0; h.next < hi && done < max_chunks; done++) {
        const uint64_t end = chunk >= hi - h.next ? hi : h.next + chunk;
        NvtxRange r_chunk("bnx.checkpoint.chunk");
        size_t np = 0;
        rc = search_one(c, h.next, end, kinds, part.data(), part.size(), &np);
        if (rc == BNX_E_TRUNCATED) {
            part.resize(np);
            rc = search_one(c, h.next, end, kinds, part.data(), part.size(), &np);
        }
        if (rc) return rc;  // the checkpoint still holds the last finished chunk
        pairs.insert(pairs.end(), part.begin(), part.begin() + np);
        h.next = end;
        h.npairs = pairs.size();
        NvtxRange r_write("bnx.checkpoint.write");
        if ((rc = write_checkpoint(path, h, pairs))) return rc;
    }
    if (next) *next = h.next;
    if (n_out) *n_out = pairs.size();
    if (pairs.size() > cap) return fail(BNX_E_TRUNCATED, "%zu pairs, buffer holds %zu", pairs.size(), cap);
    if (!pairs.empty() && !out) return fail(BNX_E_ARG, "out is NULL");
    if (!pairs.empty()) memcpy(out, pairs.data(), pairs.size() * sizeof(bnx_pair));
    if (h.next < hi) return fail(BNX_E_BUSY, "stopped at %llu: call again to resume", (unsigned long long)h.next);
    return BNX_OK;
}

int bnx_search_checkpointed(bnx_ctx *c, uint64_t lo, uint64_t hi, uint32_t kinds, const char *path, uint64_t chunk,
                            uint64_t max_chunks, bnx_pair *out, size_t cap, size_t *n_out, uint64_t *next) {
    return guarded([&] { return search_checkpointed(c, lo, hi, kinds, path, chunk, max_chunks, out, cap, n_out, next); });
}

int bnx_batch(bnx_ctx *c, const bnx_interval *ivs, size_t k, bnx_pair *out, size_t cap, size_t *n_out,
              uint64_t *offsets) {
    if (!c || (!ivs && k)) return fail(BNX_E_ARG, "NULL argument");
    if (k == 0) {
        if (n_out) *n_out = 0;
        if (offsets) offsets[0] = 0;
        return BNX_OK;
    }
    if (k > (1u << 24)) return fail(BNX_E_ARG, "at most 2^24 intervals per batch");
    for (size_t i = 0; i < k; i++) {
        int rc = validate_interval(c, ivs[i].lo, ivs[i].hi, ivs[i].kinds);
        if (rc) return rc;
    }
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    int rc = ensure_staging(c, k);
    if (rc) return rc;
    for (size_t i = 0; i < k; i++) {
        IvDev &d = c->h_ivs[i];
        memset(&d, 0, sizeof d);
        d.lo = ivs[i].lo;
        d.hi = ivs[i].hi;
        d.kinds = ivs[i].kinds;
        d.id = ivs[i].id;
    }
    return search_staged(c, k, out, cap, n_out, offsets);
}

int bnx_search_hash(bnx_ctx *c, uint64_t S, uint32_t kinds, bnx_pair *out, size_t cap, size_t *n_out) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    if (S < 2 || S > (1ull << 40) || S > c->max_hi) return fail(BNX_E_ARG, "need 2 <= S <= min(2^40, max_hi)");
    if (kinds < 1 || kinds > 3) return fail(BNX_E_ARG, "kinds must be 1, 2 or 3");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    cudaStream_t s = c->stream;
    IvDev iv;
    memset(&iv, 0, sizeof iv);
    iv.lo = 1;
    iv.hi = S;
    iv.kinds = 3;
    PlanTotals t;
    plan_host(c, &iv, 1, &t);
    for (int attempt = 0; attempt < 4; attempt++) {
        int rc = ensure_ws(c, t, 1);
        if (rc) return rc;
        c->h_ivs[0] = iv;
        c->h_nk = 1;
        CUDA_TRY(cudaMemcpyAsync(c->ivs.p, c->h_ivs, sizeof(IvDev), cudaMemcpyHostToDevice, s));
        CUDA_TRY(cudaMemcpyAsync(c->n_iv.p, &c->h_nk, sizeof(uint32_t), cudaMemcpyHostToDevice, s));
        c->hash_S = S;
        CUDA_TRY(cudaEventRecord(c->ev0, s));
        if ((rc = record_pipeline(c, kModeHash, s, true))) return rc;
        CUDA_TRY(cudaStreamSynchronize(s));
        if (c->h_ctr->err & (kErrSurvOverflow | kErrCandOverflow)) {
            if (c->h_ctr->err & kErrSurvOverflow) c->surv_want = (size_t)(c->h_ctr->n_surv + c->h_ctr->n_surv / 2 + 1024);
            if (c->h_ctr->err & kErrCandOverflow) c->cand_want = (size_t)(c->h_ctr->n_cand + c->h_ctr->n_cand / 2 + 1024);
            continue;
        }
        if (c->h_ctr->err) return fail(BNX_E_OVERFLOW, "device capacity exceeded (flags 0x%x)", c->h_ctr->err);
        const uint64_t ns = c->h_ctr->n_surv;
        uint64_t slots = 1024;
        while (slots < 2 * ns) slots <<= 1;
        if ((rc = grow(c->hkeys, slots * 8)) || (rc = grow(c->hheads, slots * 4)) ||
            (rc = grow(c->hnext, (ns + 1) * 4)) || (rc = grow(c->hslot, (ns + 1) * 4)))
            return rc;
        c->hash_mask = slots - 1;
        CUDA_TRY(cudaMemsetAsync(c->hkeys.p, 0, slots * 8, s));
        CUDA_TRY(cudaMemsetAsync(c->hheads.p, 0xff, slots * 4, s));
        Plan P = make_plan(c);
        launch_hash_insert(P, c->n_sm * 4, s);
        launch_hash_pairs(P, kinds, c->n_sm * 4, s);
        launch_sort(P, c->n_sm * 2, s);
        CUDA_TRY(cudaMemcpyAsync(c->h_ctr, c->ctr.p, sizeof(Counters), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(c->ev1, s));
        CUDA_TRY(cudaStreamSynchronize(s));
        bool rerun = false;
        rc = check_counters(c, &rerun);
        if (rerun) continue;
        if (rc) return rc;
        fill_stats(c, t.integers);
        const size_t np = (size_t)c->h_ctr->n_pairs;
        if (n_out) *n_out = np;
        const size_t ncopy = std::min(np, cap);
        if (ncopy) {
            if (!out) return fail(BNX_E_ARG, "out is NULL");
            CUDA_TRY(cudaMemcpy(out, c->pairs_sorted.p, sizeof(PairDev) * ncopy, cudaMemcpyDeviceToHost));
        }
        if (np > cap) return fail(BNX_E_TRUNCATED, "%zu pairs, buffer holds %zu", np, cap);
        return BNX_OK;
    }
    return fail(BNX_E_OVERFLOW, "device capacities kept overflowing");
}

}  // extern "C"
