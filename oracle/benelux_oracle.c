/*
 * Benelux-pair oracle: a plain, slow, obviously correct CPU implementation.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path (the CUDA library and
 * its Python binding) may include, link, load or call this file.  Only the test
 * suite, the smoke check and the benchmark's CPU-baseline leg use it.  It shares
 * no code, header, table or constant with the CUDA path.
 *
 * What it computes (Hercher, "On one of Erdos' Problems -- An Efficient Search
 * for Benelux Pairs", arXiv 2506.01099):
 *
 *   rad(x)      product of the distinct primes dividing x, rad(1) = 1   (Sec. 2.1)
 *   first kind  1 <= m < n, rad(m) = rad(n) and rad(m+1) = rad(n+1)      (Sec. 1)
 *   second kind 1 <= m < n, rad(m) = rad(n+1) and rad(m+1) = rad(n)      (Sec. 1)
 *   three-term  a first-kind pair with also rad(m+2) = rad(n+2): the question
 *               Erdos asked, quoted in Sec. 1 (kind 4 in the output)
 *
 * The search contract is the one of Algorithm 3: for n in [lo, hi) report every
 * pair (m, n) of the requested kinds with any m < n.  Results are sorted by
 * (n, m, kind).
 *
 * Functions and the passage each follows:
 *   orc_rad_td       definition of rad (Sec. 2.1), by trial division
 *   orc_rad_sieve    Algorithm 1 (radicals of an interval by prime-power sieving)
 *   orc_pairs_brute  definitions of Sec. 1, every m < n compared (tiny N only)
 *   orc_pairs_sort   Algorithm 2 (sort the 2-sets {rad n, rad n+1}); every pair
 *                    inside a group of equal sets is reported, not only adjacent
 *                    entries (a group can hold three integers: {2,3} for 2, 3, 8)
 *   orc_pairs_map    the same 2-sets collected in a hash table of key -> list of n
 *                    (the collision search of Algorithm 3, Sec. 2.2, over one
 *                    range), an independent route to orc_pairs_sort's result
 *   orc_pairs_crt    the candidate enumeration that the Chinese remainder theorem
 *                    forces on any pair (derived below); candidates are verified
 *                    with orc_rad_td, never with the gcd shortcut of the GPU path
 *   orc_filter_counts  the per-kind necessary conditions, counted (diagnostic)
 *   orc_hash_keys    integers whose key a full-range hash search has to insert
 *
 * CRT argument (not in the paper; it is what makes windows far above 1
 * checkable).  Let a = rad(n), b = rad(n+1); gcd(a, b) = 1.
 *   first kind : a | m, a | n, b | m+1, b | n+1  =>  ab | n - m, so the only
 *                candidates are m = n - j*ab, 1 <= j <= (n-1)/ab.
 *   second kind: b | m, b | n+1, a | m+1, a | n  =>  ab | m + n + 1, so the only
 *                candidates are m = j*ab - n - 1 with n+2 <= j*ab <= 2n.
 *
 * Plausible-mistake hooks: building with -DORC_MUTANT=<k> plants one deliberate
 * error (see the ORC_MUTANT blocks).  The CPU tests build each mutant and check
 * that at least one pin catches it.  The default build has none of them.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

typedef unsigned __int128 u128;

typedef struct {
    uint64_t m, n;
    uint32_t kind;
    uint32_t pad;
} orc_pair;

/* ------------------------------------------------------------------------ */
/* primes by the sieve of Eratosthenes (textbook)                             */
/* ------------------------------------------------------------------------ */

static uint32_t *g_primes = NULL; /* all primes <= g_plim */
static uint64_t g_nprimes = 0;
static uint64_t g_plim = 0;

static int ensure_primes(uint64_t lim) {
    if (lim <= g_plim && g_primes) return 0;
    if (lim < 1024) lim = 1024;
    unsigned char *comp = (unsigned char *)calloc(lim + 1, 1);
    if (!comp) return -1;
    for (uint64_t i = 2; i * i <= lim; i++)
        if (!comp[i])
            for (uint64_t j = i * i; j <= lim; j += i) comp[j] = 1;
    uint64_t cnt = 0;
    for (uint64_t i = 2; i <= lim; i++) cnt += !comp[i];
    uint32_t *pr = (uint32_t *)malloc(cnt * sizeof(uint32_t));
    if (!pr) {
        free(comp);
        return -1;
    }
    cnt = 0;
    for (uint64_t i = 2; i <= lim; i++)
        if (!comp[i]) pr[cnt++] = (uint32_t)i;
    free(comp);
    free(g_primes);
    g_primes = pr;
    g_nprimes = cnt;
    g_plim = lim;
    return 0;
}

static uint64_t isqrt_u64(uint64_t x) {
    uint64_t r = 0;
    /* r = largest integer with r*r <= x, found bit by bit */
    for (int b = 31; b >= 0; b--) {
        uint64_t t = r | ((uint64_t)1 << b);
        if ((u128)t * t <= x) r = t;
    }
    return r;
}

/* Prepare the prime list for arguments up to x_max (called once by the host
 * before any parallel region; the functions below also call it). */
int orc_init(uint64_t x_max) { return ensure_primes(isqrt_u64(x_max) + 1); }

uint64_t orc_nprimes_upto(uint64_t lim) {
    if (ensure_primes(lim)) return 0;
    uint64_t c = 0;
    while (c < g_nprimes && g_primes[c] <= lim) c++;
    return c;
}

/* ------------------------------------------------------------------------ */
/* rad by its definition (Sec. 2.1)                                            */
/* ------------------------------------------------------------------------ */

/* rad(x) = product of the distinct primes p | x; rad(1) = 1; rad(0) is not
 * defined and returns 0.  Trial division by the primes while p*p <= cofactor;
 * a cofactor > 1 left at the end is itself prime. */
uint64_t orc_rad_td(uint64_t x) {
    if (x == 0) return 0;
    if (ensure_primes(isqrt_u64(x) + 1)) return 0;
    uint64_t c = x, r = 1;
    for (uint64_t i = 0; i < g_nprimes; i++) {
        uint64_t p = g_primes[i];
        if (p * p > c) break;
        if (c % p == 0) {
            r *= p;
            while (c % p == 0) c /= p;
        }
    }
#if ORC_MUTANT == 1 /* mistake: the last prime cofactor is dropped */
    (void)c;
#else
    if (c > 1) r *= c;
#endif
    return r;
}

/* x / rad(x): the product of p^(e-1) over the prime powers p^e || x. */
uint64_t orc_sq_td(uint64_t x) {
    uint64_t r = orc_rad_td(x);
    return r ? x / r : 0;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 1: radicals of [start, start+length) by prime-power sieving       */
/* ------------------------------------------------------------------------ */

/* Readings of the printed algorithm: the "continue, move to the next prime"
 * inside the exponent loop ends that loop (a prime power with no multiple in
 * the interval leaves none for its higher powers either), and the test is
 * shift >= length (shift == length already lies outside the interval).
 * S = start + length - 1 is the largest integer of the interval. */
int orc_rad_sieve(uint64_t start, uint64_t length, uint64_t *r) {
    if (start == 0 || length == 0) return -1;
    uint64_t S = start + length - 1;
    uint64_t plim = isqrt_u64(S);
    if (ensure_primes(plim + 1)) return -1;
    for (uint64_t i = 0; i < length; i++) r[i] = start + i;
    for (uint64_t t = 0; t < g_nprimes; t++) {
        uint64_t p = g_primes[t];
#if ORC_MUTANT == 7 /* mistake: primes p < sqrt(S) only */
        if (p * p >= S) break;
#else
        if (p > plim) break;
#endif
#if ORC_MUTANT == 3 /* mistake: exponent starts at 1 */
        uint64_t pe = p;
#else
        uint64_t pe = p * p; /* p^exponent, exponent = 2 */
#endif
        while (pe <= S) {
            uint64_t res = start % pe;
#if ORC_MUTANT == 2 /* mistake: the res = 0 case is not mapped to p^e */
#else
            if (res == 0) res = pe;
#endif
            uint64_t shift = pe - res;
            if (shift >= length) break;
            for (uint64_t k = 0; k <= (length - 1 - shift) / pe; k++) r[shift + k * pe] /= p;
            if (pe > S / p) break; /* next power exceeds S */
            pe *= p;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* pair predicates by definition (Sec. 1)                                      */
/* ------------------------------------------------------------------------ */

static int cmp_pair(const void *x, const void *y) {
    const orc_pair *a = (const orc_pair *)x, *b = (const orc_pair *)y;
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    if (a->m != b->m) return a->m < b->m ? -1 : 1;
    if (a->kind != b->kind) return a->kind < b->kind ? -1 : 1;
    return 0;
}

static void push_pair(orc_pair *out, size_t cap, size_t *cnt, uint64_t m, uint64_t n, uint32_t kind) {
    if (*cnt < cap) {
        out[*cnt].m = m;
        out[*cnt].n = n;
        out[*cnt].kind = kind;
        out[*cnt].pad = 0;
    }
    (*cnt)++;
}

/* The definitions of Sec. 1 applied to a given array of radicals r[1 .. N+1]
 * (r[0] unused): every 1 <= m < n < N is compared, first kind r[m] = r[n] and
 * r[m+1] = r[n+1], second kind r[m] = r[n+1] and r[m+1] = r[n], three-term a
 * first-kind pair with also r[m+2] = r[n+2] (Erdos's question, Sec. 1).  The
 * array may be anything (the tests plant collisions no real radicals give).
 * Returns the number of pairs (which may exceed cap; only cap are written),
 * sorted by (n, m, kind).  2 <= N <= 2^14. */
size_t orc_pairs_brute_rad(const uint64_t *r, uint64_t N, uint32_t kinds, orc_pair *out, size_t cap) {
    if (!r || N < 2 || N > (1u << 14)) return 0;
    size_t cnt = 0;
    for (uint64_t n = 2; n < N; n++)
        for (uint64_t m = 1; m < n; m++) {
#if ORC_MUTANT == 8 /* mistake: operands transposed in the first-kind test */
            if ((kinds & 1) && r[m] == r[n + 1] && r[m + 1] == r[n + 1]) push_pair(out, cap, &cnt, m, n, 1);
#else
            if ((kinds & 1) && r[m] == r[n] && r[m + 1] == r[n + 1]) push_pair(out, cap, &cnt, m, n, 1);
#endif
            if ((kinds & 2) && r[m] == r[n + 1] && r[m + 1] == r[n]) push_pair(out, cap, &cnt, m, n, 2);
#if ORC_MUTANT == 9 /* mistake: the three-term rule compares m + 2 with n + 1 */
            if ((kinds & 4) && r[m] == r[n] && r[m + 1] == r[n + 1] && r[m + 2] == r[n + 1])
#else
            if ((kinds & 4) && r[m] == r[n] && r[m + 1] == r[n + 1] && r[m + 2] == r[n + 2])
#endif
                push_pair(out, cap, &cnt, m, n, 4);
        }
    if (cnt && cnt <= cap) qsort(out, cnt, sizeof(orc_pair), cmp_pair);
    return cnt;
}

/* Every 1 <= m < n < N is compared; rad by trial division.  Returns the number
 * of pairs (which may exceed cap; only cap are written).  N <= 2^14. */
size_t orc_pairs_brute(uint64_t N, uint32_t kinds, orc_pair *out, size_t cap) {
    if (N < 2 || N > (1u << 14)) return 0;
    uint64_t *r = (uint64_t *)malloc((N + 3) * sizeof(uint64_t));
    if (!r) return 0;
    r[0] = 0;
    for (uint64_t x = 1; x <= N + 2; x++) r[x] = orc_rad_td(x);
    const size_t cnt = orc_pairs_brute_rad(r, N, kinds, out, cap);
    free(r);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Algorithm 2: sort the 2-sets S_n = {rad n, rad n+1}                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint64_t k1, k2; /* k1 < k2 : the 2-set in the order of Sec. 2.1 */
    uint64_t n;
} set_entry;

static int cmp_set(const void *x, const void *y) {
    const set_entry *a = (const set_entry *)x, *b = (const set_entry *)y;
    if (a->k1 != b->k1) return a->k1 < b->k1 ? -1 : 1;
    if (a->k2 != b->k2) return a->k2 < b->k2 ? -1 : 1;
    if (a->n != b->n) return a->n < b->n ? -1 : 1;
    return 0;
}

/* All pairs with m < n < S.  Radicals of [1, S] by Algorithm 1, the sets sorted
 * by the lexicographic order on {a1 < a2}; inside every group of equal sets all
 * pairs m < n are reported, with kind 1 when r[m] = r[n] and kind 2 otherwise
 * (the rule of Algorithm 2).  S <= 2^26. */
size_t orc_pairs_sort(uint64_t S, uint32_t kinds, orc_pair *out, size_t cap) {
    if (S < 2 || S > (1u << 26)) return 0;
    uint64_t *r = (uint64_t *)malloc((S + 1) * sizeof(uint64_t));
    set_entry *list = (set_entry *)malloc((S - 1) * sizeof(set_entry));
    if (!r || !list) {
        free(r);
        free(list);
        return 0;
    }
    /* r[x] for x in [1, S] */
    orc_rad_sieve(1, S, r + 1);
    for (uint64_t n = 1; n < S; n++) {
        uint64_t u = r[n], v = r[n + 1];
        list[n - 1].k1 = u < v ? u : v;
        list[n - 1].k2 = u < v ? v : u;
        list[n - 1].n = n;
    }
    qsort(list, S - 1, sizeof(set_entry), cmp_set);
    size_t cnt = 0;
    uint64_t g = 0;
    while (g < S - 1) {
        uint64_t e = g + 1;
        while (e < S - 1 && list[e].k1 == list[g].k1 && list[e].k2 == list[g].k2) e++;
        for (uint64_t i = g; i < e; i++)
            for (uint64_t j = i + 1; j < e; j++) {
                uint64_t m = list[i].n, n = list[j].n; /* m < n: entries sorted by n inside a group */
#if ORC_MUTANT == 4 /* mistake: the kind rule is inverted */
                uint32_t kind = (r[m] == r[n]) ? 2 : 1;
#else
                uint32_t kind = (r[m] == r[n]) ? 1 : 2;
#endif
                if (kinds & kind) push_pair(out, cap, &cnt, m, n, kind);
            }
        g = e;
    }
    free(r);
    free(list);
    if (cnt && cnt <= cap) qsort(out, cnt, sizeof(orc_pair), cmp_pair);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* Key search by a hash table (Algorithm 3's collision detection, Sec. 2.2)    */
/* ------------------------------------------------------------------------ */

/* Open addressing, linear probing; a slot holds a key {k1 < k2} and the last n
 * inserted with it, and nxt[n] links the earlier n of the same key.  Every n
 * pairs with every earlier n of its key. */
size_t orc_pairs_map(uint64_t S, uint32_t kinds, orc_pair *out, size_t cap) {
    if (S < 2 || S > (1u << 26)) return 0;
    uint64_t slots = 1;
    while (slots < 2 * S) slots <<= 1;
    uint64_t *r = (uint64_t *)malloc((S + 1) * sizeof(uint64_t));
    uint64_t *key1 = (uint64_t *)calloc(slots, sizeof(uint64_t));
    uint64_t *key2 = (uint64_t *)calloc(slots, sizeof(uint64_t));
    uint64_t *last = (uint64_t *)calloc(slots, sizeof(uint64_t)); /* 0 = empty slot */
    uint64_t *nxt = (uint64_t *)calloc(S + 1, sizeof(uint64_t));
    size_t cnt = 0;
    if (!r || !key1 || !key2 || !last || !nxt) goto done;
    orc_rad_sieve(1, S, r + 1);
    for (uint64_t n = 1; n < S; n++) {
        const uint64_t u = r[n], v = r[n + 1];
        const uint64_t k1 = u < v ? u : v, k2 = u < v ? v : u;
        uint64_t h = (k1 * 0x9e3779b97f4a7c15ull) ^ (k2 * 0xc2b2ae3d27d4eb4full);
        h ^= h >> 29;
        uint64_t i = h & (slots - 1);
        while (last[i] && !(key1[i] == k1 && key2[i] == k2)) i = (i + 1) & (slots - 1);
        if (last[i]) {
            for (uint64_t m = last[i]; m; m = nxt[m]) {
                const uint32_t kind = (r[m] == r[n]) ? 1 : 2;
                if (kinds & kind) push_pair(out, cap, &cnt, m, n, kind);
            }
        } else {
            key1[i] = k1;
            key2[i] = k2;
        }
        nxt[n] = last[i];
        last[i] = n;
    }
    if (cnt && cnt <= cap) qsort(out, cnt, sizeof(orc_pair), cmp_pair);
done:
    free(r);
    free(key1);
    free(key2);
    free(last);
    free(nxt);
    return cnt;
}

/* ------------------------------------------------------------------------ */
/* CRT candidate enumeration for n in [lo, hi)                                 */
/* ------------------------------------------------------------------------ */

#define ORC_CHUNK ((uint64_t)1 << 20)

/* Pairs found for n in one chunk [c0, c1), appended to a growing buffer. */
typedef struct {
    orc_pair *p;
    size_t n, cap;
    int oom;
} pair_buf;

static void buf_push(pair_buf *b, uint64_t m, uint64_t n, uint32_t kind) {
    if (b->n == b->cap) {
        size_t nc = b->cap ? 2 * b->cap : 16;
        orc_pair *q = (orc_pair *)realloc(b->p, nc * sizeof(orc_pair));
        if (!q) {
            b->oom = 1;
            return;
        }
        b->p = q;
        b->cap = nc;
    }
    b->p[b->n].m = m;
    b->p[b->n].n = n;
    b->p[b->n].kind = kind;
    b->p[b->n].pad = 0;
    b->n++;
}

static void crt_chunk(uint64_t c0, uint64_t c1, uint32_t kinds, uint64_t *r, pair_buf *b, uint64_t *cnt1,
                      uint64_t *cnt2) {
    /* r[i] = rad(c0 + i) for i in [0, c1 - c0] (one extra for n+1) */
    orc_rad_sieve(c0, c1 - c0 + 1, r);
    for (uint64_t n = c0; n < c1; n++) {
        uint64_t a = r[n - c0], b2 = r[n + 1 - c0];
        u128 ab = (u128)a * b2;
        if ((kinds & 5) && ab <= (u128)(n - 1)) {
            (*cnt1)++;
            uint64_t abl = (uint64_t)ab;
            for (uint64_t j = 1; j <= (n - 1) / abl; j++) {
                uint64_t m = n - j * abl;
                if (orc_rad_td(m) == a && orc_rad_td(m + 1) == b2) {
                    if (kinds & 1) buf_push(b, m, n, 1);
                    /* three-term: also rad(m+2) = rad(n+2) (Erdos's question, Sec. 1) */
                    if ((kinds & 4) && orc_rad_td(m + 2) == orc_rad_td(n + 2)) buf_push(b, m, n, 4);
                }
            }
        }
#if ORC_MUTANT == 6 /* mistake: the first-kind inequality applied to the second kind */
        if ((kinds & 2) && ab <= (u128)(n - 1)) {
#else
        if ((kinds & 2) && ab <= (u128)2 * n) {
#endif
            uint64_t abl = (uint64_t)ab;
            uint64_t jlo = (n + 2 + abl - 1) / abl, jhi = (2 * n) / abl;
            if (jlo <= jhi) (*cnt2)++;
            for (uint64_t j = jlo; j <= jhi; j++) {
#if ORC_MUTANT == 5 /* mistake: m = j*ab - n (sign of the 1 lost) */
                uint64_t m = j * abl - n;
#else
                uint64_t m = j * abl - n - 1;
#endif
                if (m >= 1 && m < n && orc_rad_td(m) == b2 && orc_rad_td(m + 1) == a) buf_push(b, m, n, 2);
            }
        }
    }
}

static size_t crt_run(uint64_t lo, uint64_t hi, uint32_t kinds, orc_pair *out, size_t cap, int nthreads,
                      uint64_t *c1out, uint64_t *c2out) {
    if (lo < 1 || hi <= lo) return 0;
    if (orc_init(2 * hi + 2)) return 0;
    uint64_t nchunks = (hi - lo + ORC_CHUNK - 1) / ORC_CHUNK;
    pair_buf *bufs = (pair_buf *)calloc(nchunks, sizeof(pair_buf));
    uint64_t *k1 = (uint64_t *)calloc(nchunks, sizeof(uint64_t));
    uint64_t *k2 = (uint64_t *)calloc(nchunks, sizeof(uint64_t));
    if (!bufs || !k1 || !k2) {
        free(bufs);
        free(k1);
        free(k2);
        return 0;
    }
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        uint64_t *r = (uint64_t *)malloc((ORC_CHUNK + 1) * sizeof(uint64_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t c = 0; c < (int64_t)nchunks; c++) {
            uint64_t c0 = lo + (uint64_t)c * ORC_CHUNK;
            uint64_t c1 = c0 + ORC_CHUNK < hi ? c0 + ORC_CHUNK : hi;
            if (r) crt_chunk(c0, c1, kinds, r, &bufs[c], &k1[c], &k2[c]);
            else bufs[c].oom = 1;
        }
        free(r);
    }
    (void)nthreads;
    size_t cnt = 0;
    uint64_t s1 = 0, s2 = 0;
    int oom = 0;
    for (uint64_t c = 0; c < nchunks; c++) {
        for (size_t i = 0; i < bufs[c].n; i++)
            push_pair(out, cap, &cnt, bufs[c].p[i].m, bufs[c].p[i].n, bufs[c].p[i].kind);
        oom |= bufs[c].oom;
        s1 += k1[c];
        s2 += k2[c];
        free(bufs[c].p);
    }
    free(bufs);
    free(k1);
    free(k2);
    if (c1out) *c1out = s1;
    if (c2out) *c2out = s2;
    if (oom) return (size_t)-1;
    if (cnt && cnt <= cap) qsort(out, cnt, sizeof(orc_pair), cmp_pair);
    return cnt;
}

/* Every pair (m, n) of the requested kinds (bit 1: first, bit 2: second, bit 4:
 * three-term) with
 * lo <= n < hi and 1 <= m < n, sorted by (n, m, kind).  Returns the count (only
 * cap are written) or (size_t)-1 when memory ran out.  nthreads <= 0: all. */
size_t orc_pairs_crt(uint64_t lo, uint64_t hi, uint32_t kinds, orc_pair *out, size_t cap, int nthreads) {
    return crt_run(lo, hi, kinds, out, cap, nthreads, NULL, NULL);
}

/* Counts of n in [lo, hi) that pass the necessary conditions: first kind
 * rad(n)rad(n+1) <= n-1; second kind some multiple of rad(n)rad(n+1) lies in
 * [n+2, 2n].  A diagnostic of the filter stage. */
int orc_filter_counts(uint64_t lo, uint64_t hi, uint32_t kinds, uint64_t *cnt1, uint64_t *cnt2, int nthreads) {
    /* the pair buffer is thrown away: cap 0 */
    size_t r = crt_run(lo, hi, kinds, NULL, 0, nthreads, cnt1, cnt2);
    return r == (size_t)-1 ? -1 : 0;
}

/* Number of x in [1, S) with rad(x)*rad(x+1) <= 2S: the keys a full-range hash
 * search over n < S has to insert (every member m or n of a pair with n < S
 * has rad(m)rad(m+1) = rad(n)rad(n+1) <= 2n < 2S).  Radicals by trial division. */
uint64_t orc_hash_keys(uint64_t S) {
    if (S < 2) return 0;
    orc_init(S + 1);
    uint64_t c = 0, prev = orc_rad_td(1);
    for (uint64_t x = 1; x < S; x++) {
        uint64_t nx = orc_rad_td(x + 1);
        if ((u128)prev * nx <= (u128)2 * S) c++;
        prev = nx;
    }
    return c;
}
