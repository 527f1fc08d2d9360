// Candidate verification, the device hash table of the full-range search, and
// the output sort.
//
// Verification (one warp per survivor n, lanes over the candidates j):
//   first kind : m = n - j*ab, 1 <= j <= (n-1)/ab; accept if rad(m) = a and
//                rad(m+1) = b
//   second kind: m = j*ab - n - 1, n+2 <= j*ab <= 2n; accept if rad(m) = b and
//                rad(m+1) = a
// The candidates already satisfy a | m and b | m+1 (or b | m, a | m+1), so
// rad(m) = r exactly when every prime of m/r divides r: strip gcd(x, r) from
// x = m/r until it is 1 (accept) or the gcd is 1 (reject).  No factorisation.
//
// Hash table (the collision detection of Algorithms 2 and 3, Sec. 2.2 and
// 3.1): open addressing over 64-bit keys.  For a key {a, b} with ab <= 2S <= 2^41,
// min(a, b) < 2^21, so key = (ab << 21) | min(a, b) is exact and nonzero.  A slot
// is claimed with one compare-and-swap; the integers sharing a slot are chained
// through an exchange on the slot's head.  Every two integers on one chain have
// equal 2-sets and form a pair; its kind is 1 when their radicals agree
// (Algorithm 2's test r[m] = r[n]).
#include "bnx_internal.cuh"

namespace bnx {

namespace {

__device__ __forceinline__ uint64_t gcd64(uint64_t u, uint64_t v) {
    if (u == 0) return v;
    if (v == 0) return u;
    const uint32_t shift = __ffsll((long long)(u | v)) - 1;
    u >>= __ffsll((long long)u) - 1;
    do {
        v >>= __ffsll((long long)v) - 1;
        if (u > v) {
            const uint64_t t = u;
            u = v;
            v = t;
        }
        v -= u;
    } while (v != 0);
    return u << shift;
}

// rad(m) == r, given that r is squarefree and r | m
__device__ __forceinline__ bool rad_is(uint64_t m, uint64_t r) {
    uint64_t x = m / r;
    while (x > 1) {
        const uint64_t g = gcd64(x, r);
        if (g == 1) return false;
        x /= g;
    }
    return true;
}

// rad(x) == rad(y): every prime of x divides y and every prime of y divides x
__device__ __forceinline__ bool strip_by(uint64_t x, uint64_t y) {
    while (x > 1) {
        const uint64_t g = gcd64(x, y);
        if (g == 1) return false;
        x /= g;
    }
    return true;
}

__device__ __forceinline__ bool same_rad(uint64_t x, uint64_t y) { return strip_by(x, y) && strip_by(y, x); }

__device__ __forceinline__ void emit_pair(const Plan &P, uint64_t m, uint64_t n, uint32_t kind, uint32_t iv) {
    const unsigned long long at = atomicAdd(&P.ctr->n_pairs, 1ull);
    if (at < P.pair_cap) {
        PairDev pr;
        pr.m = m;
        pr.n = n;
        pr.kind = kind;
        pr.iv = iv;
        P.pairs[at] = pr;
    } else {
        atomicOr(&P.ctr->err, kErrPairOverflow);
    }
}

__global__ void k_verify(Plan P) {
    const unsigned long long ns0 = P.ctr->n_surv;
    const unsigned long long ns = ns0 < P.surv_cap ? ns0 : P.surv_cap;
    const uint32_t lane = threadIdx.x & 31;
    const unsigned long long gw = ((unsigned long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const unsigned long long nw = ((unsigned long long)gridDim.x * blockDim.x) >> 5;
    for (unsigned long long w = gw; w < ns; w += nw) {
        const Survivor s = P.surv[w];
        const uint64_t n = s.n;
        const uint64_t ab = s.a * s.b;  // <= 2n: passed the filter
        unsigned long long cands = 0;
        const uint32_t want = P.ivs[s.iv].kinds;
        if (s.kinds & 1) {
            const uint64_t J = (n - 1) / ab;
            cands += J;
            for (uint64_t j = 1 + lane; j <= J; j += 32) {
                const uint64_t m = n - j * ab;
                if (rad_is(m, s.a) && rad_is(m + 1, s.b)) {
                    if (want & 1) emit_pair(P, m, n, 1, s.iv);
                    // Erdos's three-term question (Sec. 1): also rad(m+2) = rad(n+2)
                    if ((want & 4) && same_rad(m + 2, n + 2)) emit_pair(P, m, n, 4, s.iv);
                }
            }
        }
        if (s.kinds & 2) {
            const uint64_t jlo = (n + 2 + ab - 1) / ab, jhi = (2 * n) / ab;
            cands += jhi >= jlo ? jhi - jlo + 1 : 0;
            for (uint64_t j = jlo + lane; j <= jhi; j += 32) {
                const uint64_t m = j * ab - n - 1;
                if (rad_is(m, s.b) && rad_is(m + 1, s.a)) emit_pair(P, m, n, 2, s.iv);
            }
        }
        if (lane == 0 && cands) atomicAdd(&P.ctr->candidates, cands);
    }
}

__device__ __forceinline__ bool key_less(const PairDev &x, const PairDev &y) {
    if (x.iv != y.iv) return x.iv < y.iv;
    if (x.n != y.n) return x.n < y.n;
    if (x.m != y.m) return x.m < y.m;
    return x.kind < y.kind;
}

// rank sort: out[#{j : key_j < key_i, or equal with j < i}] = in[i]
__global__ void k_sort(Plan P) {
    const unsigned long long np0 = P.ctr->n_pairs;
    const unsigned long long np = np0 < P.pair_cap ? np0 : P.pair_cap;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < np;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const PairDev me = P.pairs[i];
        unsigned long long r = 0;
        for (unsigned long long j = 0; j < np; j++) {
            const PairDev o = P.pairs[j];
            if (key_less(o, me) || (!key_less(me, o) && j < i)) r++;
        }
        P.pairs_sorted[r] = me;
    }
}

// offsets[v] = first sorted pair of interval v (lower bound), v in [0, k]
__global__ void k_offsets(Plan P) {
    const unsigned long long np0 = P.ctr->n_pairs;
    const unsigned long long np = np0 < P.pair_cap ? np0 : P.pair_cap;
    const uint32_t k = *P.n_iv;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v <= k; v += gridDim.x * blockDim.x) {
        unsigned long long lo = 0, hi = np;
        while (lo < hi) {
            const unsigned long long mid = (lo + hi) >> 1;
            if (P.pairs_sorted[mid].iv < v) lo = mid + 1;
            else hi = mid;
        }
        P.iv_offsets[v] = lo;
    }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void k_hash_insert(Plan P) {
    const unsigned long long ns0 = P.ctr->n_surv;
    const unsigned long long ns = ns0 < P.surv_cap ? ns0 : P.surv_cap;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ns;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const Survivor s = P.surv[i];
        const uint64_t mn = s.a < s.b ? s.a : s.b;
        const unsigned long long key = ((unsigned long long)(s.a * s.b) << 21) | mn;
        uint64_t h = mix64(key) & P.hash_mask;
        bool done = false;
        for (uint64_t probe = 0; probe <= P.hash_mask; probe++) {
            const unsigned long long old = atomicCAS(&P.hkeys[h], 0ull, key);
            if (old == 0ull || old == key) {
                P.hslot[i] = (uint32_t)h;
                P.hnext[i] = atomicExch(&P.hheads[h], (uint32_t)i);
                done = true;
                break;
            }
            h = (h + 1) & P.hash_mask;
        }
        if (!done) atomicOr(&P.ctr->err, kErrHashFull);
        else atomicAdd(&P.ctr->hash_keys, 1ull);
    }
}

__global__ void k_hash_pairs(Plan P, uint32_t kinds) {
    const unsigned long long ns0 = P.ctr->n_surv;
    const unsigned long long ns = ns0 < P.surv_cap ? ns0 : P.surv_cap;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ns;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const Survivor me = P.surv[i];
        uint32_t j = P.hheads[P.hslot[i]];
        for (unsigned long long steps = 0; j != 0xffffffffu && steps < ns; steps++) {
            const Survivor o = P.surv[j];
            if (o.n < me.n) {
                const uint32_t kind = o.a == me.a ? 1u : 2u;
                if (kinds & kind) emit_pair(P, o.n, me.n, kind, 0);
            }
            j = P.hnext[j];
        }
    }
}

// out[i] = rad(x[i]) == rad(y[i]) by the gcd strips k_verify uses (its three-term test)
__global__ void k_same_rad(const uint64_t *x, const uint64_t *y, uint64_t n, uint8_t *out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x)
        out[i] = same_rad(x[i], y[i]) ? 1 : 0;
}

}  // namespace

void launch_same_rad(const uint64_t *x, const uint64_t *y, uint64_t n, uint8_t *out, cudaStream_t s) {
    const uint64_t blocks = (n + 255) / 256;
    k_same_rad<<<(unsigned)(blocks < 4096 ? (blocks ? blocks : 1) : 4096), 256, 0, s>>>(x, y, n, out);
}
void launch_verify(const Plan &P, int grid, cudaStream_t s) { k_verify<<<grid, 256, 0, s>>>(P); }
void launch_sort(const Plan &P, int grid, cudaStream_t s) { k_sort<<<grid, 256, 0, s>>>(P); }
void launch_offsets(const Plan &P, int grid, cudaStream_t s) { k_offsets<<<grid, 256, 0, s>>>(P); }
void launch_hash_insert(const Plan &P, int grid, cudaStream_t s) { k_hash_insert<<<grid, 256, 0, s>>>(P); }
void launch_hash_pairs(const Plan &P, uint32_t kinds, int grid, cudaStream_t s) {
    k_hash_pairs<<<grid, 256, 0, s>>>(P, kinds);
}
void launch_zero_counters(Counters *c, cudaStream_t s) { cudaMemsetAsync(c, 0, sizeof(Counters), s); }

}  // namespace bnx
