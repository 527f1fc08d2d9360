// Exact odd square part of one value from a segment's tables (internal).
//
// The odd square part s_odd(x) = prod p^(e-1) over the odd primes p with p^e || x,
// e >= 2.  The in-tile primes (p^2 <= Q) are found by exact-division tests
// (y p^-1 mod 2^64 <= floor((2^64 - 1) / p) exactly when p | y); every larger
// prime whose square divides x has one bucket entry per power p^k (k >= 2)
// dividing x at x's offset in its segment, so multiplying s by p for each of
// those entries adds its p^(e-1).  Used where a tile's own record of x cannot
// give s_odd(x): the log tiles' candidates, and the values whose square part
// overflowed the radical kernel's 32-bit tile.
#pragma once
#include "bnx_internal.cuh"

namespace bnx {

constexpr int kMaxSmallPrimes = 128;  // in-tile primes: p^2 <= Q <= 2^16 gives at most 53 odd ones

struct SmallPrimes {
    uint32_t n;
    uint32_t p[kMaxSmallPrimes];
    unsigned long long inv[kMaxSmallPrimes];  // p^-1 mod 2^64
    unsigned long long lim[kMaxSmallPrimes];  // floor((2^64 - 1) / p)
};

// The distinct in-tile primes (those whose square is an in-tile prime power) with
// their inverses; the whole block calls it, and reads *sp after a barrier.
static __device__ __forceinline__ void load_small_primes(const Plan &P, SmallPrimes *sp) {
    if (threadIdx.x == 0) {
        uint32_t c = 0;
        for (uint32_t j = 0; j < P.n_spp && c < kMaxSmallPrimes; j++)
            if (P.spp[j].k == 2) sp->p[c++] = P.spp[j].p;
        sp->n = c;
    }
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < sp->n; t += blockDim.x) {
        const unsigned long long p = sp->p[t];
        unsigned long long inv = p;  // Newton: each step doubles the correct low bits
        for (int it = 0; it < 6; it++) inv *= 2ull - p * inv;
        sp->inv[t] = inv;
        sp->lim[t] = ~0ull / p;
    }
}

// exact odd square part of the value v at offset o of its segment, whose bucket
// entries are bent[gb .. ge)
static __device__ __noinline__ uint64_t sodd_exact(uint64_t v, uint32_t o, const SmallPrimes *sp, uint32_t sqrt_q,
                                                   const uint2 *bent, unsigned long long gb, unsigned long long ge) {
    uint64_t y = v >> (__ffsll((long long)v) - 1);
    uint64_t s = 1;
    for (uint32_t t = 0; t < sp->n; t++) {
        const unsigned long long inv = sp->inv[t], lim = sp->lim[t];
        if (y * inv <= lim) {  // p | y (exact-division test)
            y *= inv;
            while (y * inv <= lim) {
                y *= inv;
                s *= sp->p[t];
            }
        }
    }
    for (unsigned long long e = gb; e < ge; e++) {
        const uint2 h = bent[e];
        if (h.x == o && h.y > sqrt_q) s *= h.y;
    }
    return s;
}

}  // namespace bnx
