// Log-domain tile sieve for the search and hash modes (the default).
//
// The tile holds, per value x, L(x) = the sum of w(p) over the prime-power
// strikes at x, where w(p) >= F log2 p in the tile's units per bit F (2^16 for
// u32 values, 2^8 for u16, 5/4 for u8): the weights of bnx_internal.cuh, bit
// lengths of powers of p computed in integers (no floating point decides
// anything here).  So L(x) is an upper bound of F log2 s_odd(x), s_odd(x) being
// the odd part of x / rad(x).  Strikes are 32-bit shared-memory reductions (no read-modify-write
// loop: addition commutes, so strikes of different prime powers at one x need
// no ordering).  Algorithm 1 (Sec. 2.1) still decides which x a prime power
// touches; only what is recorded there changes.
//
// Filter.  With P = s(n)s(n+1) (powers of 2 included), the per-kind necessary
// conditions need 2P >= n+1 (second kind, and a fortiori the first) or
// P >= n(n+1)/(2S) (hash search).  If neither n nor n+1 is divisible by 2^M
// (M = 16), the power of 2 in P is at most 2^(M-2), so
//   log2 P <= (L(n) + L(n+1)) / F + M - 2,
// and n is rejected when that bound falls below the tile's smallest threshold.
// Every other n (a bound that does not reject, or n, n+1 next to a multiple of
// 2^M) is a candidate.  A candidate whose exact power of 2 still rejects it is
// dropped; the rest go to a list that k_cand (below) checks with exact square
// parts (exact-division tests by the in-tile primes, plus the segment's bucket
// entries of the larger primes) and the exact 128-bit conditions.
#include <algorithm>

#include "bnx_exact.cuh"
#include "bnx_internal.cuh"

namespace bnx {

namespace {

// The first 512 bucket entries of a segment (a segment of 2^19 values near 2^40
// holds about 370 at Q = 2^16) are cached in shared memory, each packed into one
// word: (offset in the segment) << 12 | cache_weight(p) (below 2^12 for
// p < 2^21).  Offsets reach the segment length, so the cache is used for
// segments of at most 2^19 values; the entries of larger segments, and those
// beyond the cache, are read from global memory.  Either way a strike adds
// bucket_weight(p) -- the u8 tile's own weight, or the weight in units of 2^-7
// scaled by 2 (u16 tile) or 2^9 (u32 tile) -- an over-estimate of F log2 p, as
// the rejection rule needs.
constexpr int kLogBucketCache = 512;
// The cached entries are then binned by tile (bsort), so that a tile reads only its own;
// an entry on a tile boundary (x = L_tile of one tile, x = 0 of the next) is in both bins.
constexpr uint32_t kMaxSegTiles = 64;
constexpr uint32_t kHigh2 = 16;
// Runs of dense strike rounds per warp (a warp's equal share of all dense rounds of a tile
// touches at most every dense prime power once; for tiles up to 2^16 there are at most 21:
// odd p^k <= 2^16/31 with k >= 2)
constexpr uint32_t kMaxRuns = 24;

// shared-memory reduction (no return value) at a 32-bit shared-window address
__device__ __forceinline__ void red_add_shared(uint32_t addr, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t ctz64(uint64_t x) { return (uint32_t)(__ffsll((long long)x) - 1); }
__device__ __forceinline__ uint32_t flog2_64(uint64_t x) { return 63u - (uint32_t)__clzll((long long)x); }

struct LogLayout {
    size_t tile, spp, sched, bcache, bsort, total;
};

__host__ __device__ inline size_t al16(size_t x) { return (x + 15) & ~(size_t)15; }

// Tile words: one u32 value per word, or two u16 or four u8 values per word
// (vb = bytes per value); the slack covers the epilogue's read past the last value.
__host__ __device__ inline LogLayout log_layout(uint32_t tile_log2, uint32_t nspp, uint32_t nsched, int vb) {
    LogLayout L;
    L.tile = 0;
    const size_t words = ((size_t)1 << tile_log2) * vb / 4 + 8;
    L.spp = al16(words * sizeof(uint32_t));
    L.sched = L.spp + al16((size_t)5 * (nspp ? nspp : 1) * sizeof(uint32_t));
    L.bcache = L.sched + al16((size_t)(nsched ? nsched : 1) * sizeof(uint16_t));
    L.bsort = L.bcache + (size_t)kLogBucketCache * sizeof(uint32_t);
    L.total = L.bsort + (size_t)(kLogBucketCache + kMaxSegTiles) * sizeof(uint32_t);
    return L;
}

// a bucket entry packed for the shared cache: its offset and its weight field
template <int VB>
__device__ __forceinline__ uint32_t pack_hit(uint2 h) {
    return (h.x << 12) | cache_weight<VB>(h.y);
}

// exact per-kind decision from the odd square parts of n and n+1
__device__ __noinline__ uint32_t exact_kinds_log(uint64_t n, uint64_t s0, uint64_t s1, uint32_t kinds, int mode,
                                                 uint64_t hash_S, uint64_t *pa, uint64_t *pb) {
    const uint32_t t0 = ctz64(n), t1 = ctz64(n + 1);
    const uint64_t sn = s0 << (t0 ? t0 - 1 : 0);
    const uint64_t sn1 = s1 << (t1 ? t1 - 1 : 0);
    const uint64_t a = n / sn, b = (n + 1) / sn1;
    *pa = a;
    *pb = b;
    const unsigned __int128 ab = (unsigned __int128)a * b;
    if (mode == kModeHash) return ab <= (unsigned __int128)2 * hash_S ? 3u : 0u;
    uint32_t r = 0;
    if ((kinds & 5) && ab <= (unsigned __int128)(n - 1)) r |= 1;  // three-term pairs are first-kind pairs
    if ((kinds & 2) && ab <= (unsigned __int128)2 * n) {
        const uint64_t abl = (uint64_t)ab;
        const uint64_t jlo = (n + 2 + abl - 1) / abl, jhi = (2 * n) / abl;
        if (jlo <= jhi) r |= 2;
    }
    return r;
}

// CTAs per SM the register allocation must allow: 64 registers per thread, or for the
// u8 tile (about 44 KB of shared memory per CTA at 2^15 values) 5 CTAs of 256 threads
// (46 registers, no spills), which measured 2% faster than 4.
template <int NT, int VB>
struct LogMinBlocks {
    static constexpr int value = NT <= 128 ? 8 : NT <= 256 ? (VB == 1 ? 5 : 4) : NT <= 512 ? 2 : 1;
};

// VB = bytes per tile value.
//  VB = 4: L(x) in 32 bits with 16 fractional bits.
//  VB = 2: 16 bits with 8 fractional bits, two values per 32-bit word.  For x < 2^42
//    L(x) <= 2^8 log2 s_odd(x) + (strikes at x) < 42 * 2^8 + 42 < 2^14, and a pair sum
//    L(n) + L(n+1) < 2^15, so a strike's addition of lg << 16*(x&1) never carries into
//    the neighbour, nor does a pair sum.
//  VB = 1: 8 bits in units of 4/5 bit (F = 5/4), four values per word.  w(p) =
//    ceil(bitlen(p^5) / 4) > (5/4) log2 p is at most 1.468 units per bit of p (p = 17,
//    w = 6, is the worst over all primes below 2^22).  s_odd(x) <= x / 3 whenever it
//    exceeds 1, so for x < 2^42, L(x) <= 1.468 (42 - log2 3) < 60 and a pair sum
//    L(n) + L(n+1) < 120 < 2^7: no strike, pair sum or threshold add below carries
//    into the neighbouring byte.
template <int MODE, int NT, int VB>
__global__ void __launch_bounds__(NT, LogMinBlocks<NT, VB>::value) k_sieve_log(Plan P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // units of L per bit: FN / FD
    constexpr uint32_t FN = VB == 4 ? 65536u : VB == 2 ? 256u : 5u;
    constexpr uint32_t FD = VB == 1 ? 4u : 1u;
    constexpr uint32_t VSH = VB == 4 ? 0u : VB == 2 ? 1u : 2u;       // value index >> VSH = word index
    constexpr uint32_t VPW = 1u << VSH;                             // values per word
    constexpr uint32_t VBITS = 8u * VB;
    constexpr uint32_t VMASK = VB == 4 ? 0xffffffffu : (1u << VBITS) - 1u;
    const uint32_t tile_log2 = P.tile_log2;
    const uint32_t LT = 1u << tile_log2;
    const uint32_t nspp = P.n_spp;
    const LogLayout lay = log_layout(tile_log2, nspp, P.n_sched, VB);
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_raw + lay.tile);
    // per in-tile prime power j: {q, lg, offset of its first multiple in the tile, 32-multiple rounds per tile}
    uint4 *sdesc = reinterpret_cast<uint4 *>(smem_raw + lay.spp);
    uint32_t *slmod = reinterpret_cast<uint32_t *>(sdesc + nspp);  // L_tile mod q
    uint16_t *sched = reinterpret_cast<uint16_t *>(smem_raw + lay.sched);
    uint32_t *bcache = reinterpret_cast<uint32_t *>(smem_raw + lay.bcache);
    uint32_t *bsort = reinterpret_cast<uint32_t *>(smem_raw + lay.bsort);
    // per-tile bins of the cached bucket entries: starts, and counts / write cursors
    __shared__ uint32_t s_bstart[kMaxSegTiles + 1], s_bcnt[kMaxSegTiles + 1];
    const uint32_t tile_s = (uint32_t)__cvta_generic_to_shared(tile);  // the tile's shared-window address
    // bytes of the tile region, for the bounds-checked build (BNX_GUARD)
    const uint32_t tile_bytes = (uint32_t)(lay.spp - lay.tile);
    unsigned int *const gerr = &P.ctr->err;
    // a strike at a shared-window address inside the tile
    auto red_tile = [&](uint32_t addr, uint32_t v) {
        if (BNX_GUARD(addr - tile_s <= tile_bytes - 4u, gerr)) red_add_shared(addr, v);
    };
    // the CTA's next queue segment: index, interval, interval record and bucket range
    __shared__ unsigned long long s_seg, s_b0, s_b1;
    __shared__ IvDev s_ivd;
    __shared__ uint32_t s_iv, s_nsparse;
    // dense runs of warp w: s_runs[w][0 .. s_nruns[w]), each j | first round << 8 | rounds << 20
    __shared__ uint32_t s_runs[NT / 32][kMaxRuns];
    __shared__ uint32_t s_nruns[NT / 32];

    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t nwarps = NT / 32;
    const uint32_t k = *P.n_iv;
    // (segments beyond the workspace's capacity are never planned: the bucket count flags them)
    const unsigned long long total_segs = min(P.ctr->total_segs, (unsigned long long)P.seg_cap);

    // u8 tile: the strikes of 9, 27 and 81 repeat with period 81.  Their sum at n is
    // lg(3) * #{k in 2..4 : 3^k | n}, and a tile word holds the values n .. n+3, so the word
    // is a function of n mod 81 alone (gcd(4, 81) = 1 makes every residue occur): the tile
    // is initialised from that 81-word table instead of zeros, and 9, 27, 81 leave the
    // strike schedule.
    constexpr bool kPat = VB == 1;
    // entry r': the words of residues r, r+4, r+8, r+12 for r = 16 r' mod 81, so that the
    // consecutive 16-byte stores of a warp (16 values apart) read consecutive entries
    __shared__ uint4 s_pat[kPat ? 81 : 1];
    for (uint32_t j = tid; j < nspp; j += NT) {
        const SmallPP e = P.spp[j];
        const uint32_t lg = tile_weight<VB>(e.p);
        const bool in_pat = kPat && (e.q == 9 || e.q == 27 || e.q == 81);
        // rounds: at most floor(L_tile/q)+1 multiples of q per tile; 0 = not in the schedule
        sdesc[j] = make_uint4(e.q, lg, 0u, in_pat ? 0u : (LT / e.q + 1 + 31) / 32);
        slmod[j] = LT % e.q;
    }
    if (kPat && tid < 81) {
        const uint32_t lg3 = tile_weight<VB>(3);
        uint32_t w[4] = {0, 0, 0, 0};
        for (uint32_t c = 0; c < 4; c++)
            for (uint32_t b = 0; b < 4; b++) {
                const uint32_t m = (16 * tid + 4 * c + b) % 81;
                w[c] |= lg3 * ((m % 9 == 0) + (m % 27 == 0) + (m == 0)) << (8 * b);
            }
        s_pat[tid] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    __syncthreads();
    // Static strike schedule, built once per launch.
    //  - Dense prime powers (at least two rounds of 32 multiples per tile): their rounds, in
    //    order of j, are cut into NT/32 contiguous shares of equal estimated cost (below), one
    //    per warp.  A warp's share is a list of runs (j, first round, rounds), each struck as
    //    consecutive rounds of 32 multiples, so a warp sets up each prime power it touches
    //    once per tile.
    //  - Single-round prime powers (at most 32 multiples per tile): one slot (j, m) per
    //    possible multiple m, packed 32 to a warp pass in `sched`, so that a warp pass is not
    //    spent on a handful of strikes.
    if (warp == 0) {
        constexpr int kPer = kMaxSpp / 32;
        auto slots = [&](uint32_t j) -> uint32_t {  // at most 32
            return j < nspp && sdesc[j].w == 1 ? LT / sdesc[j].x + 1 : 0u;
        };
        uint32_t sumw = 0;
        for (int u = 0; u < kPer; u++) sumw += slots(lane * kPer + u);
        uint32_t incw = sumw;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incw, o);
            if (lane >= (uint32_t)o) incw += y;
        }
        uint32_t runw = incw - sumw;
        for (int u = 0; u < kPer; u++) {
            const uint32_t j = lane * kPer + u, w = slots(j);
            for (uint32_t m = 0; m < w; m++)
                if (runw + m < P.n_sched) sched[runw + m] = (uint16_t)(j | (m << 8));
            runw += w;
        }
        if (lane == 31) {
            s_nsparse = incw <= P.n_sched ? incw : 0u;  // n_sched always covers them
            if (incw > P.n_sched && blockIdx.x == 0) atomicOr(&P.ctr->err, kErrSchedule);
        }
        // every packed slot after a warp's first pass (a dependent shared-load chain and a
        // reduction) counts against that warp's share of the dense rounds
        const uint32_t ns_all = __shfl_sync(0xffffffffu, incw <= P.n_sched ? incw : 0u, 31);
        // lane w < NT/32 lists the runs of warp w.  The shares are equal in estimated cost, not
        // in rounds: a run costs about kRunSetup instructions to set up and kRoundCost per
        // round, and the prime powers with few rounds (and so many runs) come last.  Round k of
        // a prime power whose cost span starts at cs sits at cs + kRunSetup + (k + 1/2) kRoundCost;
        // warp w takes the rounds that sit in [T w / NT*32, T (w+1) / NT*32).
        if (lane < nwarps) {
            constexpr int kRunSetup = 80, kRoundCost = 8;
            int T = 0;
            for (uint32_t j = 0; j < nspp; j++) {
                const int r = (int)sdesc[j].w;
                if (r > 1) T += kRunSetup + r * kRoundCost;
            }
            // warp w takes the rounds whose cost position lies in [B_w, B_(w+1)), B_w the running
            // maximum of (T + E) w / nwarps - (extra cost of warps below w), clamped to [0, T]:
            // contiguous, non-overlapping shares that cover [0, T) whatever the extra costs
            constexpr int kSlotPass = 40;
            auto extra = [&](uint32_t w) -> int {
                int c = 0;
                for (uint32_t p = NT + 32 * w; p < ns_all; p += NT) c++;
                return c * kSlotPass;
            };
            int E = 0;
            for (uint32_t v = 0; v < nwarps; v++) E += extra(v);
            auto bound = [&](uint32_t w) -> int {  // B_w
                int best = 0, pre = 0;
                for (uint32_t v = 0; v <= w && v <= nwarps; v++) {
                    int r = v == nwarps ? T : (int)((int64_t)(T + E) * v / nwarps) - pre;
                    r = r < 0 ? 0 : r > T ? T : r;
                    best = r > best ? r : best;
                    if (v < nwarps) pre += extra(v);
                }
                return best;
            };
            const int b = bound(lane), e = bound(lane + 1);
            auto first_at = [&](int pos, int cs, int r) -> int {  // first round k sitting at or after pos
                const int x = 2 * (pos - cs - kRunSetup) - kRoundCost;  // in half-units
                const int k = x <= 0 ? 0 : (x + 2 * kRoundCost - 1) / (2 * kRoundCost);
                return k < r ? k : r;
            };
            int cs = 0;
            uint32_t nr = 0;
            for (uint32_t j = 0; j < nspp; j++) {
                const int r = (int)sdesc[j].w;
                if (r < 2) continue;
                const int k0 = first_at(b, cs, r), k1 = first_at(e, cs, r);
                if (k0 < k1) {
                    if (nr < kMaxRuns) s_runs[lane][nr] = j | ((uint32_t)k0 << 8) | ((uint32_t)(k1 - k0) << 20);
                    nr++;
                }
                cs += kRunSetup + r * kRoundCost;
            }
            s_nruns[lane] = nr < kMaxRuns ? nr : kMaxRuns;
            if (nr > kMaxRuns) atomicOr(&P.ctr->err, kErrSchedule);
        }
    }

    // Work queue: a CTA pops its next segment while it sieves the current one (the pop's
    // latency is hidden), and looks up its interval in the segment map at the end.
    auto fetch = [&](unsigned long long sg) {  // one thread
        s_seg = sg;
        if (sg < total_segs) {
            const uint32_t i = min(P.seg_iv[sg], k - 1);
            s_iv = i;
            s_ivd = P.ivs[i];
            s_b0 = P.boff[sg];
            s_b1 = P.boff[sg + 1];
        }
    };
    if (tid == 0) fetch(atomicAdd(&P.ctr->queue_head, 1ull));
    if (tid <= kMaxSegTiles) s_bcnt[tid] = 0;
    for (;;) {
        __syncthreads();
        const unsigned long long seg = s_seg;
        if (seg >= total_segs) break;
        const uint32_t ivi = s_iv;
        const IvDev iv = s_ivd;
        const unsigned long long b0 = s_b0, b1 = s_b1;
        unsigned long long nxt = 0;
        if (tid == NT - 1) nxt = atomicAdd(&P.ctr->queue_head, 1ull);
        const uint64_t seg_lo = iv.lo + ((seg - iv.seg_base) << P.seg_log2);
        const uint64_t rem = iv.hi - seg_lo;
        const uint32_t seg_len = rem < (1ull << P.seg_log2) ? (uint32_t)rem : (1u << P.seg_log2);
        const unsigned long long ncache = P.seg_log2 <= 19 ? (unsigned long long)kLogBucketCache : 0ull;
        const uint32_t nbc = (uint32_t)((b1 - b0) < ncache ? (b1 - b0) : ncache);
        for (uint32_t j = tid; j < nspp; j += NT) {
            const uint32_t q = sdesc[j].x;
            const uint32_t r = (uint32_t)(seg_lo % q);
            sdesc[j].z = r ? q - r : 0;
        }
        const uint32_t ntl = (seg_len + LT - 1) >> tile_log2;  // tiles of this segment (<= kMaxSegTiles)
        for (uint32_t e = tid; e < nbc; e += NT) {
            if (!BNX_GUARD(b0 + e < P.bucket_cap && e < (uint32_t)kLogBucketCache, gerr)) continue;
            const uint32_t w = pack_hit<VB>(P.bent[b0 + e]);
            bcache[e] = w;
            const uint32_t o = w >> 12, t1 = o >> tile_log2;
            if (t1 < ntl) atomicAdd(&s_bcnt[t1], 1u);
            if ((o & (LT - 1)) == 0 && t1 >= 1) atomicAdd(&s_bcnt[t1 - 1], 1u);
        }
        __syncthreads();
        if (warp == 0) {  // exclusive prefix of the bin counts; the counts become write cursors
            const uint32_t i0 = 2 * lane, i1 = 2 * lane + 1;
            const uint32_t c0 = i0 < ntl ? s_bcnt[i0] : 0u, c1 = i1 < ntl ? s_bcnt[i1] : 0u;
            uint32_t inc = c0 + c1;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= (uint32_t)o) inc += y;
            }
            const uint32_t ex = inc - c0 - c1;
            if (i0 < ntl) s_bstart[i0] = s_bcnt[i0] = ex;
            if (i1 < ntl) s_bstart[i1] = s_bcnt[i1] = ex + c0;
            if (lane == 31) s_bstart[ntl] = inc;
        }
        __syncthreads();
        for (uint32_t e = tid; e < nbc; e += NT) {
            const uint32_t w = bcache[e];
            const uint32_t o = w >> 12, t1 = o >> tile_log2;
            constexpr uint32_t kBsort = kLogBucketCache + kMaxSegTiles;
            if (t1 < ntl) {
                const uint32_t at = atomicAdd(&s_bcnt[t1], 1u);
                if (BNX_GUARD(at < kBsort, gerr)) bsort[at] = w;
            }
            if ((o & (LT - 1)) == 0 && t1 >= 1) {
                const uint32_t at = atomicAdd(&s_bcnt[t1 - 1], 1u);
                if (BNX_GUARD(at < kBsort, gerr)) bsort[at] = w;
            }
        }
        const uint32_t nsparse = s_nsparse, nruns = s_nruns[warp];
        const uint32_t kinds = iv.kinds;

        for (uint32_t t0 = 0; t0 < seg_len; t0 += LT) {
            const uint32_t tl = (seg_len - t0) < LT ? (seg_len - t0) : LT;
            const uint64_t t_lo = seg_lo + t0;
            // fixed-point threshold of L(n) + L(n+1) below which n is rejected
            int64_t T;
            int lthr;  // integer log2 bound for the exact power-of-2 check
            if (MODE == kModeSearch) {
                lthr = (int)flog2_64(t_lo + 1) - 1;  // need log2 P >= log2(n+1) - 1
            } else {
                const uint64_t S2 = 2 * P.hash_S;
                const int clog = (int)flog2_64(S2) + ((S2 & (S2 - 1)) ? 1 : 0);
                lthr = (int)flog2_64(t_lo) + (int)flog2_64(t_lo + 1) - clog;  // need log2 P >= log2(n(n+1)/2S)
            }
            // n is rejected when L(n) + L(n+1) < F (lthr - (M - 2)), i.e. below its ceiling T
            const int64_t tb = (int64_t)lthr - (int64_t)(kHigh2 - 2);
            T = tb <= 0 ? tb : (tb * FN + FD - 1) / FD;
            const bool all_cand = T <= 0;
            const uint32_t T32 = all_cand ? 0u : (uint32_t)T;
            __syncthreads();
            {
                uint4 *t4 = reinterpret_cast<uint4 *>(tile);
                const uint4 z = make_uint4(0, 0, 0, 0);
                // values [0, tl] and the slack after them (the epilogue's reads past tl see only
                // zeros or values of earlier tiles; either only adds candidates, which are masked)
                const uint32_t n4 = VB == 4 ? ((tl + 4) >> 2) + 1 : ((tl >> VSH) + 8 + 3) >> 2;
                if constexpr (kPat) {
                    // word w of the tile starts at n = t_lo + 4w: store i (words 4i ..) starts at
                    // t_lo + 16 i, whose entry is r' = (t_lo + 16 i) / 16 mod 81 = 76 t_lo + i
                    // (16 * 76 = 1 mod 81).  Thread t < NS (NS the largest multiple of 81 not above
                    // NT) makes the stores i = t mod NS, which all take the same entry 76 t_lo + t
                    // mod 81: one table load per tile, then plain 16-byte stores.
                    constexpr uint32_t NS = NT / 81u * 81u;
                    if (tid < NS) {
                        const uint4 e = s_pat[(uint32_t)((t_lo * 76ull + tid) % 81ull)];
                        for (uint32_t i = tid; i < n4; i += NS)
                            if (BNX_GUARD(16u * (i + 1) <= tile_bytes, gerr)) t4[i] = e;
                    }
                } else {
                    for (uint32_t i = tid; i < n4; i += NT)
                        if (BNX_GUARD(16u * (i + 1) <= tile_bytes, gerr)) t4[i] = z;
                }
            }
            __syncthreads();
            // the first pass of packed slots (below) is loaded now and struck after the runs, so
            // that its two dependent shared loads overlap the runs
            uint32_t sa0 = 0, sv0 = 0;
            bool sp0 = false;
            {
                const uint32_t sl = warp * 32 + lane;
                if (sl < nsparse) {
                    const uint32_t e = sched[sl];
                    const uint4 d = sdesc[e & 255u];
                    const uint32_t x = d.z + (e >> 8) * d.x;
                    sp0 = x <= tl;
                    sa0 = tile_s + ((x >> VSH) << 2);
                    sv0 = d.y << ((x & (VPW - 1)) * VBITS);
                }
            }
            if (sp0) red_tile(sa0, sv0);
            // this warp's runs of dense rounds
            for (uint32_t k = 0; k < nruns; k++) {
                const uint32_t run = s_runs[warp][k];
                const uint4 d = sdesc[run & 255u];
                const uint32_t q = d.x, r0 = (run >> 8) & 0xfffu, reps = run >> 20;
                const uint32_t x = d.z + ((r0 << 5) + lane) * q;
                // 32q is a multiple of 4: x mod 4, hence the value's place in its word, is fixed
                // per lane.  The lane strikes x, x + 32q, ... up to xl, the last of its multiples
                // in this run and in the tile; in words: up to the word of the largest value
                // <= xl congruent to x mod VPW.  For VPW <= 2 that bound cannot wrap (xl = 0
                // only when x = 0); for VPW = 4 the lanes with x > xl skip the run.
                const uint32_t xl = min(tl, x + (reps - 1) * 32 * q);
                if (VPW < 4 || x <= xl) {
                    const uint32_t lg = d.y << ((x & (VPW - 1)) * VBITS);
                    uint32_t a = tile_s + ((x >> VSH) << 2);
                    const uint32_t alim = tile_s + (((xl - ((xl - x) & (VPW - 1))) >> VSH) << 2);
                    const uint32_t bstep = ((32 >> VSH) * q) << 2;
                    // rounds bounded by the lane's last address alone (no trip count), two per step
                    for (; a + bstep <= alim; a += 2 * bstep) {
                        red_tile(a, lg);
                        red_tile(a + bstep, lg);
                    }
                    if (a <= alim) red_tile(a, lg);
                }
            }
            // packed slots of the single-round prime powers
            for (uint32_t sl = warp * 32 + lane + NT; sl < ((nsparse + 31) & ~31u); sl += NT) {
                if (sl < nsparse) {
                    const uint32_t e = sched[sl];
                    const uint4 d = sdesc[e & 255u];
                    const uint32_t x = d.z + (e >> 8) * d.x;
                    if (x <= tl) red_tile(tile_s + ((x >> VSH) << 2), d.y << ((x & (VPW - 1)) * VBITS));
                }
            }
            for (uint32_t e = s_bstart[t0 >> tile_log2] + tid, e1 = s_bstart[(t0 >> tile_log2) + 1]; e < e1; e += NT) {
                const uint32_t w = bsort[e];
                const uint32_t x = (w >> 12) - t0;
                if (x <= tl) {
                    const uint32_t lg = cache_to_tile<VB>(w & 0xfffu);
                    red_tile(tile_s + ((x >> VSH) << 2), lg << ((x & (VPW - 1)) * VBITS));
                }
            }
            for (unsigned long long e = b0 + nbc + tid; e < b1; e += NT) {
                if (!BNX_GUARD(e < P.bucket_cap, gerr)) break;
                const uint2 h = P.bent[e];
                if (h.x >= t0 && h.x <= t0 + tl) {
                    const uint32_t x = h.x - t0;
                    const uint32_t lg = bucket_weight<VB>(h.y);
                    if (BNX_GUARD((x >> VSH) < tile_bytes / 4u, gerr))
                        atomicAdd(&tile[x >> VSH], lg << ((x & (VPW - 1)) * VBITS));
                }
            }
            __syncthreads();
            for (uint32_t j = tid; j < nspp; j += NT) {
                const uint32_t off = sdesc[j].z, lm = slmod[j];
                sdesc[j].z = off >= lm ? off - lm : off + sdesc[j].x - lm;
            }
            // epilogue: G n per thread (4 u32 values per 16-byte load; 16 u16 or 32 u8 values per two
            // 16-byte loads), consecutive except in the u8 tile (below)
            constexpr uint32_t M2 = 1u << kHigh2;
            constexpr uint32_t G = VB == 4 ? 4u : VB == 2 ? 16u : 32u;
            // u8 tile: a warp reads a block of 1024 values, lane l the 16-byte chunks l and 32 + l
            // (values 16 l .. 16 l + 15 and 512 + 16 l .. 512 + 16 l + 15 of the block), so that both
            // 16-byte loads of the warp are free of bank conflicts; bit u of the candidate mask is
            // value ibase + uoff(u)
            constexpr bool kSplit = VB == 1;
            const uint32_t ngroups = kSplit ? ((tl + 1023u) >> 10) << 5 : (tl + G - 1) / G;
            auto uoff = [](uint32_t u) -> uint32_t { return kSplit && u >= 16u ? u + 496u : u; };
            // offset of the first multiple of 2^M at or after t_lo (the others in the tile are at
            // sp + k 2^M)
            const uint32_t sp = (0u - (uint32_t)t_lo) & (M2 - 1);
            // the exact power of 2 of P for a candidate at tile offset i, and warp-ballot compaction
            // of those whose bound still reaches the threshold into the list of the exact check
            // (k_cand: about 2 per 2^23 integers near 2^40); the whole warp calls it
            auto consider = [&](bool has, uint32_t i) {
                bool defer = false;
                uint64_t n = 0;
                if (has) {
                    n = t_lo + i;
                    const uint32_t e2 = ctz64(n + (n & 1)) - 1;  // power of 2 in P
                    const bool in_tile = BNX_GUARD(((i + 1) >> VSH) < tile_bytes / 4u, gerr);
                    const uint32_t L0 = in_tile ? (tile[i >> VSH] >> ((i & (VPW - 1)) * VBITS)) & VMASK : 0u;
                    const uint32_t L1 = in_tile ? (tile[(i + 1) >> VSH] >> (((i + 1) & (VPW - 1)) * VBITS)) & VMASK : 0u;
                    // log2 P <= (L0 + L1) / F + e2 must reach `need`
                    const int64_t ub = (int64_t)(L0 + L1) * FD + (int64_t)e2 * FN;
                    int need;
                    if (MODE == kModeSearch) {
                        need = (int)flog2_64(n + 1) - 1;
                    } else {
                        const uint64_t S2 = 2 * P.hash_S;
                        need = (int)flog2_64(n) + (int)flog2_64(n + 1) - (int)flog2_64(S2) - ((S2 & (S2 - 1)) ? 1 : 0);
                    }
                    defer = ub >= (int64_t)need * FN;
                }
                const uint32_t m = __ballot_sync(0xffffffffu, defer);
                if (m) {
                    unsigned long long wbase = 0;
                    if (lane == 0) wbase = atomicAdd(&P.ctr->n_cand, (unsigned long long)__popc(m));
                    wbase = __shfl_sync(0xffffffffu, wbase, 0);
                    if (defer) {
                        const unsigned long long at = wbase + __popc(m & ((1u << lane) - 1));
                        if (at < P.cand_cap) {
                            Cand cd;
                            cd.n = n;
                            cd.b0 = b0;
                            cd.nb = (uint32_t)(b1 - b0);
                            cd.o = t0 + i;
                            cd.kinds = kinds;
                            cd.iv = ivi;
                            P.cand[at] = cd;
                        } else {
                            atomicOr(&P.ctr->err, kErrCandOverflow);
                        }
                    }
                }
            };
            const uint4 *t4 = reinterpret_cast<const uint4 *>(tile);
            for (uint32_t base = 0; base < ngroups; base += NT) {
                const uint32_t g = base + tid;
                const uint32_t ibase = kSplit ? ((g >> 5) << 10) + ((g & 31u) << 4) : G * g;
                uint32_t cm = 0;  // candidates among the group's n (bit u: n = t_lo + ibase + uoff(u))
                // the group's furthest read: the word after its last chunk
                const uint32_t g_end = kSplit ? ibase + 532u : VB == 4 ? 16u * g + 20u : 32u * g + 36u;
                if (g < ngroups && BNX_GUARD(g_end <= tile_bytes, gerr)) {
                    uint32_t ss[G];
                    bool logc;
                    if constexpr (VB == 4) {
                        const uint4 v = t4[g];
                        const uint32_t w = tile[4 * g + 4];
                        ss[0] = v.x + v.y;
                        ss[1] = v.y + v.z;
                        ss[2] = v.z + v.w;
                        ss[3] = v.w + w;
                        logc = max(max(ss[0], ss[1]), max(ss[2], ss[3])) >= T32;
                    } else {
                        // u8: the chunks at bytes ibase and ibase + 512, and the word after each
                        const unsigned char *tb = reinterpret_cast<const unsigned char *>(tile) + ibase;
                        const uint4 v = kSplit ? *reinterpret_cast<const uint4 *>(tb) : t4[2 * g];
                        const uint4 v2 = kSplit ? *reinterpret_cast<const uint4 *>(tb + 512) : t4[2 * g + 1];
                        const uint32_t w = kSplit ? *reinterpret_cast<const uint32_t *>(tb + 528) : tile[8 * g + 8];
                        // packed pair sums: field i of pw[k] is L(j) + L(j + 1) for the group's value j =
                        // VPW k + i (u8: j = uoff(4 k + i))
                        uint32_t pw[8];
                        pw[0] = v.x + __funnelshift_r(v.x, v.y, VBITS);
                        pw[1] = v.y + __funnelshift_r(v.y, v.z, VBITS);
                        pw[2] = v.z + __funnelshift_r(v.z, v.w, VBITS);
                        if constexpr (kSplit) {
                            pw[3] = v.w + __funnelshift_r(v.w, *reinterpret_cast<const uint32_t *>(tb + 16), VBITS);
                        } else {
                            pw[3] = v.w + __funnelshift_r(v.w, v2.x, VBITS);
                        }
                        pw[4] = v2.x + __funnelshift_r(v2.x, v2.y, VBITS);
                        pw[5] = v2.y + __funnelshift_r(v2.y, v2.z, VBITS);
                        pw[6] = v2.z + __funnelshift_r(v2.z, v2.w, VBITS);
                        pw[7] = v2.w + __funnelshift_r(v2.w, w, VBITS);
                        if constexpr (VB == 2) {
                            // a pair sum is below 2^15: adding 2^15 - T to its half-word sets bit 15
                            // exactly when the sum reaches T, and never carries into the other half
                            const uint32_t K = (0x8000u - (T32 < 0x8000u ? T32 : 0x8000u)) * 0x10001u;
                            logc = (((pw[0] + K) | (pw[1] + K) | (pw[2] + K) | (pw[3] + K) | (pw[4] + K) |
                                     (pw[5] + K) | (pw[6] + K) | (pw[7] + K)) & 0x80008000u) != 0u;
                        } else {
                            // a byte pair sum s is below 2^7: with T' = min(T, 127) and K = 128 - T',
                            // s + K stays below 2^8 and has bit 7 set exactly when s >= T' (and s >= T
                            // needs s >= T')
                            const uint32_t K = (0x80u - (T32 < 0x7fu ? T32 : 0x7fu)) * 0x01010101u;
                            uint32_t acc = 0;
#pragma unroll
                            for (uint32_t u = 0; u < 8; u++) acc |= pw[u] + K;
                            logc = (acc & 0x80808080u) != 0u;
                        }
#pragma unroll
                        for (uint32_t u = 0; u < 8; u++)
#pragma unroll
                            for (uint32_t b = 0; b < VPW; b++) ss[VPW * u + b] = (pw[u] >> (b * VBITS)) & VMASK;
                    }
                    const uint32_t n0 = (uint32_t)(t_lo + ibase);  // low 32 bits suffice modulo 2^M
                    // does [n0, n0 + G] hold a multiple of 2^M?  (u8: the n next to one are taken
                    // after the group loop)
                    const bool hi2 = !kSplit && ((n0 + G) & (M2 - 1)) <= G;
                    if (all_cand || logc) {
#pragma unroll
                        for (uint32_t u = 0; u < G; u++) {
                            const uint32_t nl = n0 + uoff(u);
                            const bool h = ((nl & (M2 - 1)) == 0) || (((nl + 1) & (M2 - 1)) == 0);
                            const bool pick = kSplit ? (all_cand || ss[u] >= T32) && !h : all_cand || ss[u] >= T32 || h;
                            if (pick && ibase + uoff(u) < tl) cm |= 1u << u;
                        }
                    } else if (hi2) {
                        // about one group per tile: only the n next to the multiple n0 + u0 of 2^M
                        // (n = n0 + u0 and n = n0 + u0 - 1), without the loop over the group
                        const uint32_t u0 = (0u - n0) & (M2 - 1);  // <= G here
                        if (u0 < G) cm |= 1u << u0;
                        if (u0 >= 1) cm |= 1u << (u0 - 1);
                        const uint32_t left = tl - G * g;  // values of the group inside the tile
                        if (left < G) cm &= (1u << left) - 1u;
                    }
                }
                while (__any_sync(0xffffffffu, cm != 0)) {
                    uint32_t i = 0;
                    const bool has = cm != 0;
                    if (has) {
                        const uint32_t u = (uint32_t)(__ffs(cm) - 1);
                        cm &= cm - 1;
                        i = ibase + uoff(u);
                    }
                    consider(has, i);
                }
            }
            if (kSplit && warp == 0) {
                // u8: the n next to a multiple of 2^M (their power of 2 may exceed 2^(M-2)), at the
                // tile offsets sp - 1, sp, sp + 2^M - 1 and sp + 2^M that lie in [0, tl)
                const uint32_t i = sp + (lane >> 1) * M2 + (lane & 1u) - 1u;
                consider(lane < 4u && i < tl, i);
            }
        }
        // every thread has read s_seg .. s_b1 and is done with the bins (a barrier of the tile
        // loop lies between)
        if (tid == NT - 1) fetch(nxt);
        if (tid <= kMaxSegTiles) s_bcnt[tid] = 0;
    }
}

// Exact check of the log tile's candidates (one thread each; they are rare): the odd
// square parts of n and n+1 by exact-division tests with the in-tile primes and by the
// segment's bucket entries, then the exact 128-bit per-kind conditions.  Survivors are
// compacted into P.surv, as the exact tile's sieve writes them.
template <int MODE>
__global__ void __launch_bounds__(256) k_cand(Plan P) {
    __shared__ SmallPrimes sprimes;
    const uint32_t tid = threadIdx.x, lane = tid & 31;
    load_small_primes(P, &sprimes);
    __syncthreads();
    const unsigned long long nc = min(P.ctr->n_cand, (unsigned long long)P.cand_cap);
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (tid & ~31u); base < nc;
         base += stride) {
        const unsigned long long c = base + lane;
        uint32_t kk = 0, iv = 0;
        uint64_t n = 0, a = 0, b = 0;
        if (c < nc) {
            const Cand cd = P.cand[c];
            n = cd.n;
            iv = cd.iv;
            const unsigned long long ge = BNX_GUARD(cd.b0 + cd.nb <= P.bucket_cap, &P.ctr->err) ? cd.b0 + cd.nb : cd.b0;
            const uint64_t s0 = sodd_exact(n, cd.o, &sprimes, P.sqrt_q, P.bent, cd.b0, ge);
            const uint64_t s1 = sodd_exact(n + 1, cd.o + 1, &sprimes, P.sqrt_q, P.bent, cd.b0, ge);
            kk = exact_kinds_log(n, s0, s1, cd.kinds, MODE, P.hash_S, &a, &b);
        }
        const uint32_t m = __ballot_sync(0xffffffffu, kk != 0);  // warp-ballot compaction
        if (m) {
            unsigned long long wbase = 0;
            if (lane == 0) wbase = atomicAdd(&P.ctr->n_surv, (unsigned long long)__popc(m));
            wbase = __shfl_sync(0xffffffffu, wbase, 0);
            if (kk) {
                const unsigned long long at = wbase + __popc(m & ((1u << lane) - 1));
                if (at < P.surv_cap) {
                    Survivor sv;
                    sv.n = n;
                    sv.a = a;
                    sv.b = b;
                    sv.kinds = kk;
                    sv.iv = iv;
                    P.surv[at] = sv;
                } else {
                    atomicOr(&P.ctr->err, kErrSurvOverflow);
                }
                if (MODE == kModeSearch) {
                    if (kk & 1) atomicAdd(&P.ctr->surv1, 1ull);
                    if (kk & 2) atomicAdd(&P.ctr->surv2, 1ull);
                }
            }
        }
    }
}

template <int MODE, int VB>
const void *log_fn_t(int threads) {
    switch (threads) {
        case 128: return (const void *)k_sieve_log<MODE, 128, VB>;
        case 256: return (const void *)k_sieve_log<MODE, 256, VB>;
        case 512: return (const void *)k_sieve_log<MODE, 512, VB>;
        default: return (const void *)k_sieve_log<MODE, 1024, VB>;
    }
}

template <int MODE>
const void *log_fn_m(int threads, int vb) {
    return vb == 1 ? log_fn_t<MODE, 1>(threads) : vb == 2 ? log_fn_t<MODE, 2>(threads) : log_fn_t<MODE, 4>(threads);
}

const void *log_fn(int mode, int threads, int vb) {
    return mode == kModeHash ? log_fn_m<kModeHash>(threads, vb) : log_fn_m<kModeSearch>(threads, vb);
}

// The weights a log tile of VB bytes per value adds for each prime of the table,
// taken along the kernel's own paths: out[4i .. 4i+4) = {p, in-tile strike weight,
// weight of a bucket hit through the shared cache (packed and unpacked as the
// sieve does), weight of a bucket hit read from global memory}.
template <int VB>
__global__ void k_log_weights(const uint32_t *primes, uint32_t np, uint32_t *out) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const uint32_t p = primes[i];
        out[4 * (size_t)i] = p;
        out[4 * (size_t)i + 1] = tile_weight<VB>(p);
        out[4 * (size_t)i + 2] = cache_to_tile<VB>(pack_hit<VB>(make_uint2(0u, p)) & 0xfffu);
        out[4 * (size_t)i + 3] = bucket_weight<VB>(p);
    }
}

}  // namespace

void launch_log_weights(const uint32_t *primes, uint32_t np, int vb, uint32_t *out, cudaStream_t s) {
    const int grid = (int)std::min<uint32_t>((np + 255) / 256 + 1, 1024u);
    if (vb == 1) k_log_weights<1><<<grid, 256, 0, s>>>(primes, np, out);
    else if (vb == 2) k_log_weights<2><<<grid, 256, 0, s>>>(primes, np, out);
    else k_log_weights<4><<<grid, 256, 0, s>>>(primes, np, out);
}

size_t sieve_log_smem_bytes(uint32_t tile_log2, uint32_t nspp, uint32_t nsched, int vb) {
    return log_layout(tile_log2, nspp, nsched, vb).total;
}

int sieve_log_occupancy(int mode, int threads, int vb, size_t smem, int *ctas_per_sm) {
    const void *fn = log_fn(mode, threads, vb);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, threads, smem);
}

void launch_cand(const Plan &P, int mode, int grid, cudaStream_t s) {
    if (mode == kModeHash) k_cand<kModeHash><<<grid, 256, 0, s>>>(P);
    else k_cand<kModeSearch><<<grid, 256, 0, s>>>(P);
}

void launch_sieve_log(const Plan &P, int mode, int vb, int grid, int threads, size_t smem, cudaStream_t s) {
    void *args[] = {(void *)&P};
    cudaLaunchKernel(log_fn(mode, threads, vb), dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace bnx
