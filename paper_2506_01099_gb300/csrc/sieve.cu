// Planning, large-prime bucket fill and the shared-memory tile sieve.
//
// The n-range [lo, hi) of every interval is cut into queue segments of
// L_seg = 2^seg_log2 integers; a segment sieves the values [seg_lo, seg_lo+len]
// (len n values plus the one-integer halo that rad(n+1) of its last n needs --
// the overlap of consecutive chunks in Sec. 2.2).
//
// Per value x the tile holds s(x) = x_odd / rad(x_odd), the product of p^(e-1)
// over the odd prime powers p^e || x (the "square part"; rad(x) = x / s(x) up to
// the power of 2, which comes from counting trailing zeros as in Sec. 3.1).  It
// is Algorithm 1 (Sec. 2.1) restated multiplicatively: where Algorithm 1 divides
// r[x] by p at every multiple of p^k (k >= 2), the tile multiplies s[x] by p.
//   - prime powers q = p^k <= Q: struck inside the shared-memory tile, 32 lanes
//     of a warp on 32 consecutive multiples of one q (Sec. 3.1: once the first
//     multiple is known all strikes of a prime power are independent);
//   - prime powers q > Q: a bucket-fill pass lists each hit (value offset in its
//     segment, p) in the segment's HBM bucket; the tile applies them.
// Strikes of different prime powers may meet at one x, so every strike is a
// 64-bit shared-memory compare-and-swap multiply.
//
// The per-n filter uses exact necessary conditions (derived from the Chinese
// remainder theorem; a = rad(n), b = rad(n+1), coprime):
//   first kind : ab | n - m   ->  ab <= n - 1
//   second kind: ab | m+n+1   ->  some multiple of ab lies in [n+2, 2n]
// In terms of the square parts, ab = n(n+1) / (s(n) s(n+1)), so ab <= 2n iff
// s(n)s(n+1) >= (n+1)/2 (s including the power of 2).  A bit-length bound on
// s(n)s(n+1) rejects almost every n with a few integer instructions; the rare
// rest is decided exactly (64-bit divisions and 128-bit products).
#include "bnx_internal.cuh"

namespace bnx {

namespace {

__device__ __forceinline__ uint32_t ctz64(uint64_t x) { return (uint32_t)(__ffsll((long long)x) - 1); }
__device__ __forceinline__ uint32_t bitlen64(uint64_t x) { return 64u - (uint32_t)__clzll((long long)x); }
__device__ __forceinline__ uint32_t flog2_64(uint64_t x) { return 63u - (uint32_t)__clzll((long long)x); }

// index of the interval owning item `x`: the last v with base(v) <= x
template <bool SEG>
__device__ __forceinline__ uint32_t find_iv(const IvDev *ivs, uint32_t k, uint64_t x) {
    uint32_t lo = 0, hi = k;  // invariant: answer in [lo, hi)
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        uint64_t b = SEG ? ivs[mid].seg_base : ivs[mid].chunk_base;
        if (b <= x) lo = mid;
        else hi = mid;
    }
    return lo;
}

// ---------------------------------------------------------------- plan ----
// One block: per interval the number of queue segments (ceil((hi-lo)/L_seg))
// and of bucket-fill chunks (ceil((hi-lo+1)/2^chunk_log2)), exclusive scans of
// both, and the totals.
__global__ void k_plan(IvDev *ivs, const uint32_t *n_iv_dev, uint32_t seg_log2, uint32_t chunk_log2,
                       Counters *ctr) {
    __shared__ unsigned long long sbuf[1024], cbuf[1024];
    __shared__ unsigned long long scarry, ccarry;
    uint32_t k = *n_iv_dev;
    if (threadIdx.x == 0) scarry = ccarry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < k; base += blockDim.x) {
        uint32_t i = base + threadIdx.x;
        unsigned long long ns = 0, nc = 0;
        if (i < k) {
            uint64_t len = ivs[i].hi - ivs[i].lo;
            ns = (len + (1ull << seg_log2) - 1) >> seg_log2;
            nc = (len + 1 + (1ull << chunk_log2) - 1) >> chunk_log2;
        }
        sbuf[threadIdx.x] = ns;
        cbuf[threadIdx.x] = nc;
        __syncthreads();
        for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
            unsigned long long ts = threadIdx.x >= o ? sbuf[threadIdx.x - o] : 0;
            unsigned long long tc = threadIdx.x >= o ? cbuf[threadIdx.x - o] : 0;
            __syncthreads();
            sbuf[threadIdx.x] += ts;
            cbuf[threadIdx.x] += tc;
            __syncthreads();
        }
        if (i < k) {
            ivs[i].seg_base = scarry + sbuf[threadIdx.x] - ns;
            ivs[i].chunk_base = ccarry + cbuf[threadIdx.x] - nc;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            scarry += sbuf[blockDim.x - 1];
            ccarry += cbuf[blockDim.x - 1];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        ctr->total_segs = scarry;
        ctr->total_chunks = ccarry;
    }
}

// ------------------------------------------------------------- buckets ----
// A bucket-fill chunk is 2^kChunkSegsLog2 whole queue segments of one interval
// (the last chunk may be shorter).  One block owns a chunk: it finds every
// multiple y of every large prime power q <= the chunk's last value and
// records (y - seg_lo, p) for y's segment -- and, when y starts a segment, also
// for the previous segment as its halo value.  Counts and write cursors of the
// chunk's own segments live in shared memory; only a halo that belongs to the
// previous chunk's last segment goes through a global counter (those entries
// are written from the end of that segment's bucket, so the two writers never
// meet).  Prime powers with many multiples per chunk (at least 32, and q <= 2^20)
// are walked by a whole warp, the rest one thread each; the table is sorted by
// q, so a thread stops at the first q above the chunk.
constexpr uint32_t kChunkSegs = 1u << kChunkSegsLog2;

__device__ __forceinline__ uint64_t fast_mod(uint64_t v, uint64_t q, uint64_t m) {
    uint64_t r = v - q * __umul64hi(v, m);
    return r >= q ? r - q : r;
}

// gcur (fill only): the write cursors are the global per-segment counters (zeroed after
// the count), for launches in which several blocks share a chunk
template <bool FILL>
__device__ __forceinline__ void bucket_hit(const Plan &P, const IvDev &iv, uint64_t y, uint32_t p, uint64_t nseg,
                                           uint64_t s_first, uint32_t *hist, const unsigned long long *sbase,
                                           bool gcur) {
    const uint64_t lseg = 1ull << P.seg_log2;
    const uint64_t d = y - iv.lo;
    const uint64_t s = d >> P.seg_log2;
    const uint32_t o = (uint32_t)(d & (lseg - 1));
    // (bounds-checked build: every entry lands inside its segment's range of the array)
    unsigned int *const gerr = &P.ctr->err;
    if (FILL && gcur) {
        if (s < nseg) {
            const uint64_t seg = iv.seg_base + s;
            const unsigned long long at = P.boff[seg] + atomicAdd(&P.bcnt[seg], 1u);
            if (BNX_GUARD(at < P.boff[seg + 1] && at < P.bucket_cap, gerr)) P.bent[at] = make_uint2(o, p);
        }
        if (o == 0 && s > 0) {  // the previous segment's halo value
            const uint64_t seg = iv.seg_base + s - 1;
            const unsigned long long at = P.boff[seg] + atomicAdd(&P.bcnt[seg], 1u);
            if (BNX_GUARD(at < P.boff[seg + 1] && at < P.bucket_cap, gerr)) P.bent[at] = make_uint2((uint32_t)lseg, p);
        }
        return;
    }
    if (s < nseg) {
        const uint32_t l = (uint32_t)(s - s_first);
        const uint32_t pos = atomicAdd(&hist[l], 1u);
        if (FILL && BNX_GUARD(sbase[l] + pos < P.boff[iv.seg_base + s + 1] && sbase[l] + pos < P.bucket_cap, gerr))
            P.bent[sbase[l] + pos] = make_uint2(o, p);
    }
    if (o == 0 && s > 0) {
        if (s > s_first) {  // halo of a segment of this chunk
            const uint32_t l = (uint32_t)(s - 1 - s_first);
            const uint32_t pos = atomicAdd(&hist[l], 1u);
            if (FILL && BNX_GUARD(sbase[l] + pos < P.boff[iv.seg_base + s] && sbase[l] + pos < P.bucket_cap, gerr))
                P.bent[sbase[l] + pos] = make_uint2((uint32_t)lseg, p);
        } else {  // halo of the previous chunk's last segment: written from its end
            const uint64_t seg = iv.seg_base + s - 1;
            const uint32_t pos = atomicAdd(&P.bcnt[seg], 1u);
            if (FILL && BNX_GUARD(pos < P.boff[seg + 1] - P.boff[seg] && P.boff[seg + 1] <= P.bucket_cap, gerr))
                P.bent[P.boff[seg + 1] - 1 - pos] = make_uint2((uint32_t)lseg, p);
        }
    }
}

template <bool FILL>
__global__ void __launch_bounds__(256) k_bucket(Plan P) {
    __shared__ uint32_t s_iv;
    __shared__ uint32_t hist[kChunkSegs];
    __shared__ unsigned long long sbase[FILL ? kChunkSegs : 1];
    const uint64_t total_chunks = P.ctr->total_chunks;
    const uint32_t k = *P.n_iv;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    if (FILL && blockIdx.x == 0 && threadIdx.x == 0) P.ctr->bucket_hits = P.boff[P.ctr->total_segs];
    if (P.ctr->total_segs > P.seg_cap) {
        if (blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&P.ctr->err, kErrBucketOverflow);
        return;
    }
    if (total_chunks == 0) return;
    // A launch with few chunks (a single short search) shares each chunk among `parts`
    // blocks, each taking every parts-th prime power; the fill then writes through global
    // cursors.  With more chunks a block owns a chunk, with its cursors in shared memory.
    const uint32_t parts = total_chunks <= 8 ? max(1u, gridDim.x / (uint32_t)total_chunks) : 1u;
    const bool gcur = parts > 1;
    for (uint64_t item = blockIdx.x; item < total_chunks * parts; item += gridDim.x) {
        const uint64_t c = item / parts;
        const uint32_t part = (uint32_t)(item % parts);
        if (threadIdx.x == 0) s_iv = find_iv<false>(P.ivs, k, c);
        __syncthreads();
        const IvDev iv = P.ivs[s_iv];
        const uint64_t c_in = c - iv.chunk_base;
        const uint64_t v0 = iv.lo + (c_in << P.chunk_log2);
        uint64_t v1 = v0 + (1ull << P.chunk_log2) - 1;
        if (v1 > iv.hi) v1 = iv.hi;
        const uint64_t nseg = (iv.hi - iv.lo + (1ull << P.seg_log2) - 1) >> P.seg_log2;
        const uint64_t s_first = c_in << kChunkSegsLog2;
        const uint32_t nsc = (uint32_t)(nseg - s_first < kChunkSegs ? nseg - s_first : kChunkSegs);
        for (uint32_t i = threadIdx.x; i < kChunkSegs; i += blockDim.x) {
            hist[i] = 0;
            if (FILL && !gcur && i < nsc) sbase[i] = P.boff[iv.seg_base + s_first + i];
            if (!FILL && part == 0 && i < nsc) P.seg_iv[iv.seg_base + s_first + i] = s_iv;  // for the sieve's queue
        }
        __syncthreads();
        // dense prime powers: a warp per q, lanes on consecutive multiples
        for (uint32_t j = part * nwarps + warp; j < P.n_lpp_dense; j += nwarps * parts) {
            const LargePP e = P.lpp[j];
            if (e.q > v1) break;
            const uint64_t r = fast_mod(v0, e.q, e.m);
            for (uint64_t y = (r ? v0 + (e.q - r) : v0) + lane * e.q; y <= v1; y += 32 * e.q)
                bucket_hit<FILL>(P, iv, y, e.p, nseg, s_first, hist, sbase, gcur);
        }
        // sparse prime powers: a thread per q
        for (uint32_t j = P.n_lpp_dense + part * blockDim.x + threadIdx.x; j < P.n_lpp; j += blockDim.x * parts) {
            const LargePP e = P.lpp[j];
            if (e.q > v1) break;
            const uint64_t r = fast_mod(v0, e.q, e.m);
            for (uint64_t y = r ? v0 + (e.q - r) : v0; y <= v1; y += e.q)
                bucket_hit<FILL>(P, iv, y, e.p, nseg, s_first, hist, sbase, gcur);
        }
        __syncthreads();
        if (!FILL)
            for (uint32_t i = threadIdx.x; i < nsc; i += blockDim.x)
                if (hist[i]) atomicAdd(&P.bcnt[iv.seg_base + s_first + i], hist[i]);
        __syncthreads();
    }
}

// --------------------------------------------------------------- sieve ----
// Shared memory of one CTA (sizes from the tile length, the number of in-tile
// prime powers and the length of the static strike schedule):
//   tile    u64[L_tile + 2]   s[x] for the values t_lo .. t_lo + tl
//   bitmap  u32[L_tile/32+2]  candidate n of the tile (search and hash modes)
//   sq, sp, soff, slmod       per in-tile prime power: q, p, first multiple in
//                             the current tile, L_tile mod q
//   sched   u16[n_chunks]     static strike schedule: (prime power j, chunk c);
//                             chunk c of q covers its multiples 32c .. 32c+31
//   bcache  uint2[256]        the segment's bucket entries
constexpr int kBucketCache = 256;
constexpr uint32_t kHighTwoLog2 = 9;  // n with 2^9 | n or 2^9 | n+1 are always checked

struct SmemLayout {
    size_t tile, bitmap, spp, sched, bcache, total;
};

__host__ __device__ inline size_t align16(size_t x) { return (x + 15) & ~(size_t)15; }

__host__ __device__ inline SmemLayout smem_layout(uint32_t tile_log2, uint32_t nspp, uint32_t nsched) {
    SmemLayout L;
    L.tile = 0;
    L.bitmap = L.tile + align16((((size_t)1 << tile_log2) + 2) * sizeof(unsigned long long));
    L.spp = L.bitmap + align16((((size_t)1 << tile_log2) / 32 + 2) * sizeof(uint32_t));
    L.sched = L.spp + align16((size_t)4 * (nspp ? nspp : 1) * sizeof(uint32_t));
    L.bcache = L.sched + align16((size_t)(nsched ? nsched : 1) * sizeof(uint16_t));
    L.total = L.bcache + (size_t)kBucketCache * sizeof(uint2);
    return L;
}

// exact decision for one candidate n (s0, s1: odd square parts of n and n+1)
__device__ __noinline__ uint32_t exact_kinds(uint64_t n, uint64_t s0, uint64_t s1, uint32_t kinds, int mode,
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

// s[x] *= p.  With MARK, the strike that lifts s[x] across tau marks n = x and
// n = x - 1 as candidates (s only grows, so exactly one strike crosses).
template <bool MARK>
__device__ __forceinline__ void strike(unsigned long long *tile, uint32_t *bitmap, uint32_t x, uint32_t p,
                                       unsigned long long tau, uint32_t tl) {
    unsigned long long old = tile[x], assumed;
    do {
        assumed = old;
        old = atomicCAS(&tile[x], assumed, assumed * p);
    } while (old != assumed);
    if (MARK && assumed < tau && assumed * p >= tau) {
        if (x < tl) atomicOr(&bitmap[x >> 5], 1u << (x & 31));
        if (x > 0) atomicOr(&bitmap[(x - 1) >> 5], 1u << ((x - 1) & 31));
    }
}

template <int NT>
struct MinBlocks {
    static constexpr int value = NT <= 128 ? 8 : NT <= 256 ? 6 : NT <= 512 ? 3 : 1;
};

template <int MODE, int NT>
__global__ void __launch_bounds__(NT, MinBlocks<NT>::value) k_sieve(Plan P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr bool MARK = true;  // search and hash modes (the radicals have their own kernel, rad.cu)
    const uint32_t tile_log2 = P.tile_log2;
    const uint32_t LT = 1u << tile_log2;
    const uint32_t nspp = P.n_spp;
    const SmemLayout lay = smem_layout(tile_log2, nspp, P.n_sched);
    unsigned long long *tile = reinterpret_cast<unsigned long long *>(smem_raw + lay.tile);
    uint32_t *bitmap = reinterpret_cast<uint32_t *>(smem_raw + lay.bitmap);
    uint32_t *sq = reinterpret_cast<uint32_t *>(smem_raw + lay.spp);
    uint32_t *sp = sq + nspp;
    uint32_t *soff = sp + nspp;
    uint32_t *slmod = soff + nspp;
    uint16_t *sched = reinterpret_cast<uint16_t *>(smem_raw + lay.sched);
    uint2 *bcache = reinterpret_cast<uint2 *>(smem_raw + lay.bcache);
    __shared__ unsigned long long s_seg;
    __shared__ uint32_t s_iv, s_nsched;

    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t nwarps = NT / 32;
    const uint32_t k = *P.n_iv;
    const unsigned long long total_segs = P.ctr->total_segs;

    for (uint32_t j = tid; j < nspp; j += NT) {
        const SmallPP e = P.spp[j];
        sq[j] = e.q;
        sp[j] = e.p;
        slmod[j] = LT % e.q;
    }
    __syncthreads();
    if (warp == 0) {
        // static schedule: prime power j has at most floor(L_tile/q)+1 multiples
        // in a tile, i.e. ceil((floor(L_tile/q)+1)/32) warp-chunks
        constexpr int kPer = kMaxSpp / 32;
        uint32_t v[kPer];
        uint32_t sum = 0;
#pragma unroll
        for (int u = 0; u < kPer; u++) {
            const uint32_t j = lane * kPer + u;
            v[u] = j < nspp ? (LT / sq[j] + 1 + 31) / 32 : 0;
            sum += v[u];
        }
        uint32_t inc = sum;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += x;
        }
        uint32_t run = inc - sum;
#pragma unroll
        for (int u = 0; u < kPer; u++) {
            const uint32_t j = lane * kPer + u;
            for (uint32_t c = 0; c < v[u]; c++)
                if (run + c < P.n_sched) sched[run + c] = (uint16_t)(j | (c << 8));
            run += v[u];
        }
        if (lane == 31) s_nsched = inc < P.n_sched ? inc : P.n_sched;
    }

    for (;;) {
        __syncthreads();  // previous segment done
        if (tid == 0) {
            s_seg = atomicAdd(&P.ctr->queue_head, 1ull);
            s_iv = s_seg < total_segs ? find_iv<true>(P.ivs, k, s_seg) : 0;
        }
        __syncthreads();
        const unsigned long long seg = s_seg;
        if (seg >= total_segs) break;
        const IvDev iv = P.ivs[s_iv];
        const uint64_t seg_lo = iv.lo + ((seg - iv.seg_base) << P.seg_log2);
        const uint64_t rem = iv.hi - seg_lo;
        const uint32_t seg_len = rem < (1ull << P.seg_log2) ? (uint32_t)rem : (1u << P.seg_log2);
        const unsigned long long b0 = P.boff[seg], b1 = P.boff[seg + 1];
        const uint32_t nb_cached = (uint32_t)((b1 - b0) < (unsigned long long)kBucketCache ? (b1 - b0) : kBucketCache);
        for (uint32_t j = tid; j < nspp; j += NT) {
            const uint32_t q = sq[j];
            const uint32_t r = (uint32_t)(seg_lo % q);
            soff[j] = r ? q - r : 0;
        }
        for (uint32_t e = tid; e < nb_cached; e += NT) bcache[e] = P.bent[b0 + e];
        const uint32_t nsched = s_nsched;
        const uint32_t kinds = iv.kinds;

        for (uint32_t t0 = 0; t0 < seg_len; t0 += LT) {
            // tile: n in [t_lo, t_lo + tl); values t_lo .. t_lo + tl (the last is the halo)
            const uint32_t tl = (seg_len - t0) < LT ? (seg_len - t0) : LT;
            const uint64_t t_lo = seg_lo + t0;
            const uint32_t nwords = (tl + 31) >> 5;
            // Candidate threshold tau (uniform per tile).  An n with s(n), s(n+1)
            // < tau and 2^9 dividing neither n nor n+1 has
            // s(n)s(n+1) < tau^2 2^7 (the power of 2 included); tau is the largest
            // power of two for which that bound already fails the filter at the
            // tile's smallest n.  tau = 0: every n is a candidate.
            unsigned long long tau = ~0ull;
            if (MARK) {
                int v;
                if (MODE == kModeSearch) {
                    // need 2 s(n)s(n+1) >= n+1:  tau^2 2^8 <= t_lo + 1
                    v = (int)flog2_64(t_lo + 1) - (int)kHighTwoLog2 + 1;
                } else {
                    // need s(n)s(n+1) >= n(n+1)/(2S):  tau^2 2^7 <= t_lo(t_lo+1)/(2S)
                    const uint64_t S2 = 2 * P.hash_S;
                    const int clog = (int)flog2_64(S2) + ((S2 & (S2 - 1)) ? 1 : 0);
                    v = (int)flog2_64(t_lo) + (int)flog2_64(t_lo + 1) - clog - (int)kHighTwoLog2 + 2;
                }
                tau = v >= 2 ? (1ull << (v / 2 < 62 ? v / 2 : 62)) : 0ull;
            }
            // bit-length reject for single candidates: s(n)s(n+1) < 2^lb fails the
            // filter when lb <= thr_lb (search: 2^(lb+1) <= n+1; hash: 2^lb <= n(n+1)/(2S))
            int thr_lb = 0;
            if (MODE == kModeSearch) {
                thr_lb = (int)flog2_64(t_lo + 1) - 1;
            } else if (MODE == kModeHash) {
                const uint64_t S2 = 2 * P.hash_S;
                const int clog = (int)flog2_64(S2) + ((S2 & (S2 - 1)) ? 1 : 0);
                thr_lb = (int)flog2_64(t_lo) + (int)flog2_64(t_lo + 1) - clog;
            }
            __syncthreads();  // offsets and bucket cache ready, previous tile's epilogue done
            {
                // vectorised init: s = 1 for values 0 .. tl
                ulonglong2 *t2 = reinterpret_cast<ulonglong2 *>(tile);
                const ulonglong2 one = make_ulonglong2(1ull, 1ull);
                for (uint32_t i = tid; i <= (tl >> 1); i += NT) t2[i] = one;
                if (MARK) {
                    const uint32_t fill = tau == 0 ? ~0u : 0u;
                    for (uint32_t w = tid; w < nwords; w += NT) bitmap[w] = fill;
                }
            }
            __syncthreads();
            // small prime powers: one warp-chunk = 32 consecutive multiples of q
            for (uint32_t g = warp; g < nsched; g += nwarps) {
                const uint32_t e = sched[g];
                const uint32_t j = e & 255u;
                const uint32_t x = soff[j] + (((e >> 8) << 5) + lane) * sq[j];
                if (x <= tl) strike<MARK>(tile, bitmap, x, sp[j], tau, tl);
            }
            // large prime powers: this segment's bucket
            for (uint32_t e = tid; e < nb_cached; e += NT) {
                const uint2 h = bcache[e];
                if (h.x >= t0 && h.x <= t0 + tl) strike<MARK>(tile, bitmap, h.x - t0, h.y, tau, tl);
            }
            for (unsigned long long e = b0 + kBucketCache + tid; e < b1; e += NT) {
                const uint2 h = P.bent[e];
                if (h.x >= t0 && h.x <= t0 + tl) strike<MARK>(tile, bitmap, h.x - t0, h.y, tau, tl);
            }
            __syncthreads();
            // offsets of the next tile: (off - L_tile) mod q
            for (uint32_t j = tid; j < nspp; j += NT) {
                const uint32_t off = soff[j], lm = slmod[j];
                soff[j] = off >= lm ? off - lm : off + sq[j] - lm;
            }

            // sparse epilogue: only the marked n and the n next to a multiple of 2^9
            constexpr uint32_t M2 = 1u << kHighTwoLog2;
            for (uint32_t w0 = warp * 32; w0 < nwords; w0 += nwarps * 32) {
                const uint32_t w = w0 + lane;
                uint32_t bits = 0;
                if (w < nwords) {
                    bits = bitmap[w];
                    if (tau != 0) {
                        const uint32_t r = (uint32_t)((t_lo + 32ull * w) & (M2 - 1));
                        const uint32_t d0 = (M2 - r) & (M2 - 1);  // bit of the n with 2^9 | n
                        const uint32_t d1 = (d0 + M2 - 1) & (M2 - 1);  // bit of the n with 2^9 | n+1
                        if (d0 < 32) bits |= 1u << d0;
                        if (d1 < 32) bits |= 1u << d1;
                    }
                    const uint32_t lim = tl - 32 * w;  // >= 1
                    if (lim < 32) bits &= (1u << lim) - 1;
                }
                while (__any_sync(0xffffffffu, bits != 0)) {
                    uint32_t kk = 0;
                    uint64_t n = 0, a = 0, b = 0;
                    if (bits) {
                        const uint32_t i = 32 * w + (uint32_t)(__ffs(bits) - 1);
                        bits &= bits - 1;
                        n = t_lo + i;
                        const uint64_t s0 = tile[i], s1 = tile[i + 1];
                        // bit-length bound first: s(n)s(n+1) < 2^lb, power of 2 included
                        const int lb = (int)(bitlen64(s0) + bitlen64(s1) + ctz64(n + (n & 1))) - 1;
                        if (lb > thr_lb) kk = exact_kinds(n, s0, s1, kinds, MODE, P.hash_S, &a, &b);
                    }
                    // warp-ballot compaction: one atomic per warp
                    const uint32_t m = __ballot_sync(0xffffffffu, kk != 0);
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
                                sv.iv = s_iv;
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
        }
    }
}

template <int MODE>
const void *sieve_fn_t(int threads) {
    switch (threads) {
        case 128: return (const void *)k_sieve<MODE, 128>;
        case 256: return (const void *)k_sieve<MODE, 256>;
        case 512: return (const void *)k_sieve<MODE, 512>;
        default: return (const void *)k_sieve<MODE, 1024>;
    }
}

const void *sieve_fn(int mode, int threads) {
    if (mode == kModeHash) return sieve_fn_t<kModeHash>(threads);
    return sieve_fn_t<kModeSearch>(threads);
}

}  // namespace

// Words of the strike schedule: the exact tile needs one per round of 32
// multiples of each q; the log-domain tile needs fewer for q with several
// rounds, and floor(L/q) + 1 slots for q with a single round.
uint32_t sched_length(uint32_t tile_log2, const uint32_t *q, uint32_t nspp) {
    uint32_t n = 0;
    for (uint32_t j = 0; j < nspp; j++) {
        const uint32_t mult = ((1u << tile_log2) / q[j]) + 1, rounds = (mult + 31) / 32;
        n += rounds == 1 ? mult : rounds;
    }
    return n;
}

size_t sieve_smem_bytes(uint32_t tile_log2, uint32_t nspp, uint32_t nsched) {
    return smem_layout(tile_log2, nspp, nsched).total;
}

void launch_plan(const Plan &P, uint32_t *n_iv_dev, IvDev *ivs, uint64_t max_iv, cudaStream_t s) {
    (void)max_iv;
    k_plan<<<1, 1024, 0, s>>>(ivs, n_iv_dev, P.seg_log2, P.chunk_log2, P.ctr);
}

void launch_bucket(const Plan &P, bool fill, int grid, cudaStream_t s) {
    if (fill) k_bucket<true><<<grid, 256, 0, s>>>(P);
    else k_bucket<false><<<grid, 256, 0, s>>>(P);
}

int sieve_occupancy(int mode, int threads, size_t smem, int *ctas_per_sm) {
    const void *fn = sieve_fn(mode, threads);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, threads, smem);
}

void launch_sieve(const Plan &P, int mode, int grid, int threads, size_t smem, cudaStream_t s) {
    void *args[] = {(void *)&P};
    cudaLaunchKernel(sieve_fn(mode, threads), dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace bnx
