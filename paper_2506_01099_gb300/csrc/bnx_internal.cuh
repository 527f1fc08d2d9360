// Internal declarations of libbenelux (not part of the ABI).
//
// Data layout in HBM (all device-resident for the life of a context):
//   primes      u32[np]          every prime <= sqrt(max_hi), by a device sieve
//   spp         SmallPP[n_spp]   odd prime powers q = p^k (k >= 2) with q <= Q:
//                                struck inside the shared-memory tile
//   lpp         LargePP[n_lpp]   odd prime powers q = p^k (k >= 2) with Q < q <= max_hi:
//                                their hits go through the per-segment HBM buckets
// Per pipeline run (workspace, grown on demand):
//   ivs         IvDev[k]         the intervals with their segment and chunk bases
//   bcnt/boff   u32/u64          bucket sizes and offsets per queue segment
//   seg_iv      u32              interval of each queue segment
//   bent        uint2[]          bucket entries (value offset in segment, prime)
//   cand        Cand[]           log-tile candidates left for the exact check (compacted)
//   surv        Survivor[]       n passing a necessary condition (compacted)
//   pairs       PairDev[]        verified pairs, then sorted
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bnx {

constexpr int kMaxSpp = 256;    // in-tile prime powers per context
constexpr int kMaxThreads = 1024;

// Fixed-point scale of the u32 log-domain tile: weights in units of 2^-16 bit.
constexpr uint32_t kLogFrac = 16;

// ---- log weights of the log-domain tiles, in integers only ----------------
// The log tiles add, per prime-power strike at x, a weight w(p) that must be at
// least F log2 p (F = 2^f units per bit): then their sum is an upper bound of
// F log2 of the odd square part, and rejecting n on that bound loses nothing.
// log_weight(p, f) is the smallest integer L with 2^L > p^(2^f), i.e. the bit
// length of p^(2^f) = floor(2^f log2 p) + 1 (p odd, so 2^f log2 p is never an
// integer), computed without floating point: write p = 2^e m with m in [1, 2)
// as a 62-bit fraction M / 2^62 and square it f times, rounding each square UP
// to 62 fractional bits and halving (again rounding up) when it reaches 2; k
// collects the halvings as binary digits.  By induction 2^k (M / 2^62) >=
// m^(2^i) after i squarings, so m^(2^f) < 2^(k+1) and L = e 2^f + k + 1 >
// 2^f log2 p: the weight can only over-estimate.  It equals the exact bit
// length unless some 2^i log2 m lies within the accumulated rounding (about
// 2^(i-61)) of an integer; the tests compare it with exact big-integer bit
// lengths for every prime the tables hold.  M < 2^63 throughout, so M^2 <
// 2^126 and the rounded square fits 64 bits.
__host__ __device__ inline uint32_t log_weight(uint64_t p, uint32_t f) {
    if (p < 2 || p >= (1ull << 32) || f > 16) return 0;
#ifdef __CUDA_ARCH__
    const uint32_t e = 63u - (uint32_t)__clzll((long long)p);
#else
    const uint32_t e = 63u - (uint32_t)__builtin_clzll(p);
#endif
    uint64_t M = p << (62 - e);
    uint32_t k = 0;
    for (uint32_t i = 0; i < f; i++) {
#ifdef __CUDA_ARCH__
        const uint64_t hi = __umul64hi(M, M), lo = M * M;
#else
        const unsigned __int128 sq = (unsigned __int128)M * M;
        const uint64_t hi = (uint64_t)(sq >> 64), lo = (uint64_t)sq;
#endif
        // ceil(M^2 / 2^62): the square in 62 fractional bits, rounded up
        uint64_t S = (hi << 2) | (lo >> 62);
        if (lo & ((1ull << 62) - 1)) S++;
        k <<= 1;
        if (S >> 63) {  // the square reached 2: halve it, rounding up
            S = (S >> 1) + (S & 1);
            k |= 1;
        }
        M = S;
    }
    return (e << f) + k + 1;
}

// log_weight54(p) = ceil(bitlen(p^5) / 4), the u8 tile's weight in units of 4/5
// bit: bitlen(p^5) = floor(5 log2 p) + 1 > 5 log2 p, so the weight exceeds
// (5/4) log2 p.  p^5 is computed exactly in 128 bits (2 <= p < 2^25, else 0).
__host__ __device__ inline uint32_t log_weight54(uint64_t p) {
    if (p < 2 || p >= (1ull << 25)) return 0;
    const unsigned __int128 p2 = (unsigned __int128)p * p;
    const unsigned __int128 p5 = p2 * p2 * p;  // below 2^125
    const uint64_t hi = (uint64_t)(p5 >> 64), lo = (uint64_t)p5;
#ifdef __CUDA_ARCH__
    const uint32_t bl = hi ? 128u - (uint32_t)__clzll((long long)hi) : 64u - (uint32_t)__clzll((long long)lo);
#else
    const uint32_t bl = hi ? 128u - (uint32_t)__builtin_clzll(hi) : 64u - (uint32_t)__builtin_clzll(lo);
#endif
    return (bl + 3) / 4;
}

// Weight of an in-tile strike (q = p^k <= Q) in the tile's units: VB bytes per
// tile value; units of 4/5 bit (VB = 1), 2^-8 (VB = 2) or 2^-16 (VB = 4).
template <int VB>
__host__ __device__ inline uint32_t tile_weight(uint64_t p) {
    return VB == 1 ? log_weight54(p) : log_weight(p, VB == 2 ? 8u : 16u);
}
// The 12-bit weight field of a bucket entry cached in shared memory: the u8
// tile's own weight (at most 28 for p < 2^22), else the weight in units of
// 2^-7 bit (below 2^12 for p < 2^21), scaled up by cache_to_tile.
template <int VB>
__host__ __device__ inline uint32_t cache_weight(uint64_t p) {
    return VB == 1 ? log_weight54(p) : log_weight(p, 7);
}
template <int VB>
__host__ __device__ inline uint32_t cache_to_tile(uint32_t w) {
    return VB == 1 ? w : VB == 2 ? w << 1 : w << 9;
}
// Weight of a bucket hit (a large prime power) in the tile's units, whether it
// comes from the shared cache or from global memory.
template <int VB>
__host__ __device__ inline uint32_t bucket_weight(uint64_t p) {
    return cache_to_tile<VB>(cache_weight<VB>(p));
}

struct SmallPP {
    uint32_t q;   // p^k
    uint32_t p;
    uint32_t lg;  // log_weight(p, 16): the u32 tile's weight, units of 2^-16
    uint32_t k;   // exponent
};

struct LargePP {
    uint64_t q;  // p^k
    uint64_t m;  // floor((2^64 - 1) / q): v mod q by a multiply-high and one correction
    uint32_t p;
    uint32_t pad;
};

// A bucket-fill chunk is 2^kChunkSegsLog2 whole queue segments.
constexpr uint32_t kChunkSegsLog2 = 9;

// One interval of a pipeline run.  n-range [lo, hi); sieved values [lo, hi].
struct IvDev {
    uint64_t lo, hi;
    uint32_t kinds, id;
    uint64_t seg_base;    // index of its first queue segment
    uint64_t chunk_base;  // index of its first bucket-fill chunk
};

// Survivor of the per-kind necessary conditions (or a hash-search key).
struct Survivor {
    uint64_t n, a, b;  // a = rad(n), b = rad(n+1)
    uint32_t kinds;    // bit 1: first-kind condition holds, bit 2: second-kind
    uint32_t iv;
};

// A log-tile candidate whose bound still reaches the threshold with its exact power
// of 2: the exact square parts and the per-kind conditions decide (k_cand).
struct Cand {
    uint64_t n;
    uint64_t b0;     // its segment's bucket entries: bent[b0 .. b0 + nb)
    uint32_t nb;
    uint32_t o;      // offset of n in its segment
    uint32_t kinds;  // the interval's kinds
    uint32_t iv;
};

struct PairDev {
    uint64_t m, n;
    uint32_t kind, iv;
};

// Device counters of one run (zeroed at its start).
struct Counters {
    unsigned long long queue_head;   // next queue segment to pop
    unsigned long long n_surv;       // survivors written (may exceed capacity)
    unsigned long long n_pairs;      // pairs written (may exceed capacity)
    unsigned long long bucket_hits;
    unsigned long long surv1, surv2, candidates, hash_keys;
    unsigned long long n_cand;       // log-tile candidates written (may exceed capacity)
    unsigned long long total_segs, total_chunks;  // plan totals
    unsigned int err;                // nonzero: a device-side limit was hit
    unsigned int pad;
};

// Error bits in Counters::err.
constexpr unsigned kErrSurvOverflow = 1u;
constexpr unsigned kErrPairOverflow = 2u;
constexpr unsigned kErrBucketOverflow = 4u;
constexpr unsigned kErrHashFull = 8u;
constexpr unsigned kErrSchedule = 32u;  // a strike schedule did not fit its array (never expected)
constexpr unsigned kErrCandOverflow = 64u;
constexpr unsigned kErrBounds = 256u;  // bounds-checked build: an index fell outside its buffer

// Bounds checks of the tile and bucket indices.  Built with -DBNX_CHECK_BOUNDS (the
// checked library of build.py), BNX_GUARD(cond, err) is cond, and a false cond sets
// kErrBounds in *err: the access it guards is skipped and the run fails with an error,
// nothing traps.  In the normal build it is true, and the guarded access runs
// unconditionally.
#ifdef BNX_CHECK_BOUNDS
__device__ __forceinline__ bool bnx_guard(bool ok, unsigned int *err) {
    if (!ok) atomicOr(err, kErrBounds);
    return ok;
}
#define BNX_GUARD(cond, err) bnx_guard((cond), (err))
#else
#define BNX_GUARD(cond, err) true
#endif

// Everything a pipeline's kernels read.  Passed by value to every launch; the
// sizes that vary per run live in device memory (Counters, IvDev) so that one
// captured graph serves every batch that fits the workspace.
struct Plan {
    const IvDev *ivs;
    const uint32_t *n_iv;  // device: number of intervals in this run
    const SmallPP *spp;
    uint32_t n_spp;
    uint32_t n_sched;  // length of the static strike schedule
    uint32_t sqrt_q;   // floor(sqrt(Q)): primes above it reach the tile only through buckets
    const LargePP *lpp;  // sorted by q
    uint32_t n_lpp;
    uint32_t n_lpp_dense;  // entries with q <= min(2^(chunk_log2 - 5), 2^20): walked by a whole warp
    uint32_t tile_log2, seg_log2;  // tile 2^tile_log2 integers, queue segment 2^seg_log2
    uint32_t chunk_log2;           // bucket-fill chunk: 2^chunk_log2 sieved values
    uint32_t *bcnt;                // [seg capacity]
    uint32_t *seg_iv;              // [seg capacity] interval of each queue segment (written by the bucket count)
    unsigned long long *boff;      // [seg capacity + 1]
    uint2 *bent;                   // [bucket capacity]
    uint64_t seg_cap, bucket_cap;
    Counters *ctr;
    Survivor *surv;
    uint64_t surv_cap;
    Cand *cand;
    uint64_t cand_cap;
    PairDev *pairs;
    PairDev *pairs_sorted;
    uint64_t pair_cap;
    uint64_t *iv_offsets;  // [k+1] pair offsets per interval
    // rad mode
    uint64_t *rad_out, *sq_out;
    uint64_t rad_lo, rad_len;
    // hash mode
    uint64_t hash_S;
    unsigned long long *hkeys;  // [hash slots], 0 = empty
    uint32_t *hheads;           // [hash slots], 0xffffffff = empty chain
    uint32_t *hnext;            // [surv cap]
    uint32_t *hslot;            // [surv cap]
    uint64_t hash_mask;
};

enum SieveMode { kModeSearch = 0, kModeRad = 1, kModeHash = 2 };
// which tile the search and hash modes use
enum TileKind { kTileLog32 = 0, kTileExact = 1, kTileLog16 = 2, kTileLog8 = 3 };

// ---------------------------------------------------------------- kernels --
// tables.cu
void launch_prime_sieve(uint8_t *comp, uint64_t lim, cudaStream_t s);
uint32_t flags_blocks(uint64_t n);
void launch_scan_u8_count(const uint8_t *flags, uint64_t n, uint32_t *block_sums, uint32_t nblocks, cudaStream_t s);
void launch_compact_primes(const uint8_t *comp, uint64_t lim, const uint32_t *block_offsets, uint32_t *primes,
                           uint32_t nblocks, cudaStream_t s);
void launch_exclusive_scan_u32(const uint32_t *in, unsigned long long *out, const unsigned long long *n_dev,
                               uint64_t n_cap, unsigned long long *tmp, uint32_t tmp_cap, cudaStream_t s);
void launch_build_pp(const uint32_t *primes, uint32_t np, uint64_t max_hi, uint32_t q_small, SmallPP *spp,
                     uint32_t *n_spp, LargePP *lpp, uint32_t *n_lpp, uint64_t lpp_cap, uint32_t *scratch,
                     cudaStream_t s);
// sort lpp[0 .. n_pow2) by q (entries beyond the table hold q = 2^64 - 1)
void launch_sort_lpp(LargePP *lpp, uint32_t n_valid, uint32_t n_pow2, cudaStream_t s);

// sieve.cu
void launch_plan(const Plan &P, uint32_t *n_iv_dev, IvDev *ivs, uint64_t max_iv, cudaStream_t s);
void launch_bucket(const Plan &P, bool fill, int grid, cudaStream_t s);
void launch_sieve(const Plan &P, int mode, int grid, int threads, size_t smem, cudaStream_t s);
int sieve_occupancy(int mode, int threads, size_t smem, int *ctas_per_sm);
// rad.cu: exact radicals (rad mode)
void launch_rad(const Plan &P, int grid, int threads, size_t smem, cudaStream_t s);
int rad_occupancy(int threads, size_t smem, int *ctas_per_sm);
size_t rad_smem_bytes(uint32_t tile_log2, uint32_t nspp, uint32_t nsched);
// sieve_log.cu: log-domain tile for the search and hash modes
// vb: bytes per tile value (4, 2 or 1)
void launch_sieve_log(const Plan &P, int mode, int vb, int grid, int threads, size_t smem, cudaStream_t s);
int sieve_log_occupancy(int mode, int threads, int vb, size_t smem, int *ctas_per_sm);
// exact check of the log tile's candidates: survivors into P.surv
void launch_cand(const Plan &P, int mode, int grid, cudaStream_t s);
size_t sieve_log_smem_bytes(uint32_t tile_log2, uint32_t nspp, uint32_t nsched, int vb);
// the weights each prime of the table gets in the log tile of vb bytes per value (4 u32 each)
void launch_log_weights(const uint32_t *primes, uint32_t np, int vb, uint32_t *out, cudaStream_t s);
size_t sieve_smem_bytes(uint32_t tile_log2, uint32_t nspp, uint32_t nsched);
uint32_t sched_length(uint32_t tile_log2, const uint32_t *q, uint32_t nspp);

// verify.cu
void launch_verify(const Plan &P, int grid, cudaStream_t s);
// out[i] = (rad(x[i]) == rad(y[i])), by k_verify's gcd strips
void launch_same_rad(const uint64_t *x, const uint64_t *y, uint64_t n, uint8_t *out, cudaStream_t s);
void launch_sort(const Plan &P, int grid, cudaStream_t s);
void launch_offsets(const Plan &P, int grid, cudaStream_t s);
void launch_hash_insert(const Plan &P, int grid, cudaStream_t s);
void launch_hash_pairs(const Plan &P, uint32_t kinds, int grid, cudaStream_t s);
void launch_zero_counters(Counters *c, cudaStream_t s);

}  // namespace bnx
