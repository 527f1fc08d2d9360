// Algorithm 2 of the paper (Sec. 2.1) on the device: sort the 2-sets of every
// n < S and read the pairs off runs of equal sets.
//
//   1. radicals of [1, S] by the tile sieve (bnx_rad_segment's pipeline);
//   2. per n the exact key {rad n, rad n+1} = max << 32 | min (S <= 2^32, so
//      both radicals are below 2^32), stored as h = mix(key), a bijection of
//      64-bit words (so h(m) = h(n) exactly when the 2-sets are equal), with n
//      as the value; the same kernel counts the digits the sort will use, so
//      every pass's global digit starts are known before the sort begins;
//   3. a stable least-significant-digit radix sort of (h, n) on the top 32
//      bits of h, 4 passes of 8 bits, one kernel each (a one-sweep pass): a
//      block claims the next tile of 7168 records in order, holds them in
//      registers, counts its digits per warp, publishes its per-digit counts,
//      adds up the counts of the tiles before it (look-back over published
//      prefixes), ranks every record among the equal digits of its warp round
//      (lane masks from 8 ballots) and writes the tile out through a
//      shared-memory stage so that each digit's run goes to consecutive
//      addresses: one read and one write of each record per pass;
//   4. every pair of records with equal 64-bit h, i.e. equal 2-sets: they lie
//      in one run of equal 32-bit prefixes (at S = 2^32 a run holds one record
//      on average), found by comparing each record with those after it while
//      the prefix holds (Algorithm 2 compares only neighbours, which would lose
//      pairs in runs of three or more); the first kind when rad(m) = rad(n).
// Ordering by a bijective relabelling of the 2-sets, and by its top half only,
// leaves what Algorithm 2 needs -- every set of equal 2-sets contiguous among
// records with its prefix -- and halves the passes of a full 64-bit sort.
// Memory: about 32 S bytes (radicals, and two key and value buffers) -- the
// O(S) space that made the paper give the algorithm up beyond 2^32 fits the
// GPU's HBM at S = 2^32.
#include <algorithm>
#include <cstring>

#include "benelux.h"
#include "bnx_ctx.cuh"

namespace bnx {
namespace {

constexpr uint32_t kOsThreads = 256;  // one thread per 8-bit digit
constexpr uint32_t kOsWarps = kOsThreads / 32;
constexpr uint32_t kOsItems = 28;                          // records per thread (no spills at 2 blocks/SM)
constexpr uint32_t kOsTile = kOsThreads * kOsItems;        // 7168 records per tile
constexpr uint32_t kOsWarpItems = kOsTile / kOsWarps;      // consecutive records of one warp
constexpr size_t kOsStageBytes = (size_t)kOsTile * 12;     // staged keys and values of one tile
constexpr uint32_t kPasses = 4;
constexpr uint32_t kLowBits = 32;  // the sort orders by bits 32..63 of h
// Error bit of a look-back wait that ran out in pass p: kErrLookback << p (never expected).
// Each pass, and the pair-run kernel, return at once when an earlier pass set one: its
// output is then incomplete, and a partial prefix can leave slots unwritten, which a
// later pass would read.  Only finished kernels set the bits a kernel reads, so every
// block of it sees the same value.
constexpr unsigned kErrLookback = 16u;
constexpr unsigned kErrLookbackAll = kErrLookback * 15u;  // the bits of all four passes
constexpr uint32_t kSpinLimit = 1u << 22;

// Look-back words: (state << 59) | value, state = 1 + 2 * pass + inclusive,
// value < 2^59.  A word of another pass (or 0) reads as "not published yet",
// so the array is cleared once per call, not once per pass.
__device__ __forceinline__ unsigned long long lb_word(uint32_t pass, bool inclusive, unsigned long long v) {
    return ((unsigned long long)(1 + 2 * pass + (inclusive ? 1 : 0)) << 59) | v;
}

__device__ __forceinline__ unsigned long long ld_volatile(const unsigned long long *p) {
    return *(const volatile unsigned long long *)p;
}

__device__ __forceinline__ void st_volatile(unsigned long long *p, unsigned long long v) {
    *(volatile unsigned long long *)p = v;
}

// splitmix64's finalizer: xor-shifts and odd multipliers, each invertible, so a
// bijection of 64-bit words
__device__ __forceinline__ unsigned long long mix(unsigned long long z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint32_t digit(unsigned long long h, uint32_t pass) {
    return (uint32_t)(h >> (kLowBits + 8 * pass)) & 255u;
}

// h = mix(key), values, and the digit counts of all passes: hist[p * 256 + d]
__global__ void __launch_bounds__(256) k_a2_keys(const uint64_t *rad, uint64_t N, unsigned long long *key,
                                                 uint32_t *val, unsigned long long *hist) {
    __shared__ uint32_t h[kPasses * 256];
    for (uint32_t i = threadIdx.x; i < kPasses * 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < N; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = rad[i], b = rad[i + 1];
        const unsigned long long k = mix(a < b ? ((unsigned long long)b << 32) | a : ((unsigned long long)a << 32) | b);
        key[i] = k;
        val[i] = (uint32_t)(i + 1);  // n = i + 1 <= S - 1 < 2^32
#pragma unroll
        for (uint32_t p = 0; p < kPasses; p++) atomicAdd(&h[p * 256 + digit(k, p)], 1u);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kPasses * 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

// start[p * 256 + d] = number of keys whose pass-p digit is below d
__global__ void k_a2_starts(const unsigned long long *hist, unsigned long long *start) {
    const uint32_t p = threadIdx.x;
    if (p >= kPasses) return;
    unsigned long long run = 0;
    for (uint32_t d = 0; d < 256; d++) {
        start[p * 256 + d] = run;
        run += hist[p * 256 + d];
    }
}

// One stable pass over digit `pass` of h (bits 32 + 8 pass .. 32 + 8 pass + 7).  A
// look-back wait gives up after spin_limit polls.  withhold (a test hook, 0 in normal
// use) makes tile 0 keep its counts to itself, so that the waits on it run out: every
// index still stays in bounds (a prefix can only fall short, and the keys of pass 0
// are the real ones) and every wait ends.
template <uint32_t pass>
__global__ void __launch_bounds__(kOsThreads, 2)
    k_rs_onesweep(const unsigned long long *kin, const uint32_t *vin, unsigned long long *kout, uint32_t *vout,
                  uint64_t N, const unsigned long long *gstart, unsigned long long *look, unsigned int *tile_ctr,
                  unsigned int *err, uint32_t spin_limit, uint32_t withhold) {
    extern __shared__ unsigned long long stage[];  // kOsTile keys, then kOsTile values
    uint32_t *vstage = (uint32_t *)(stage + kOsTile);
    __shared__ uint32_t wcnt[kOsWarps][256];
    __shared__ uint32_t wsum[kOsWarps];
    __shared__ unsigned long long dst[256];
    __shared__ uint32_t s_tile;
    const uint32_t tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t lt = (1u << lane) - 1;
    __shared__ bool s_abort;
    if (tid == 0) {
        s_tile = atomicAdd(tile_ctr, 1u);  // tiles are claimed in launch order
        s_abort = pass > 0 && (*(volatile unsigned int *)err & (kErrLookback * ((1u << pass) - 1u))) != 0u;
    }
    for (uint32_t d = lane; d < 256; d += 32) wcnt[warp][d] = 0;
    __syncthreads();
    if (s_abort) return;
    const uint64_t t = s_tile;
    const uint64_t t0 = t * kOsTile;
    const uint64_t w0 = t0 + (uint64_t)warp * kOsWarpItems;
    // records of this warp: j * 32 + lane < nw
    const uint32_t nw = w0 >= N ? 0u : (N - w0 < kOsWarpItems ? (uint32_t)(N - w0) : kOsWarpItems);
    unsigned long long k[kOsItems];
    uint32_t v[kOsItems];
#pragma unroll
    for (uint32_t j = 0; j < kOsItems; j++) k[j] = j * 32 + lane < nw ? kin[w0 + j * 32 + lane] : 0ull;
#pragma unroll
    for (uint32_t j = 0; j < kOsItems; j++) v[j] = j * 32 + lane < nw ? vin[w0 + j * 32 + lane] : 0u;
    // per-warp digit counts (the order of the additions does not matter)
#pragma unroll
    for (uint32_t j = 0; j < kOsItems; j++)
        if (j * 32 + lane < nw) atomicAdd(&wcnt[warp][digit(k[j], pass)], 1u);
    __syncthreads();
    {  // thread = digit
        uint32_t tot = 0;
        for (uint32_t w = 0; w < kOsWarps; w++) tot += wcnt[w][tid];
        unsigned long long *mine = look + t * 256 + tid;
        if (!(pass == 0 && withhold && t == 0)) st_volatile(mine, lb_word(pass, t == 0, tot));
        // block-local start of the digit, then each warp's first slot
        uint32_t inc = tot;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= (uint32_t)o) inc += x;
        }
        if (lane == 31) wsum[warp] = inc;
        __syncthreads();
        uint32_t run = inc - tot;
        for (uint32_t w = 0; w < warp; w++) run += wsum[w];
        const uint32_t local = run;
        for (uint32_t w = 0; w < kOsWarps; w++) {
            const uint32_t c = wcnt[w][tid];
            wcnt[w][tid] = run;
            run += c;
        }
        // records of this digit in the tiles before this one
        unsigned long long excl = 0;
        for (uint64_t j = t; j-- > 0;) {
            const unsigned long long *p = look + j * 256 + tid;
            unsigned long long w = ld_volatile(p);
            uint32_t spins = 0;
            while ((w >> 59) == 0 || (((w >> 59) - 1) >> 1) != pass) {
                if (++spins > spin_limit) break;
                __nanosleep(64);
                w = ld_volatile(p);
            }
            if (spins > spin_limit) {  // a tile before this one never published: give up, flag it
                atomicOr(err, kErrLookback << pass);
                break;
            }
            excl += w & ((1ull << 59) - 1);
            if (((w >> 59) - 1) & 1) break;  // an inclusive prefix ends the walk
        }
        if (t > 0) st_volatile(mine, lb_word(pass, true, excl + tot));
        dst[tid] = gstart[tid] + excl - local;
    }
    __syncthreads();
    // place every record at its slot: the digit's next slot of this warp + its
    // rank among the lanes of the round with the same digit (their mask is the
    // AND of 8 ballots, one per digit bit, and of the valid lanes)
#pragma unroll
    for (uint32_t j = 0; j < kOsItems; j++) {
        const bool valid = j * 32 + lane < nw;
        const uint32_t d = digit(k[j], pass);
        uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
        for (uint32_t bit = 0; bit < 8; bit++) {
            const uint32_t m = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? m : ~m;
        }
        const uint32_t slot0 = valid ? wcnt[warp][d] : 0u;
        __syncwarp();
        if (valid) {
            const uint32_t s = slot0 + __popc(peers & lt);
            stage[s] = k[j];
            vstage[s] = v[j];
            if ((peers & lt) == 0) wcnt[warp][d] = slot0 + __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    const uint32_t nloc = t0 < N ? (uint32_t)(N - t0 < kOsTile ? N - t0 : kOsTile) : 0u;
    for (uint32_t s = tid; s < nloc; s += kOsThreads) {
        const unsigned long long key = stage[s];
        const unsigned long long pos = dst[digit(key, pass)] + s;
        kout[pos] = key;
        vout[pos] = vstage[s];
    }
}

// All pairs x < y of sorted records with equal h (equal 2-sets): equal h share
// their 32-bit prefix, so they lie in one run of equal prefixes, and the pair
// is found from x by comparing h[x] with the records after it while the prefix
// holds.  Each pair is found once, from its first record (Algorithm 2 compares
// only neighbours, which would lose pairs in runs of three or more).  A warp
// streams a contiguous chunk of 32 * 32 records, one coalesced load per round,
// eight rounds' loads (and the next round's, for the last record's neighbour) in
// flight before any is compared; the record after a lane's comes by shuffle.
constexpr uint32_t kGroupRounds = 32;
constexpr uint32_t kGroupBatch = 8;  // rounds loaded before they are compared
__device__ __forceinline__ void a2_pairs_from(uint64_t x, unsigned long long hx, unsigned long long hy,
                                              const unsigned long long *key, const uint32_t *val, uint64_t N,
                                              const uint64_t *rad, uint32_t kinds, PairDev *pairs, uint64_t cap,
                                              unsigned long long *np, unsigned int *err) {
    for (uint64_t y = x + 1; (hy >> kLowBits) == (hx >> kLowBits);) {
        if (hy == hx) {
            const uint64_t u = val[x], w = val[y];
            const uint64_t m = u < w ? u : w, n = u < w ? w : u;
            const uint32_t kind = rad[m - 1] == rad[n - 1] ? 1u : 2u;  // Algorithm 2's rule
            if (kinds & kind) {
                const unsigned long long at = atomicAdd(np, 1ull);
                if (at < cap) {
                    PairDev pr;
                    pr.m = m;
                    pr.n = n;
                    pr.kind = kind;
                    pr.iv = 0;
                    pairs[at] = pr;
                } else {
                    atomicOr(err, 2u);
                }
            }
        }
        if (++y >= N) break;
        hy = key[y];
    }
}

__global__ void k_a2_groups(const unsigned long long *key, const uint32_t *val, uint64_t N, const uint64_t *rad,
                            uint32_t kinds, PairDev *pairs, uint64_t cap, unsigned long long *np, unsigned int *err) {
    if (*(volatile unsigned int *)err & kErrLookbackAll) return;  // the sort is incomplete
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t chunk = 32ull * kGroupRounds;
    for (uint64_t c0 = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * chunk; c0 < N;
         c0 += nwarps * chunk) {
        for (uint32_t r0 = 0; r0 < kGroupRounds; r0 += kGroupBatch) {
            unsigned long long h[kGroupBatch + 1];
#pragma unroll
            for (uint32_t j = 0; j <= kGroupBatch; j++) {
                const uint64_t x = c0 + (uint64_t)(r0 + j) * 32 + lane;
                h[j] = x < N ? key[x] : 0ull;
            }
#pragma unroll
            for (uint32_t j = 0; j < kGroupBatch; j++) {
                const uint64_t x = c0 + (uint64_t)(r0 + j) * 32 + lane;
                unsigned long long hy = __shfl_down_sync(0xffffffffu, h[j], 1);
                const unsigned long long next0 = __shfl_sync(0xffffffffu, h[j + 1], 0);  // record x + 1 of lane 31
                if (lane == 31) hy = next0;
                if (x + 1 < N && (hy >> kLowBits) == (h[j] >> kLowBits))
                    a2_pairs_from(x, h[j], hy, key, val, N, rad, kinds, pairs, cap, np, err);
            }
        }
    }
}

// rank sort of the found pairs by (n, m, kind) into `out`
__global__ void k_a2_sort(const PairDev *in, const unsigned long long *np_dev, uint64_t cap, PairDev *out) {
    const unsigned long long np = *np_dev < cap ? *np_dev : cap;
    for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < np;
         i += (unsigned long long)gridDim.x * blockDim.x) {
        const PairDev me = in[i];
        unsigned long long r = 0;
        for (unsigned long long j = 0; j < np; j++) {
            const PairDev o = in[j];
            const bool less = o.n != me.n ? o.n < me.n : o.m != me.m ? o.m < me.m : o.kind < me.kind;
            const bool same = o.n == me.n && o.m == me.m && o.kind == me.kind;
            if (less || (same && j < i)) r++;
        }
        out[r] = me;
    }
}

}  // namespace
}  // namespace bnx

using namespace bnx;

extern "C" int bnx_arm_lookback_timeout(bnx_ctx *c, uint32_t spin_limit) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    if (spin_limit < 1 || spin_limit > kSpinLimit) return fail(BNX_E_ARG, "spin_limit must be in [1, 2^22]");
    std::lock_guard<std::mutex> g(c->mu);
    c->lb_spin_limit = spin_limit;
    return BNX_OK;
}

extern "C" int bnx_search_sorted(bnx_ctx *c, uint64_t S, uint32_t kinds, bnx_pair *out, size_t cap, size_t *n_out) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    if (S < 3 || S > (1ull << 32) || S >= c->max_hi) return fail(BNX_E_ARG, "need 3 <= S <= 2^32 and S < max_hi");
    if (kinds < 1 || kinds > 3) return fail(BNX_E_ARG, "kinds must be 1, 2 or 3");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    const uint64_t N = S - 1;  // n = 1 .. S-1
    const uint64_t nt = (N + kOsTile - 1) / kOsTile;
    DevBuf rad, k0, k1, v0, v1, look, misc, pairs, sorted;
    struct Guard {  // frees the call's buffers on every return path
        DevBuf *b[9];
        ~Guard() {
            for (DevBuf *x : b) release(*x);
        }
    } guard{{&rad, &k0, &k1, &v0, &v1, &look, &misc, &pairs, &sorted}};
    // misc (u64 words): [0] pair count, [1] error flags, [8 .. 12) tile
    // counters, [16 .. 16 + 2048) digit counts, then 2048 digit starts
    constexpr size_t kMiscWords = 16 + 2 * kPasses * 256;
    int rc;
    if ((rc = grow(rad, 8 * (S + 1))) || (rc = grow(k0, 8 * N)) || (rc = grow(k1, 8 * N)) || (rc = grow(v0, 4 * N)) ||
        (rc = grow(v1, 4 * N)) || (rc = grow(look, 8 * 256 * nt)) || (rc = grow(misc, 8 * kMiscWords)))
        return rc;
    unsigned long long *mw = (unsigned long long *)misc.p;
    unsigned long long *np_dev = mw;
    unsigned int *err_dev = (unsigned int *)(mw + 1);
    unsigned int *tile_ctr = (unsigned int *)(mw + 8);
    unsigned long long *hist = mw + 16, *gstart = hist + kPasses * 256;
    CUDA_TRY(cudaFuncSetAttribute(k_rs_onesweep<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOsStageBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_rs_onesweep<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOsStageBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_rs_onesweep<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOsStageBytes));
    CUDA_TRY(cudaFuncSetAttribute(k_rs_onesweep<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOsStageBytes));
    static_assert(kPasses == 4, "one instantiation per pass");
    // the look-back test hook arms one call only
    const uint32_t spin_limit = c->lb_spin_limit ? c->lb_spin_limit : kSpinLimit;
    const uint32_t withhold = c->lb_spin_limit ? 1u : 0u;
    c->lb_spin_limit = 0;
    CUDA_TRY(cudaEventRecord(c->ev0, st));
    CUDA_TRY(cudaMemsetAsync(misc.p, 0, 8 * kMiscWords, st));
    CUDA_TRY(cudaMemsetAsync(look.p, 0, 8 * 256 * nt, st));
    // radicals of [1, S] in pieces of at most 2^31 values
    for (uint64_t lo = 1; lo <= S; lo += (1ull << 31)) {
        const uint64_t len = std::min<uint64_t>(1ull << 31, S + 1 - lo);
        if ((rc = rad_segment_unlocked(c, lo, len, (uint64_t *)rad.p + (lo - 1), nullptr, st))) return rc;
    }
    const int grid = c->n_sm * 8;
    k_a2_keys<<<grid, 256, 0, st>>>((uint64_t *)rad.p, N, (unsigned long long *)k0.p, (uint32_t *)v0.p, hist);
    k_a2_starts<<<1, 32, 0, st>>>(hist, gstart);
    DevBuf *kin = &k0, *kout = &k1, *vin = &v0, *vout = &v1;
    for (uint32_t pass = 0; pass < kPasses; pass++) {
        const unsigned long long *ki = (unsigned long long *)kin->p;
        const uint32_t *vi = (uint32_t *)vin->p;
        unsigned long long *ko = (unsigned long long *)kout->p;
        uint32_t *vo = (uint32_t *)vout->p;
        const unsigned long long *gs = gstart + pass * 256;
        unsigned long long *lk = (unsigned long long *)look.p;
        unsigned int *tc = tile_ctr + pass;
        const unsigned grid_t = (unsigned)nt;
        switch (pass) {
            case 0: k_rs_onesweep<0><<<grid_t, kOsThreads, kOsStageBytes, st>>>(ki, vi, ko, vo, N, gs, lk, tc, err_dev, spin_limit, withhold); break;
            case 1: k_rs_onesweep<1><<<grid_t, kOsThreads, kOsStageBytes, st>>>(ki, vi, ko, vo, N, gs, lk, tc, err_dev, spin_limit, 0u); break;
            case 2: k_rs_onesweep<2><<<grid_t, kOsThreads, kOsStageBytes, st>>>(ki, vi, ko, vo, N, gs, lk, tc, err_dev, spin_limit, 0u); break;
            default: k_rs_onesweep<3><<<grid_t, kOsThreads, kOsStageBytes, st>>>(ki, vi, ko, vo, N, gs, lk, tc, err_dev, spin_limit, 0u); break;
        }
        std::swap(kin, kout);
        std::swap(vin, vout);
    }
    CUDA_TRY(cudaGetLastError());
    for (uint64_t pcap = 1 << 12;;) {
        if ((rc = grow(pairs, sizeof(PairDev) * pcap)) || (rc = grow(sorted, sizeof(PairDev) * pcap))) return rc;
        CUDA_TRY(cudaMemsetAsync(np_dev, 0, 8, st));
        k_a2_groups<<<grid, 256, 0, st>>>((unsigned long long *)kin->p, (uint32_t *)vin->p, N, (uint64_t *)rad.p, kinds,
                                          (PairDev *)pairs.p, pcap, np_dev, err_dev);
        k_a2_sort<<<c->n_sm * 2, 256, 0, st>>>((PairDev *)pairs.p, np_dev, pcap, (PairDev *)sorted.p);
        CUDA_TRY(cudaGetLastError());
        unsigned long long h[2] = {0, 0};
        CUDA_TRY(cudaMemcpyAsync(h, misc.p, 16, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaEventRecord(c->ev1, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if ((unsigned int)h[1] & kErrLookbackAll) return fail(BNX_E_TIMEOUT, "radix sort look-back wait ran out");
        if (h[0] > pcap) {
            pcap = h[0] + 64;
            continue;
        }
        memset(&c->stats, 0, sizeof c->stats);
        c->stats.integers = N;
        c->stats.pairs = h[0];
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->stats.ms_total = ms;
        cudaGetLastError();
        if (n_out) *n_out = (size_t)h[0];
        const size_t ncopy = std::min((size_t)h[0], cap);
        if (ncopy) {
            if (!out) return fail(BNX_E_ARG, "out is NULL");
            CUDA_TRY(cudaMemcpy(out, sorted.p, sizeof(PairDev) * ncopy, cudaMemcpyDeviceToHost));
        }
        return h[0] > cap ? fail(BNX_E_TRUNCATED, "%llu pairs, buffer holds %zu", h[0], cap) : BNX_OK;
    }
}
