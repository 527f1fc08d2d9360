// Exact radicals of queue segments: bnx_rad_segment's kernel (and the radical
// arrays of the sort-based and chunked searches).
//
// Algorithm 1 (Sec. 2.1) divides r[x] by p at every multiple of p^k (k >= 2);
// here, per shared-memory tile, the odd square part s(x) = prod p^(e-1) over the
// odd p^e || x (e >= 2) is built up multiplicatively instead, and at the end
// rad(x) = x / (2^(t-1) s(x)) for x = 2^t x_odd (t >= 1; x itself when t = 0):
//   - the tile holds s(x) in 32 bits per value (2^14 values in 64 KB, so three
//     CTAs of 256 threads share an SM);
//   - the strikes of 9, 27 and 81 multiply s(x) by 3^#{k in 2..4 : 3^k | x}, a
//     function of x mod 81 alone: the tile is initialised from an 81-entry table
//     of 16-byte words (four consecutive values) instead of with ones, and those
//     three prime powers leave the strike schedule;
//   - every other prime power q = p^k <= Q strikes s(x) *= p at its multiples
//     (32 lanes of a warp on 32 consecutive multiples), and the segment's bucket
//     entries do the same for the larger ones; strikes of different prime powers
//     may meet at one x, so a strike is a 32-bit compare-and-swap multiply;
//   - a product that would pass 2^32 is replaced by 0, which stays 0 under later
//     strikes: such values (square part above 2^32, rare) get their square part
//     recomputed exactly from the segment's tables (bnx_exact.cuh);
//   - rad(x_odd) = x_odd / s(x) is taken as x_odd * s(x)^-1 mod 2^64, exact
//     because s(x) | x_odd: the inverse comes from a table for s(x) < 256 (all
//     but about 0.25% of values) and from Newton's iteration otherwise.
// The outputs are written coalesced, 8 bytes per value and array.
#include "bnx_exact.cuh"
#include "bnx_internal.cuh"

namespace bnx {
namespace {

constexpr int kRadBucketCache = 256;

struct RadLayout {
    size_t tile, spp, sched, bcache, total;
};

__host__ __device__ inline size_t ral16(size_t x) { return (x + 15) & ~(size_t)15; }

// tile: u32 values 0 .. L_tile plus slack for the 16-byte initialisation stores
__host__ __device__ inline RadLayout rad_layout(uint32_t tile_log2, uint32_t nspp, uint32_t nsched) {
    RadLayout L;
    L.tile = 0;
    L.spp = ral16((((size_t)1 << tile_log2) + 8) * sizeof(uint32_t));
    L.sched = L.spp + ral16((size_t)4 * (nspp ? nspp : 1) * sizeof(uint32_t));
    L.bcache = L.sched + ral16((size_t)(nsched ? nsched : 1) * sizeof(uint16_t));
    L.total = L.bcache + (size_t)kRadBucketCache * sizeof(uint2);
    return L;
}

// s[x] *= p, or 0 once the product would pass 2^32 (and 0 stays 0)
__device__ __forceinline__ void strike32(uint32_t *tile, uint32_t x, uint32_t p) {
    uint32_t old = tile[x], assumed;
    do {
        assumed = old;
        const unsigned long long v = (unsigned long long)assumed * p;
        old = atomicCAS(&tile[x], assumed, v >> 32 ? 0u : (uint32_t)v);
    } while (old != assumed);
}

// s^-1 mod 2^64 for odd s (s s = 1 mod 8, so s is right to 3 bits; each Newton step
// doubles the correct low bits: 3 -> 6 -> 12 -> 24 -> 48 -> 96)
__device__ __forceinline__ uint64_t inv64(uint64_t s) {
    uint32_t i32 = (uint32_t)s;
    const uint32_t s32 = (uint32_t)s;
    i32 *= 2u - s32 * i32;
    i32 *= 2u - s32 * i32;
    i32 *= 2u - s32 * i32;
    uint64_t i = i32;  // right to 24 bits
    i *= 2ull - s * i;
    i *= 2ull - s * i;
    return i;
}

template <int NT>
__global__ void __launch_bounds__(NT, NT <= 256 ? 3 : 1) k_rad(Plan P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const uint32_t tile_log2 = P.tile_log2;
    const uint32_t LT = 1u << tile_log2;
    const uint32_t nspp = P.n_spp;
    const RadLayout lay = rad_layout(tile_log2, nspp, P.n_sched);
    uint32_t *tile = reinterpret_cast<uint32_t *>(smem_raw + lay.tile);
    // words of the tile region and the error word, for the bounds-checked build (BNX_GUARD)
    const uint32_t tile_words = (uint32_t)((lay.spp - lay.tile) / sizeof(uint32_t));
    unsigned int *const gerr = &P.ctr->err;
    uint32_t *sq = reinterpret_cast<uint32_t *>(smem_raw + lay.spp);
    uint32_t *sp = sq + nspp;
    uint32_t *soff = sp + nspp;   // first multiple of q in the current tile
    uint32_t *slmod = soff + nspp;  // L_tile mod q
    uint16_t *sched = reinterpret_cast<uint16_t *>(smem_raw + lay.sched);
    uint2 *bcache = reinterpret_cast<uint2 *>(smem_raw + lay.bcache);
    __shared__ uint4 s_pat[81];  // entry r: 3^#{k in 2..4 : 3^k | x} for x = r, r+1, r+2, r+3 mod 81
    __shared__ unsigned long long s_inv[128];  // (2t + 1)^-1 mod 2^64
    __shared__ SmallPrimes sprimes;
    __shared__ unsigned long long s_seg;
    __shared__ uint32_t s_iv, s_nsched;

    const uint32_t tid = threadIdx.x;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    constexpr uint32_t nwarps = NT / 32;
    const uint32_t k = *P.n_iv;
    const unsigned long long total_segs = min(P.ctr->total_segs, (unsigned long long)P.seg_cap);
    const bool pair_ok = ((reinterpret_cast<uintptr_t>(P.rad_out) | reinterpret_cast<uintptr_t>(P.sq_out)) & 15u) == 0;

    for (uint32_t j = tid; j < nspp; j += NT) {
        const SmallPP e = P.spp[j];
        sq[j] = e.q;
        sp[j] = e.p;
        slmod[j] = LT % e.q;
    }
    for (uint32_t r = tid; r < 81; r += NT) {
        uint32_t w[4];
        for (uint32_t b = 0; b < 4; b++) {
            const uint32_t m = (r + b) % 81;
            w[b] = (m % 9 == 0 ? 3u : 1u) * (m % 27 == 0 ? 3u : 1u) * (m == 0 ? 3u : 1u);
        }
        s_pat[r] = make_uint4(w[0], w[1], w[2], w[3]);
    }
    for (uint32_t t = tid; t < 128; t += NT) s_inv[t] = inv64(2ull * t + 1);
    load_small_primes(P, &sprimes);
    __syncthreads();
    if (warp == 0) {
        // static schedule of warp-chunks (prime power j, chunk c): chunk c covers the
        // multiples 32c .. 32c+31 of q in a tile (at most floor(L_tile/q) + 1 of them);
        // 9, 27 and 81 come with the initialisation
        constexpr int kPer = kMaxSpp / 32;
        uint32_t v[kPer];
        uint32_t sum = 0;
#pragma unroll
        for (int u = 0; u < kPer; u++) {
            const uint32_t j = lane * kPer + u;
            const bool pat = j < nspp && (sq[j] == 9 || sq[j] == 27 || sq[j] == 81);
            v[u] = j < nspp && !pat ? (LT / sq[j] + 1 + 31) / 32 : 0;
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
            const unsigned long long sg = atomicAdd(&P.ctr->queue_head, 1ull);
            s_seg = sg;
            if (sg < total_segs) s_iv = min(P.seg_iv[sg], k - 1);
        }
        __syncthreads();
        const unsigned long long seg = s_seg;
        if (seg >= total_segs) break;
        const IvDev iv = P.ivs[s_iv];
        const uint64_t seg_lo = iv.lo + ((seg - iv.seg_base) << P.seg_log2);
        const uint64_t rem = iv.hi - seg_lo;
        const uint32_t seg_len = rem < (1ull << P.seg_log2) ? (uint32_t)rem : (1u << P.seg_log2);
        const unsigned long long b0 = P.boff[seg], b1 = P.boff[seg + 1];
        const uint32_t nbc = (uint32_t)((b1 - b0) < (unsigned long long)kRadBucketCache ? (b1 - b0) : kRadBucketCache);
        for (uint32_t j = tid; j < nspp; j += NT) {
            const uint32_t q = sq[j];
            const uint32_t r = (uint32_t)(seg_lo % q);
            soff[j] = r ? q - r : 0;
        }
        for (uint32_t e = tid; e < nbc; e += NT)
            if (BNX_GUARD(b0 + e < P.bucket_cap && e < (uint32_t)kRadBucketCache, gerr)) bcache[e] = P.bent[b0 + e];
        const uint32_t nsched = s_nsched;

        for (uint32_t t0 = 0; t0 < seg_len; t0 += LT) {
            // tile: values t_lo .. t_lo + tl (the last is the segment's halo)
            const uint32_t tl = (seg_len - t0) < LT ? (seg_len - t0) : LT;
            const uint64_t t_lo = seg_lo + t0;
            __syncthreads();  // offsets and bucket cache ready, previous tile written out
            {
                // 16-byte store i holds the values t_lo + 4i .. t_lo + 4i + 3, entry (t_lo + 4i)
                // mod 81; thread t < NS (the largest multiple of 81 not above NT) makes the
                // stores i = t mod NS, which all take the same entry (4 NS = 0 mod 81)
                constexpr uint32_t NS = NT / 81u * 81u;
                uint4 *t4 = reinterpret_cast<uint4 *>(tile);
                const uint32_t n4 = (tl >> 2) + 1;  // values 0 .. tl
                if (tid < NS) {
                    const uint4 e = s_pat[(uint32_t)((t_lo + 4ull * tid) % 81ull)];
                    for (uint32_t i = tid; i < n4; i += NS) t4[i] = e;
                }
            }
            __syncthreads();
            // in-tile prime powers: one warp-chunk = 32 consecutive multiples of q
            for (uint32_t g = warp; g < nsched; g += nwarps) {
                const uint32_t e = sched[g];
                const uint32_t j = e & 255u;
                const uint32_t x = soff[j] + (((e >> 8) << 5) + lane) * sq[j];
                if (x <= tl && BNX_GUARD(x < tile_words, gerr)) strike32(tile, x, sp[j]);
            }
            // large prime powers: this segment's bucket
            for (uint32_t e = tid; e < nbc; e += NT) {
                const uint2 h = bcache[e];
                if (h.x >= t0 && h.x <= t0 + tl && BNX_GUARD(h.x - t0 < tile_words, gerr)) strike32(tile, h.x - t0, h.y);
            }
            for (unsigned long long e = b0 + kRadBucketCache + tid; e < b1; e += NT) {
                if (!BNX_GUARD(e < P.bucket_cap, gerr)) break;
                const uint2 h = P.bent[e];
                if (h.x >= t0 && h.x <= t0 + tl && BNX_GUARD(h.x - t0 < tile_words, gerr)) strike32(tile, h.x - t0, h.y);
            }
            __syncthreads();
            // offsets of the next tile: (off - L_tile) mod q
            for (uint32_t j = tid; j < nspp; j += NT) {
                const uint32_t off = soff[j], lm = slmod[j];
                soff[j] = off >= lm ? off - lm : off + sq[j] - lm;
            }
            // the values of this tile (not its halo): rad and the square part
            auto finish = [&](uint32_t i, uint32_t s32, uint64_t *r, uint64_t *q) {  // value t_lo + i, tile[i]
                const uint64_t x = t_lo + i;
                const uint32_t tz = (uint32_t)(__ffsll((long long)x) - 1);
                const uint64_t xo = x >> tz;
                uint64_t so = s32;
                if (so == 0 && BNX_GUARD(b1 <= P.bucket_cap, gerr))
                    so = sodd_exact(x, t0 + i, &sprimes, P.sqrt_q, P.bent, b0, b1);  // past 2^32
                uint64_t inv;
                if (so < 256) inv = s_inv[so >> 1];
                else inv = inv64(so);
                const uint64_t ro = xo * inv;  // = x_odd / s, exactly
                *r = tz ? ro << 1 : ro;
                *q = so << (tz ? tz - 1 : 0);
            };
            // pairs of values with one 16-byte store per output: the output index of value
            // t_lo + i is t_lo - rad_lo + i, and t_lo - rad_lo is even (segments and tiles
            // start at even offsets), so an even i starts a 16-byte aligned pair when the
            // outputs are 16-byte aligned; otherwise (and for a ragged end) one value at a time
            const uint64_t g0 = t_lo - P.rad_lo;
            const bool vec = pair_ok && g0 < P.rad_len && (g0 & 1) == 0;
            const uint32_t tv = vec ? (uint32_t)min((uint64_t)tl, P.rad_len - g0) & ~1u : 0u;
            for (uint32_t i = 2 * tid; i < tv; i += 2 * NT) {
                uint64_t r0, q0, r1, q1;
                if (!BNX_GUARD(i + 1 < tile_words, gerr)) continue;
                const uint2 s2 = *reinterpret_cast<const uint2 *>(tile + i);  // i even: 8-byte aligned
                finish(i, s2.x, &r0, &q0);
                finish(i + 1, s2.y, &r1, &q1);
                *reinterpret_cast<ulonglong2 *>(P.rad_out + g0 + i) = make_ulonglong2(r0, r1);
                if (P.sq_out) *reinterpret_cast<ulonglong2 *>(P.sq_out + g0 + i) = make_ulonglong2(q0, q1);
            }
            for (uint32_t i = tv + tid; i < tl; i += NT) {
                const uint64_t gi = t_lo + i - P.rad_lo;
                if (gi < P.rad_len) {
                    uint64_t r, q;
                    if (BNX_GUARD(i < tile_words, gerr)) finish(i, tile[i], &r, &q);
                    else r = q = 0;
                    P.rad_out[gi] = r;
                    if (P.sq_out) P.sq_out[gi] = q;
                }
            }
        }
    }
}

const void *rad_fn(int threads) {
    switch (threads) {
        case 128: return (const void *)k_rad<128>;
        case 256: return (const void *)k_rad<256>;
        case 512: return (const void *)k_rad<512>;
        default: return (const void *)k_rad<1024>;
    }
}

}  // namespace

size_t rad_smem_bytes(uint32_t tile_log2, uint32_t nspp, uint32_t nsched) {
    return rad_layout(tile_log2, nspp, nsched).total;
}

int rad_occupancy(int threads, size_t smem, int *ctas_per_sm) {
    const void *fn = rad_fn(threads);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return (int)e;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, fn, threads, smem);
}

void launch_rad(const Plan &P, int grid, int threads, size_t smem, cudaStream_t s) {
    void *args[] = {(void *)&P};
    cudaLaunchKernel(rad_fn(threads), dim3(grid), dim3(threads), args, smem, s);
}

}  // namespace bnx
