// Device-resident tables of a context and a device exclusive scan.
//
// Sec. 3.1 of the paper sends "the list of primes to be used in the sieving
// process" to the GPU once; here the list is made on the GPU itself:
//   1. a sieve of Eratosthenes over [0, lim] marks composites (one block per
//      candidate factor i <= sqrt(lim), its threads striding the multiples);
//   2. per-block counts, a scan and a compaction give the ascending prime list;
//   3. one thread lists the odd prime powers p^k (k >= 2): those <= Q go to the
//      in-tile table, the larger ones (<= max_hi) to the bucket table.
#include "bnx_internal.cuh"

namespace bnx {

namespace {

constexpr int kFlagsPerBlock = 4096;

__global__ void k_mark_composites(uint8_t *comp, uint64_t lim) {
    uint64_t i = 2 + blockIdx.x;
    if (i * i > lim) return;
    for (uint64_t j = i * i + (uint64_t)threadIdx.x * i; j <= lim; j += (uint64_t)blockDim.x * i) comp[j] = 1;
}

// count of primes (comp == 0, index >= 2) in each block of kFlagsPerBlock flags
__global__ void k_count_flags(const uint8_t *comp, uint64_t n, uint32_t *block_sums) {
    __shared__ uint32_t warp_sums[32];
    uint64_t base = (uint64_t)blockIdx.x * kFlagsPerBlock;
    uint32_t c = 0;
    for (uint32_t k = threadIdx.x; k < kFlagsPerBlock; k += blockDim.x) {
        uint64_t x = base + k;
        if (x >= 2 && x < n && comp[x] == 0) c++;
    }
    for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x < 32) {
        uint32_t v = threadIdx.x < (blockDim.x >> 5) ? warp_sums[threadIdx.x] : 0;
        for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) block_sums[blockIdx.x] = v;
    }
}

// in-place exclusive scan of a short u32 array by one block
__global__ void k_scan_small(uint32_t *a, uint32_t n, uint32_t *total) {
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    __shared__ uint32_t buf[1024];
    for (uint32_t base = 0; base < n; base += blockDim.x) {
        uint32_t i = base + threadIdx.x;
        uint32_t v = i < n ? a[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
            uint32_t t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < n) a[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += buf[blockDim.x - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

// write the primes of each block at its scanned offset, in ascending order
__global__ void k_compact_primes(const uint8_t *comp, uint64_t n, const uint32_t *block_off, uint32_t *primes) {
    // one warp walks the block's flags 32 at a time, ballot-compacting
    if (threadIdx.x >= 32) return;
    uint64_t base = (uint64_t)blockIdx.x * kFlagsPerBlock;
    uint32_t out = block_off[blockIdx.x];
    for (uint32_t k = 0; k < kFlagsPerBlock; k += 32) {
        uint64_t x = base + k + threadIdx.x;
        bool is_p = x >= 2 && x < n && comp[x] == 0;
        uint32_t m = __ballot_sync(0xffffffffu, is_p);
        if (is_p) primes[out + __popc(m & ((1u << threadIdx.x) - 1))] = (uint32_t)x;
        out += __popc(m);
    }
}

// The odd prime powers q = p^k, k >= 2, q <= max_hi: those <= q_small go to the
// in-tile table (ordered by p, then k; at most kMaxSpp entries), the larger ones
// to the bucket table.  One thread per prime counts its powers of each class;
// exclusive scans of the counts give every prime its output positions; a second
// pass writes the entries.
__device__ __forceinline__ void pp_counts(uint64_t p, uint64_t max_hi, uint32_t q_small, uint32_t *ns, uint32_t *nl) {
    *ns = 0;
    *nl = 0;
    if (p == 2 || p * p > max_hi) return;  // the prime 2 is handled by counting trailing zeros
    for (uint64_t q = p * p;; q *= p) {
        if (q <= q_small) (*ns)++;
        else (*nl)++;
        if (q > max_hi / p) break;
    }
}

__global__ void k_pp_count(const uint32_t *primes, uint32_t np, uint64_t max_hi, uint32_t q_small, uint32_t *cs,
                           uint32_t *cl) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x)
        pp_counts(primes[i], max_hi, q_small, &cs[i], &cl[i]);
}

__global__ void k_pp_write(const uint32_t *primes, uint32_t np, uint64_t max_hi, uint32_t q_small,
                           const uint32_t *os, const uint32_t *ol, SmallPP *spp, LargePP *lpp, uint64_t lpp_cap) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < np; i += gridDim.x * blockDim.x) {
        const uint64_t p = primes[i];
        if (p == 2 || p * p > max_hi) continue;
        const uint32_t lg = log_weight(p, kLogFrac);
        uint32_t si = os[i], li = ol[i], e = 2;
        for (uint64_t q = p * p;; q *= p, e++) {
            if (q <= q_small) {
                if (si < kMaxSpp) {
                    spp[si].q = (uint32_t)q;
                    spp[si].p = (uint32_t)p;
                    spp[si].lg = lg;
                    spp[si].k = e;
                }
                si++;
            } else {
                if (li < lpp_cap) {
                    lpp[li].q = q;
                    lpp[li].m = ~0ull / q;
                    lpp[li].p = (uint32_t)p;
                    lpp[li].pad = 0;
                }
                li++;
            }
            if (q > max_hi / p) break;
        }
    }
}

// ---- bitonic sort of the large prime-power table by q (once per context) ----
__global__ void k_pad_lpp(LargePP *lpp, uint32_t n_valid, uint32_t n_pow2) {
    for (uint32_t i = n_valid + blockIdx.x * blockDim.x + threadIdx.x; i < n_pow2; i += gridDim.x * blockDim.x) {
        lpp[i].q = ~0ull;
        lpp[i].m = 1;
        lpp[i].p = 0;
        lpp[i].pad = 0;
    }
}

__global__ void k_bitonic_step(LargePP *a, uint32_t n, uint32_t j, uint32_t k) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t l = i ^ j;
        if (l > i) {
            const LargePP x = a[i], y = a[l];
            const bool up = (i & k) == 0;
            if ((x.q > y.q) == up) {
                a[i] = y;
                a[l] = x;
            }
        }
    }
}

// ---- exclusive scan u32 -> u64 with the element count in device memory ----
constexpr int kScanTile = 4096;

__global__ void k_scan_reduce(const uint32_t *in, const unsigned long long *n_dev, unsigned long long *tile_sums) {
    __shared__ unsigned long long warp_sums[32];
    uint64_t n = *n_dev;
    uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t base = t * kScanTile;
        unsigned long long c = 0;
        for (uint32_t k = threadIdx.x; k < kScanTile; k += blockDim.x)
            if (base + k < n) c += in[base + k];
        for (int o = 16; o; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
        if ((threadIdx.x & 31) == 0) warp_sums[threadIdx.x >> 5] = c;
        __syncthreads();
        if (threadIdx.x < 32) {
            unsigned long long v = threadIdx.x < (blockDim.x >> 5) ? warp_sums[threadIdx.x] : 0;
            for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            if (threadIdx.x == 0) tile_sums[t] = v;
        }
        __syncthreads();
    }
}

__global__ void k_scan_tiles(unsigned long long *tile_sums, const unsigned long long *n_dev) {
    __shared__ unsigned long long buf[1024];
    __shared__ unsigned long long carry;
    uint64_t n = *n_dev;
    uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint64_t base = 0; base < ntiles; base += blockDim.x) {
        uint64_t i = base + threadIdx.x;
        unsigned long long v = i < ntiles ? tile_sums[i] : 0;
        buf[threadIdx.x] = v;
        __syncthreads();
        for (uint32_t o = 1; o < blockDim.x; o <<= 1) {
            unsigned long long t = threadIdx.x >= o ? buf[threadIdx.x - o] : 0;
            __syncthreads();
            buf[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < ntiles) tile_sums[i] = carry + buf[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 0) carry += buf[blockDim.x - 1];
        __syncthreads();
    }
}

// out[i] = tile offset + exclusive prefix inside the tile; out[n] = total
__global__ void k_scan_down(const uint32_t *in, unsigned long long *out, const unsigned long long *n_dev,
                            const unsigned long long *tile_sums) {
    __shared__ unsigned long long warp_tot[32];
    uint64_t n = *n_dev;
    uint64_t ntiles = (n + kScanTile - 1) / kScanTile;
    const uint32_t per = kScanTile / blockDim.x;  // consecutive elements per thread
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
        uint64_t base = t * kScanTile + (uint64_t)threadIdx.x * per;
        unsigned long long local = 0;
        for (uint32_t k = 0; k < per; k++)
            if (base + k < n) local += in[base + k];
        // inclusive warp scan of the per-thread sums
        unsigned long long inc = local;
        for (int o = 1; o < 32; o <<= 1) {
            unsigned long long v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) warp_tot[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            unsigned long long w = lane < nwarps ? warp_tot[lane] : 0;
            unsigned long long wi = w;
            for (int o = 1; o < 32; o <<= 1) {
                unsigned long long v = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += v;
            }
            if (lane < nwarps) warp_tot[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long run = tile_sums[t] + warp_tot[warp] + inc - local;
        for (uint32_t k = 0; k < per; k++) {
            if (base + k < n) {
                out[base + k] = run;
                run += in[base + k];
            }
        }
        // the thread holding element n-1 also writes the total
        if (n > 0 && base <= n - 1 && n - 1 < base + per) out[n] = run;
        __syncthreads();
    }
    if (n == 0 && blockIdx.x == 0 && threadIdx.x == 0) out[0] = 0;
}

}  // namespace

void launch_prime_sieve(uint8_t *comp, uint64_t lim, cudaStream_t s) {
    uint64_t r = 1;
    while ((r + 1) * (r + 1) <= lim) r++;
    if (r >= 2) k_mark_composites<<<(unsigned)(r - 1), 256, 0, s>>>(comp, lim);
}

void launch_scan_u8_count(const uint8_t *flags, uint64_t n, uint32_t *block_sums, uint32_t nblocks, cudaStream_t s) {
    k_count_flags<<<nblocks, 256, 0, s>>>(flags, n, block_sums);
    k_scan_small<<<1, 1024, 0, s>>>(block_sums, nblocks, block_sums + nblocks);
}

void launch_compact_primes(const uint8_t *comp, uint64_t lim, const uint32_t *block_offsets, uint32_t *primes,
                           uint32_t nblocks, cudaStream_t s) {
    k_compact_primes<<<nblocks, 32, 0, s>>>(comp, lim + 1, block_offsets, primes);
}

void launch_build_pp(const uint32_t *primes, uint32_t np, uint64_t max_hi, uint32_t q_small, SmallPP *spp,
                     uint32_t *n_spp, LargePP *lpp, uint32_t *n_lpp, uint64_t lpp_cap, uint32_t *scratch,
                     cudaStream_t s) {
    // scratch: 4 * (np + 1) u32 -- counts and offsets of both classes
    uint32_t *cs = scratch, *cl = scratch + (np + 1), *os = scratch + 2 * (np + 1), *ol = scratch + 3 * (np + 1);
    const int grid = (int)((np + 255) / 256 < 1024 ? (np + 255) / 256 + 1 : 1024);
    k_pp_count<<<grid, 256, 0, s>>>(primes, np, max_hi, q_small, cs, cl);
    cudaMemcpyAsync(os, cs, sizeof(uint32_t) * np, cudaMemcpyDeviceToDevice, s);
    cudaMemcpyAsync(ol, cl, sizeof(uint32_t) * np, cudaMemcpyDeviceToDevice, s);
    k_scan_small<<<1, 1024, 0, s>>>(os, np, n_spp);
    k_scan_small<<<1, 1024, 0, s>>>(ol, np, n_lpp);
    k_pp_write<<<grid, 256, 0, s>>>(primes, np, max_hi, q_small, os, ol, spp, lpp, lpp_cap);
}

void launch_exclusive_scan_u32(const uint32_t *in, unsigned long long *out, const unsigned long long *n_dev,
                               uint64_t n_cap, unsigned long long *tmp, uint32_t tmp_cap, cudaStream_t s) {
    (void)tmp_cap;
    uint64_t tiles = (n_cap + kScanTile - 1) / kScanTile;
    int grid = (int)(tiles < 2048 ? (tiles ? tiles : 1) : 2048);
    k_scan_reduce<<<grid, 256, 0, s>>>(in, n_dev, tmp);
    k_scan_tiles<<<1, 1024, 0, s>>>(tmp, n_dev);
    k_scan_down<<<grid, 256, 0, s>>>(in, out, n_dev, tmp);
}

uint32_t flags_blocks(uint64_t n) { return (uint32_t)((n + kFlagsPerBlock - 1) / kFlagsPerBlock); }

void launch_sort_lpp(LargePP *lpp, uint32_t n_valid, uint32_t n_pow2, cudaStream_t s) {
    const int grid = (int)((n_pow2 + 255) / 256 < 4096 ? (n_pow2 + 255) / 256 : 4096);
    k_pad_lpp<<<grid, 256, 0, s>>>(lpp, n_valid, n_pow2);
    for (uint32_t k = 2; k <= n_pow2; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) k_bitonic_step<<<grid, 256, 0, s>>>(lpp, n_pow2, j, k);
}

}  // namespace bnx
