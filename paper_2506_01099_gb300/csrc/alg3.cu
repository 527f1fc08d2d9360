// Algorithm 3 of the paper (Sec. 2.2), as the paper runs it: the quadratic
// chunked hash search, kept as a measured baseline for the CRT path.
//
// For each chunk C_i of [1, S) (s = 2^chunk_log2 values of n, plus the halo):
//   1. sieve C_i's radicals (the same shared-memory tile sieve as
//      bnx_rad_segment), reset the table, and insert every n of C_i under its
//      key {rad n, rad n+1};
//   2. probe every n of C_i: each earlier slot with the same key gives a pair
//      with both members in C_i;
//   3. for every earlier chunk C_j, j < i: sieve C_j again and probe every m of
//      it: each slot with the same key gives the pair (m, n), n in C_i.
// The table has 4s slots (the paper's 2^29 for s = 2^27), open addressing, one
// slot per n; a probe walks from the key's hash until a free slot, as the
// paper's search does.  Keys are exact: for S <= 2^32 both radicals are below
// 2^32, so key = max << 32 | min.  A pair is of the first kind when rad(m) =
// rad(n) (Algorithm 2's rule); the slot keeps n and whether rad(n) is the
// smaller radical.  Work: (S/s)^2 / 2 chunk sieves.
#include <algorithm>
#include <cstring>

#include "benelux.h"
#include "bnx_ctx.cuh"

namespace bnx {
namespace {

struct Slot {
    unsigned long long key;  // 0 = free
    unsigned long long val;  // n | (rad(n) is the smaller radical) << 63
};

__device__ __forceinline__ uint64_t mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ unsigned long long key_of(uint64_t a, uint64_t b) {
    return a < b ? ((unsigned long long)b << 32) | a : ((unsigned long long)a << 32) | b;
}

// rad[i] = rad(lo + i), i in [0, len]; n = lo + i for i < len
__global__ void k_a3_insert(const uint64_t *rad, uint64_t lo, uint32_t len, Slot *tab, uint64_t mask,
                            unsigned int *err) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        const uint64_t a = rad[i], b = rad[i + 1];
        const unsigned long long key = key_of(a, b);
        uint64_t h = mix(key) & mask;
        bool done = false;
        for (uint64_t probe = 0; probe <= mask; probe++) {
            if (atomicCAS(&tab[h].key, 0ull, key) == 0ull) {
                tab[h].val = (unsigned long long)(lo + i) | ((unsigned long long)(a < b) << 63);
                done = true;
                break;
            }
            h = (h + 1) & mask;
        }
        if (!done) atomicOr(err, 1u);
    }
}

// For every x of the probed chunk, every slot with the same key holding an n
// with x < n gives the pair (x, n) (probing the table's own chunk finds the
// pairs inside it; probing an earlier chunk, the pairs across).
__global__ void k_a3_probe(const uint64_t *rad, uint64_t lo, uint32_t len, const Slot *tab, uint64_t mask,
                           uint32_t kinds, PairDev *pairs, uint64_t cap, unsigned long long *np, unsigned int *err) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < len; i += gridDim.x * blockDim.x) {
        const uint64_t x = lo + i;
        const uint64_t a = rad[i], b = rad[i + 1];
        const unsigned long long key = key_of(a, b);
        uint64_t h = mix(key) & mask;
        for (uint64_t probe = 0; probe <= mask; probe++) {
            const unsigned long long k = tab[h].key;
            if (k == 0ull) break;  // a free slot ends the run: no later slot can hold this key
            if (k == key) {
                const unsigned long long v = tab[h].val;
                const uint64_t n = v & ~(1ull << 63);
                if (x < n) {
                    const uint64_t rn = (v >> 63) ? (a < b ? a : b) : (a < b ? b : a);
                    const uint32_t kind = rn == a ? 1u : 2u;  // rad(x) = rad(n): first kind
                    if (kinds & kind) {
                        const unsigned long long at = atomicAdd(np, 1ull);
                        if (at < cap) {
                            PairDev p;
                            p.m = x;
                            p.n = n;
                            p.kind = kind;
                            p.iv = 0;
                            pairs[at] = p;
                        } else {
                            atomicOr(err, 2u);
                        }
                    }
                }
            }
            h = (h + 1) & mask;
        }
    }
}

// rank sort of the found pairs by (n, m, kind) into `out`
__global__ void k_a3_sort(const PairDev *in, const unsigned long long *np_dev, uint64_t cap, PairDev *out) {
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

extern "C" int bnx_search_chunked(bnx_ctx *c, uint64_t S, uint32_t chunk_log2, uint32_t kinds, bnx_pair *out,
                                  size_t cap, size_t *n_out) {
    if (!c) return fail(BNX_E_ARG, "NULL context");
    if (S < 2 || S > (1ull << 32) || S >= c->max_hi) return fail(BNX_E_ARG, "need 2 <= S <= 2^32 and S < max_hi");
    if (chunk_log2 < 10 || chunk_log2 > 28) return fail(BNX_E_ARG, "chunk_log2 must be in [10, 28]");
    if (kinds < 1 || kinds > 3) return fail(BNX_E_ARG, "kinds must be 1, 2 or 3");
    if (c->server_running()) return fail(BNX_E_STATE, "the serving loop owns the context");
    std::lock_guard<std::mutex> g(c->mu);
    cudaSetDevice(c->device);
    cudaStream_t st = c->stream;
    const uint64_t s = 1ull << chunk_log2;
    const uint64_t nchunks = (S - 1 + s - 1) / s;  // n in [1, S)
    const uint64_t slots = 4 * s;
    DevBuf tab, radi, radj, pairs, sorted, misc;
    struct Guard {  // frees the call's buffers on every return path
        DevBuf *b[6];
        ~Guard() {
            for (DevBuf *x : b) release(*x);
        }
    } guard{{&tab, &radi, &radj, &pairs, &sorted, &misc}};
    uint64_t pcap = 1 << 12;
    int rc;
    if ((rc = grow(tab, sizeof(Slot) * slots)) || (rc = grow(radi, 8 * (s + 1))) || (rc = grow(radj, 8 * (s + 1))) ||
        (rc = grow(misc, 64)))
        return rc;
    unsigned long long *np_dev = (unsigned long long *)misc.p;
    unsigned int *err_dev = (unsigned int *)((char *)misc.p + 8);
    for (int attempt = 0; attempt < 3; attempt++) {
        if ((rc = grow(pairs, sizeof(PairDev) * pcap)) || (rc = grow(sorted, sizeof(PairDev) * pcap))) break;
        CUDA_TRY(cudaMemsetAsync(misc.p, 0, 64, st));
        CUDA_TRY(cudaEventRecord(c->ev0, st));
        const int grid = c->n_sm * 8;
        for (uint64_t i = 0; i < nchunks && rc == 0; i++) {
            const uint64_t lo_i = 1 + i * s, len_i = std::min(s, S - lo_i);
            if ((rc = rad_segment_unlocked(c, lo_i, len_i + 1, (uint64_t *)radi.p, nullptr, st))) break;
            CUDA_TRY(cudaMemsetAsync(tab.p, 0, sizeof(Slot) * slots, st));
            k_a3_insert<<<grid, 256, 0, st>>>((uint64_t *)radi.p, lo_i, (uint32_t)len_i, (Slot *)tab.p, slots - 1,
                                              err_dev);
            k_a3_probe<<<grid, 256, 0, st>>>((uint64_t *)radi.p, lo_i, (uint32_t)len_i, (Slot *)tab.p, slots - 1,
                                             kinds, (PairDev *)pairs.p, pcap, np_dev, err_dev);
            for (uint64_t j = 0; j < i && rc == 0; j++) {
                const uint64_t lo_j = 1 + j * s;
                if ((rc = rad_segment_unlocked(c, lo_j, s + 1, (uint64_t *)radj.p, nullptr, st))) break;
                k_a3_probe<<<grid, 256, 0, st>>>((uint64_t *)radj.p, lo_j, (uint32_t)s, (Slot *)tab.p, slots - 1,
                                                 kinds, (PairDev *)pairs.p, pcap, np_dev, err_dev);
            }
        }
        if (rc) break;
        k_a3_sort<<<c->n_sm * 2, 256, 0, st>>>((PairDev *)pairs.p, np_dev, pcap, (PairDev *)sorted.p);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(c->ev1, st));
        unsigned long long h[2] = {0, 0};
        CUDA_TRY(cudaMemcpyAsync(h, misc.p, 16, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        const unsigned long long np = h[0];
        const unsigned int err = (unsigned int)(h[1] & 0xffffffffu);
        if (err & 1u) {
            rc = fail(BNX_E_OVERFLOW, "hash table full");
            break;
        }
        if (np > pcap) {
            pcap = np + 64;
            continue;
        }
        memset(&c->stats, 0, sizeof c->stats);
        c->stats.integers = S - 1;
        c->stats.pairs = np;
        float ms = 0;
        if (cudaEventElapsedTime(&ms, c->ev0, c->ev1) == cudaSuccess) c->stats.ms_total = ms;
        cudaGetLastError();
        if (n_out) *n_out = (size_t)np;
        const size_t ncopy = std::min((size_t)np, cap);
        if (ncopy) {
            if (!out) {
                rc = fail(BNX_E_ARG, "out is NULL");
                break;
            }
            CUDA_TRY(cudaMemcpy(out, sorted.p, sizeof(PairDev) * ncopy, cudaMemcpyDeviceToHost));
        }
        rc = np > cap ? fail(BNX_E_TRUNCATED, "%llu pairs, buffer holds %zu", np, cap) : BNX_OK;
        break;
    }
    return rc;
}
