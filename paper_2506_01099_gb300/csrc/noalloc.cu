// bnx_rad_segment_noalloc: radicals of a segment without any device allocation.
//
// For callers that must not allocate device memory -- code whose memory is
// owned by another allocator or budget, or that runs where cudaMalloc is not
// allowed -- this entry point does the radical computation of
// bnx_rad_segment with all of its scratch in one fixed array compiled into the
// library.  It needs no context.
//
// Scratch: `g_noalloc_scratch`, a file-scope static __device__ array of
// BNX_NOALLOC_SCRATCH_BYTES.  Every GPU that loads the library holds it until
// the process exits.  It is laid out as
//   [0, kFlagBytes)             composite flags for 0 .. sqrt(max value)
//   [kSqOffset, + 8*(len))      the square part s[x] = x / rad(x) of each value
// and every call overwrites both regions before reading them (flags cleared,
// s set to 1), so nothing depends on what an earlier call left behind.  All
// calls share the one array: two calls that overlap on the GPU (different
// streams or threads without ordering between them) race and give wrong
// results.
//
// Host code must not pass the array's name to a kernel (on the host it names a
// stand-in, not device memory), so the device address is taken once per device
// with cudaGetSymbolAddress, with that device current, on the first call made
// on it.  Make that first call before any stream capture begins.  The address
// is kept per device ordinal for the life of the process: it belongs to the
// device's primary context, and after cudaDeviceReset (or under another
// context current on the device) it would be stale.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "benelux.h"
#include "bnx_ctx.cuh"

namespace bnx {
namespace {

constexpr uint64_t kNaMaxHi = BNX_NOALLOC_MAX_HI;    // largest value + 1
constexpr uint64_t kNaMaxLen = BNX_NOALLOC_MAX_LEN;  // values per call
constexpr uint64_t kNaPlim = 1ull << 20;             // sqrt(kNaMaxHi)
constexpr size_t kFlagBytes = ((kNaPlim + 1 + 255) / 256) * 256;
constexpr size_t kSqOffset = kFlagBytes;
static_assert(kSqOffset + 8 * kNaMaxLen <= BNX_NOALLOC_SCRATCH_BYTES, "scratch too small");

static __device__ __align__(256) unsigned char g_noalloc_scratch[BNX_NOALLOC_SCRATCH_BYTES];

__global__ void k_na_clear(unsigned char *flags, uint64_t plim, unsigned long long *s, uint64_t len) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i <= plim || i < len;
         i += (uint64_t)gridDim.x * blockDim.x) {
        if (i <= plim) flags[i] = 0;
        if (i < len) s[i] = 1ull;
    }
}

// sieve of Eratosthenes: block i marks the multiples of i from i*i
__global__ void k_na_mark(unsigned char *flags, uint64_t plim) {
    const uint64_t i = 2 + blockIdx.x;
    if (i * i > plim) return;
    for (uint64_t j = i * i + (uint64_t)threadIdx.x * i; j <= plim; j += (uint64_t)blockDim.x * i) flags[j] = 1;
}

// thread: one odd prime p and one of gridDim.y slices of the segment.  Every
// multiple of p^k (k >= 2) in the slice multiplies s[x] by p (Algorithm 1 with
// the division replaced by a product on the square part).
__global__ void k_na_strike(const unsigned char *flags, uint64_t plim, unsigned long long *s, uint64_t lo,
                            uint64_t len) {
    const uint64_t p = 3 + 2 * (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x);
    if (p > plim || flags[p]) return;
    const uint64_t last = lo + len - 1;
    const uint64_t slice = (len + gridDim.y - 1) / gridDim.y;
    const uint64_t a = lo + blockIdx.y * slice;
    if (a > last) return;
    const uint64_t b = a + slice - 1 < last ? a + slice - 1 : last;
    for (uint64_t q = p * p; q <= last; q *= p) {
        const uint64_t r = a % q;
        for (uint64_t y = r ? a + (q - r) : a; y <= b; y += q) {
            unsigned long long *cell = s + (y - lo);
            unsigned long long old = *cell, assumed;
            do {
                assumed = old;
                old = atomicCAS(cell, assumed, assumed * p);
            } while (old != assumed);
        }
        if (q > last / p) break;
    }
}

__global__ void k_na_finish(const unsigned long long *s, uint64_t lo, uint64_t len, uint64_t *rad_out,
                            uint64_t *sq_out) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < len; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t x = lo + i;
        const uint32_t tz = (uint32_t)(__ffsll((long long)x) - 1);
        const uint64_t sq = s[i] << (tz ? tz - 1 : 0);
        rad_out[i] = x / sq;
        if (sq_out) sq_out[i] = sq;
    }
}

std::mutex g_na_mu;
void *g_na_ptr[128];  // device address of the scratch, per device ordinal

}  // namespace
}  // namespace bnx

using namespace bnx;

extern "C" int bnx_rad_segment_noalloc(uint64_t lo, uint64_t len, uint64_t *rad_out, uint64_t *sq_out,
                                       void *stream) {
    if (!rad_out) return fail(BNX_E_ARG, "rad_out is NULL");
    // (lo > max - len, not lo + len > max: the sum could wrap)
    if (lo < 1 || len < 1 || len > kNaMaxLen || lo > kNaMaxHi - len)
        return fail(BNX_E_ARG, "need 1 <= lo, 1 <= len <= %llu and lo + len <= %llu (the fixed scratch limits)",
                    (unsigned long long)kNaMaxLen, (unsigned long long)kNaMaxHi);
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 128) return fail(BNX_E_ARG, "device ordinal %d out of range", dev);
    void *base = nullptr;
    {
        std::lock_guard<std::mutex> g(g_na_mu);
        if (!g_na_ptr[dev]) {
            void *ptr = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (e != cudaSuccess || !ptr) {
                cudaGetLastError();
                return fail(BNX_E_CUDA, "cudaGetSymbolAddress of the scratch failed: %s", cudaGetErrorString(e));
            }
            g_na_ptr[dev] = ptr;
        }
        base = g_na_ptr[dev];
    }
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *flags = static_cast<unsigned char *>(base);
    unsigned long long *sq = reinterpret_cast<unsigned long long *>(static_cast<unsigned char *>(base) + kSqOffset);
    const uint64_t last = lo + len - 1;
    uint64_t plim = (uint64_t)sqrt((double)last);  // floor(sqrt(last)), corrected below
    while (plim * plim > last) plim--;
    while ((plim + 1) * (plim + 1) <= last) plim++;
    k_na_clear<<<256, 256, 0, s>>>(flags, plim, sq, len);
    uint64_t r = 1;
    while ((r + 1) * (r + 1) <= plim) r++;
    if (r >= 2) k_na_mark<<<(unsigned)(r - 1), 256, 0, s>>>(flags, plim);
    const uint64_t nodd = plim >= 3 ? (plim - 1) / 2 : 0;
    if (nodd) {
        dim3 grid((unsigned)((nodd + 255) / 256), 16);
        k_na_strike<<<grid, 256, 0, s>>>(flags, plim, sq, lo, len);
    }
    k_na_finish<<<256, 256, 0, s>>>(sq, lo, len, rad_out, sq_out);
    CUDA_TRY(cudaGetLastError());
    return BNX_OK;
}
