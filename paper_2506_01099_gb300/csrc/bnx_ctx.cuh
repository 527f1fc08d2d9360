// The context object behind the opaque bnx_ctx handle (internal).
#pragma once
#include <atomic>
#include <new>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "benelux.h"
#include "bnx_internal.cuh"

namespace bnx {

// An NVTX range over a host stage (planning, workspace, the pipeline run, copies, a
// serving iteration, a checkpoint): visible in a timeline profiler, and next to free
// when none is attached (NVTX v3 binds to a tool only when one is loaded).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};


struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct PlanTotals {
    uint64_t segs, chunks, buckets, integers;
};

struct Server;  // server.cu

struct SieveCfg {
    bool valid = false;
    int grid = 0, occ = 0;
    uint32_t threads = 0, tile_log2 = 0, ctas = 0;
    size_t smem = 0;
};

int fail(int code, const char *fmt, ...);

// An entry point's body; a C++ exception (a failed host allocation) becomes an error code,
// so that none crosses the C ABI.
template <class F>
int guarded(F &&body) noexcept {
    try {
        return body();
    } catch (const std::bad_alloc &) {
        return fail(BNX_E_NOMEM, "host allocation failed");
    } catch (...) {
        return fail(BNX_E_STATE, "unexpected host error");
    }
}
int grow(DevBuf &b, size_t bytes);
void release(DevBuf &b);

#define CUDA_TRY(x)                                                                                         \
    do {                                                                                                    \
        cudaError_t e_ = (x);                                                                               \
        if (e_ != cudaSuccess) {                                                                            \
            cudaGetLastError();                                                                             \
            return ::bnx::fail(BNX_E_CUDA, "%s: %s (%s:%d)", #x, cudaGetErrorString(e_), __FILE__, __LINE__); \
        }                                                                                                   \
    } while (0)

}  // namespace bnx

struct bnx_ctx {
    int device = 0;
    uint64_t max_hi = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int n_sm = 0;
    bnx_tune tune{};

    // device tables
    bnx::DevBuf primes, spp, lpp, tmp_counts;
    uint32_t np = 0, n_spp = 0, n_lpp = 0;
    std::vector<uint32_t> h_spp_q; // in-tile q values (host copy)
    std::vector<uint64_t> lq;     // sorted large q (host copy)
    std::vector<double> lq_inv;   // prefix sums of 1/q over lq

    // workspace
    bnx::DevBuf ivs, n_iv, ctr, bcnt, seg_iv, boff, bent, scan_tmp, cand, surv, pairs, pairs_sorted, offsets;
    bnx::DevBuf hkeys, hheads, hnext, hslot;
    bnx::DevBuf rad_stage;  // device staging of bnx_rad_segment's results for host buffers
    size_t surv_want = 1 << 16, pair_want = 1 << 12, cand_want = 1 << 16;
    bnx::Counters *h_ctr = nullptr;  // pinned
    bnx::IvDev *h_ivs = nullptr;     // pinned staging
    size_t h_ivs_cap = 0;
    uint32_t h_nk = 0;

    // rad-mode outputs of the current call
    uint64_t *rad_out = nullptr, *sq_out = nullptr;
    uint64_t rad_lo = 0, rad_len = 0;
    // hash-mode parameters of the current call
    uint64_t hash_S = 0, hash_mask = 0;

    // graphs of the search pipeline, one per queue-segment length (2^tile_log2 .. 2^(tile_log2+6))
    static constexpr int kGraphSlots = 7;
    cudaGraphExec_t gexec[kGraphSlots] = {};
    bool graph_ok[kGraphSlots] = {};
    bool capturing = false;
    // queue-segment length of the current run (log2); 0: the tuned one
    uint32_t seg_log2_run = 0;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev_s0 = nullptr, ev_s1 = nullptr;

    uint32_t lb_spin_limit = 0;  // nonzero: the next bnx_search_sorted runs the look-back test hook
    bnx::SieveCfg sieve_cfg[12];  // per (mode, tile: exact, log u32, log u16, log u8)
    bnx_stats stats{};
    std::mutex mu;
    bnx::Server *server = nullptr;
    std::atomic<bool> serving{false};
    std::mutex stats_mu;           // guards srv_stats (written by the serving thread)
    bnx_server_stats srv_stats{};  // of the current or last serving loop

    uint32_t n_sched() const { return bnx::sched_length(tune.tile_log2, h_spp_q.data(), n_spp); }
    uint32_t seg_log2_tuned() const {
        uint32_t l = 0;
        while ((1u << l) < tune.seg_tiles) l++;
        return tune.tile_log2 + l;
    }
    uint32_t seg_log2() const { return seg_log2_run ? seg_log2_run : seg_log2_tuned(); }
    void invalidate_graphs() {
        for (bool &v : graph_ok) v = false;
    }
    uint32_t chunk_log2() const { return seg_log2() + bnx::kChunkSegsLog2; }
    bool server_running() const { return serving.load(); }
    std::vector<bnx::DevBuf *> all_bufs() {
        return {&primes, &spp,   &lpp,          &tmp_counts, &ivs,  &n_iv,  &ctr,  &bcnt,  &seg_iv, &boff,  &bent,
                &scan_tmp, &cand, &surv, &pairs, &pairs_sorted, &offsets, &hkeys, &hheads, &hnext, &hslot,
                &rad_stage};
    }
};

namespace bnx {
int build_pp_tables(bnx_ctx *c);
uint64_t bucket_bound(const bnx_ctx *c, uint64_t lo, uint64_t hi, uint64_t nseg);
int plan_host(bnx_ctx *c, const IvDev *iv, size_t k, PlanTotals *t);
int ensure_ws(bnx_ctx *c, const PlanTotals &t, size_t k, uint64_t budget = 0);
int ensure_staging(bnx_ctx *c, size_t k);                          // pinned host staging of k intervals
uint64_t ws_need_bytes(bnx_ctx *c, const PlanTotals &t, size_t k);  // bytes a run needs
uint64_t ws_footprint(bnx_ctx *c);                                   // bytes the workspace holds
Plan make_plan(const bnx_ctx *c);
int sieve_config(bnx_ctx *c, int mode, int *grid, int *threads, size_t *smem);
int record_pipeline(bnx_ctx *c, int mode, cudaStream_t s, bool timing);
int run_search(bnx_ctx *c, size_t k, bool use_graph);
int check_counters(bnx_ctx *c, bool *rerun);
void fill_stats(bnx_ctx *c, uint64_t integers);
int validate_interval(const bnx_ctx *c, uint64_t lo, uint64_t hi, uint32_t kinds);
int search_staged(bnx_ctx *c, size_t k, bnx_pair *out, size_t cap, size_t *n_out, uint64_t *offsets,
                  uint64_t budget = 0);
int rad_segment_unlocked(bnx_ctx *c, uint64_t lo, uint64_t len, uint64_t *rad_out, uint64_t *sq_out,
                         cudaStream_t s);
}  // namespace bnx
