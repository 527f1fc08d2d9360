"""Benchmark: integers searched per second for Benelux pairs near n = 2^40.

Workload (one step): the batched configuration -- 4096 seeded intervals,
lengths log-uniform in [2^16, 2^30], starts uniform in [2^32, 2^40), kind 1 or
2 -- searched by one batched pipeline (bucket fill, one persistent sieve launch
over the device segment queue, verification, device sort), replayed from a
CUDA graph.  The same intervals are also searched by the plain path (one
bnx_search per interval), the large window [2^40, 2^40 + 2^37) is run plain
(one call) and batched (128 x 2^30), and a seeded Poisson request stream is
served with continuous batching for p50/p99 latency.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank searches its own 4096 intervals (seed + rank),
no collective on the data path (weak scaling); value = all ranks' integers / max time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2506_01099_gb300 import workloads as W  # noqa: E402

METRIC = "integers searched/s at n~2^40, batched (4096 seeded intervals in [2^32, 2^40))"
UNIT = "integers/s"
MAX_HI = (1 << 41) + (1 << 31)
TUNE_CACHE = os.path.join(ROOT, "paper_2506_01099_gb300", "tune_cache.json")
KERNELS_PER_STEP = 11  # plan, bucket count, 3 scan kernels, bucket fill, sieve, exact check, verify, sort, offsets
# Algorithmic integer lane-operations per searched integer of each tile kind (the method as
# built; the ALU roofline divides them by the device's SM count x 128 lanes x the maximum SM clock).
# Strikes: sum over odd prime powers q = p^k, k >= 2, of 1/q
# = sum_{p>=3} 1/(p(p-1)) = 0.2732 per integer, each an address step, a bound test and a
# shared-memory reduction (3 ops).  Log tiles: the pair test of a word of VPW values is a
# funnel shift, the pair add, the threshold add and the flag OR (4 ops per word; the u8 tile,
# whose pair sums stay below 2^7, adds pair and threshold in one 3-input add: 3 ops), plus a
# 16-byte load and a 16-byte clear per 16 bytes of tile.  The exact u64 tile: clear 1, strikes
# as 64-bit multiplies (5 ops), 2-adic valuation 2, key and filter 10.
STRIKE_OPS = 0.2732 * 3
ALG_OPS_PER_INT = {3: STRIKE_OPS + 3 / 4 + 2 / 16,     # u8: 4 values per word, 16 per 16 bytes
                   2: STRIKE_OPS + 4 / 2 + 2 / 8,      # u16
                   0: STRIKE_OPS + 4 / 1 + 2 / 4,      # u32
                   1: 1 + 0.2732 * 5 + 2 + 10}         # exact u64 tile
LANES_PER_CLK, SCHEDULERS, SM_MAX_MHZ = 128, 4, 2070.0  # per SM: 4 schedulers x 32 lanes


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return d, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "sm_max_mhz": SM_MAX_MHZ}, "fallback"


class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.idx)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for name, v in zip(names, p[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def code_sha256(path: str) -> str:
    """sha256 of a CUDA source without its // comments and blank lines, so that a record
    of counters stays valid across comment edits and is dropped by any change of code."""
    import hashlib
    import re

    lines = []
    for ln in open(path, encoding="utf-8").read().splitlines():
        ln = re.sub(r"//.*$", "", ln).rstrip()
        if ln.strip():
            lines.append(ln)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()


def sieve_record(tile_kind: int):
    """The committed ncu record (DRAM bytes and warp instructions per integer) of the sieve
    with this tile kind -- or None once the kernel's code differs from the one it measured."""
    import glob

    rec = None
    for f in glob.glob(os.path.join(ROOT, "profiles", "k_sieve_log_*_traffic.json")):
        try:
            r = json.load(open(f))
        except Exception:
            continue
        if r.get("tile_kind") == tile_kind:
            rec = r
    if rec is None:
        return None
    try:
        h = code_sha256(os.path.join(ROOT, rec["source"]))
    except Exception:
        return None
    if h != rec.get("code_sha256"):
        return None
    return rec


def load_tune(gpu_name: str) -> str | None:
    try:
        with open(TUNE_CACHE) as fh:
            cache = json.load(fh)
    except Exception:
        return None
    key = f"{gpu_name}|{MAX_HI.bit_length() - 1}"
    t = cache.get(key)
    return json.dumps(t) if t else None


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        from datetime import timedelta

        import torch.distributed as dist

        # a rank that is lost (its process gone between steps) ends the others' next
        # collective with an error after this long, instead of a hang
        timeout = timedelta(seconds=float(os.environ.get("BNX_BENCH_PG_TIMEOUT_S", "600")))
        dist.init_process_group("nccl" if os.environ.get("BNX_BENCH_BACKEND") != "gloo" else "gloo",
                                timeout=timeout)
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def _reduce(ws, x: float, op: str) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def max_over_ranks(ws, x: float) -> float:
    """Slowest rank's time: the job's time."""
    return _reduce(ws, x, "max")


def sum_over_ranks(ws, x: float) -> float:
    return _reduce(ws, x, "sum")


def rank_intervals(rank: int, count: int = 4096):
    """Each rank's own batch: the batched workload drawn with seed + rank (no
    interval is shared, no data moves between ranks)."""
    return W.batch_intervals(count, seed=(3 ^ W.SEED_SALT) + rank)


# ---------------------------------------------------------------------------
# CPU baseline: the oracle as it stands, on a bounded sample of the workload
# ---------------------------------------------------------------------------

def oracle_sample(intervals, budget_integers: int):
    """Leading pieces of the workload's intervals, clipped to budget_integers in total."""
    out, tot = [], 0
    for iv in intervals:
        take = min(iv.hi - iv.lo, budget_integers - tot)
        if take <= 0:
            break
        out.append(W.Interval(iv.lo, iv.lo + take, iv.kinds, iv.id))
        tot += take
    return out, tot


def host_cores() -> int:
    """Cores this process may run on (torchrun sets OMP_NUM_THREADS=1, so the oracle is
    given this thread count explicitly)."""
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def cpu_baseline(intervals, budget_integers: int):
    import oracle

    orc = oracle.load()
    sample, tot = oracle_sample(intervals, budget_integers)
    orc.lib.orc_init(2 * max(iv.hi for iv in sample) + 2)
    cores = host_cores()
    t0 = time.perf_counter()
    npairs = 0
    for iv in sample:
        npairs += len(orc.pairs_crt(iv.lo, iv.hi, iv.kinds, nthreads=cores))
    dt = time.perf_counter() - t0
    return {"value": tot / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {tot} integers of the batched workload ({len(sample)} leading interval pieces), "
                      f"{dt:.1f} s, CRT enumeration over Algorithm 1 radicals, OpenMP over 2^20-integer chunks",
            "seconds": dt, "pairs": npairs}


def cpu_full_ranges():
    """The oracle on the two full-range searches, all n < 2^24 and all n < 2^32
    (both kinds), on the host cores: the CPU side of the full-range GPU timings."""
    import oracle

    orc = oracle.load()
    cores = host_cores()
    out = {"cores": cores}
    for name, S in (("n_below_2p24", 1 << 24), ("n_below_2p32", 1 << 32)):
        orc.lib.orc_init(2 * S + 2)
        t0 = time.perf_counter()
        pairs = orc.pairs_crt(1, S, 3, nthreads=cores)
        out[name] = {"seconds": time.perf_counter() - t0, "pairs": len(pairs),
                     "method": "CRT enumeration over Algorithm 1 radicals (orc_pairs_crt)"}
    return out


# ---------------------------------------------------------------------------

def run_reference(args):
    # no collective: under torchrun only rank 0 works and prints, the other ranks exit at once
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    ivs = W.batch_intervals(4096)
    budget = int(args.ref_budget)
    for _ in range(args.warmup):
        cpu_baseline(ivs, budget // 8)
    vals, secs = [], []
    for _ in range(args.steps):
        r = cpu_baseline(ivs, budget)
        vals.append(r["value"])
        secs.append(r["seconds"])
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched: 4096 intervals, len log-uniform [2^16, 2^30], lo uniform [2^32, 2^40), "
                                   "kind 1|2 (seeded splitmix64); each step a bounded leading sample",
                       "sample_integers": budget},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                             "sample": f"first {budget} integers of the batched workload per step"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    ws, rank, local = dist_init()
    torch.cuda.set_device(local)
    from paper_2506_01099_gb300 import benelux as B

    gpu_name = torch.cuda.get_device_name(local)
    tune_json = merged_tune(gpu_name, args.tune)
    stream = torch.cuda.current_stream()
    ctx = B.Context(local, max_hi=MAX_HI, tune_json=tune_json, stream=stream.cuda_stream)
    if args.autotune:
        sample = [iv for iv in W.batch_intervals(4096)][:512]
        tj = ctx.autotune(sample, rounds=2)
        if rank == 0:
            print("autotuned:", tj, file=sys.stderr, flush=True)
            try:
                cache = json.load(open(TUNE_CACHE))
            except Exception:
                cache = {}
            d = json.loads(tj)
            d.pop("ms", None)
            cache[f"{gpu_name}|{MAX_HI.bit_length() - 1}"] = d
            json.dump(cache, open(TUNE_CACHE, "w"), indent=1, sort_keys=True)

    ivs = rank_intervals(rank)
    arr = B.make_intervals(ivs)
    integers = W.total_integers(ivs)

    for _ in range(args.warmup):
        B.bnx_batch(ctx.h, ivs, arr)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(ws)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
        time.sleep(0.3)
    dev_ms, sieve_ms, wall = [], [], []
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    npairs = 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        pairs, offs = B.bnx_batch(ctx.h, ivs, arr)
        wall.append(time.perf_counter() - t0)
        st = ctx.stats()
        dev_ms.append(st["ms_total"])
        sieve_ms.append(st["ms_sieve"])
        npairs = len(pairs)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop() if sampler else None
    loop_ms = e0.elapsed_time(e1)
    st = ctx.stats()

    # device-timed pipeline (inputs resident) and end-to-end through the public API
    t_dev = max_over_ranks(ws, sum(dev_ms) / 1e3)
    t_e2e = max_over_ranks(ws, sum(wall))
    total_int = sum_over_ranks(ws, float(integers)) * args.steps
    value = total_int / t_dev
    e2e = total_int / t_e2e

    extras = {}
    if rank == 0 and not args.quick:
        # plain path on the same intervals: one bnx_search per interval
        for iv in ivs[:16]:
            ctx.search(iv.lo, iv.hi, iv.kinds)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for iv in ivs:
            ctx.search(iv.lo, iv.hi, iv.kinds)
        tp = time.perf_counter() - t0
        extras["plain_same_intervals"] = {"value": integers / tp, "unit": UNIT, "seconds": tp,
                                          "note": "one blocking bnx_search per interval, same 4096 intervals"}
        # the large windows, plain (one call) vs batched (2^30-integer intervals)
        for wi, name in ((0, "window_2p40"), (1, "window_1p3e12")):
            lo, hi = W.LARGE_WINDOWS[wi]
            ctx.search(lo, lo + (1 << 30))
            t0 = time.perf_counter()
            p_plain = ctx.search(lo, hi)
            tpw = time.perf_counter() - t0
            wivs = W.large_window_intervals(wi)
            warr = B.make_intervals(wivs)
            B.bnx_batch(ctx.h, wivs, warr)
            t0 = time.perf_counter()
            p_b, _ = B.bnx_batch(ctx.h, wivs, warr)
            tbw = time.perf_counter() - t0
            extras[name] = {"range": [lo, hi], "plain": (hi - lo) / tpw, "batched": (hi - lo) / tbw, "unit": UNIT,
                            "pairs_plain": [list(p) for p in p_plain],
                            "pairs_batched": [list(p[1:]) for p in p_b]}
        extras["full_range_2p32"] = full_range_2p32(ctx)
        extras["materialised_rad"] = materialised_rad(ctx, torch, stream)
        extras["serving"] = serve_stream(B, ctx, args, throughput=value / ws)
        extras["serving_saturated"] = serve_stream(B, ctx, args, throughput=value / ws, saturate=True)
        # the same Poisson stream with 4x shorter slices: shorter iterations, lower latency, more
        # per-iteration overhead
        extras["serving_short_slices"] = serve_stream(B, ctx, args, throughput=value / ws,
                                                      slice_len=max(1 << 20, args.serve_slice // 4))

    if rank == 0:
        pk, pk_src = peaks()
        ms_sieve = statistics.mean(sieve_ms)
        sieve_rate = integers / (ms_sieve / 1e3)
        fmax = float(pk.get("sm_max_mhz", SM_MAX_MHZ))
        sms = torch.cuda.get_device_properties(local).multi_processor_count  # queried, not assumed
        alu_peak = sms * LANES_PER_CLK * fmax * 1e6 / 1e12
        tk = ctx.tune()["tile_kind"]
        achieved = sieve_rate * ALG_OPS_PER_INT[tk] / 1e12
        rec = sieve_record(tk)
        issue = None
        if rec is not None and rec.get("warp_inst_per_integer"):
            # measured warp instructions of the kernel (ncu) per integer, against the issue limit
            wipi = rec["warp_inst_per_integer"]
            issue = {"warp_inst_per_integer": wipi, "frac": sieve_rate * wipi / (sms * SCHEDULERS * fmax * 1e6),
                     "note": f"measured warp instructions x integers/s / ({sms} SMs x 4 schedulers x max clock)"}
        cpu = None
        if not args.no_cpu and ws == 1:
            cpu = cpu_baseline(W.batch_intervals(4096), int(args.cpu_budget))
            if not args.quick:
                cpu["full_ranges"] = cpu_full_ranges()
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": {"workload": "batched: 4096 intervals from seed, len log-uniform [2^16, 2^30], "
                                   "lo uniform [2^32, 2^40), kind 1|2 50/50; one persistent launch, CUDA graph",
                       "integers_per_step_per_gpu": integers, "tune": ctx.tune(),
                       "l2": "no flush needed: each step rewrites GB-scale bucket arrays (>> 129 MB L2)",
                       "parallelism": f"replicas x{ws} (independent intervals per GPU)"},
            "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 40 * len(ivs) + 4,
                    "d2h_bytes_per_step": 128 + 24 * npairs + 8 * (len(ivs) + 1)},
            "gpu_launches": KERNELS_PER_STEP * args.steps,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                         "frac": achieved / alu_peak,
                         "traffic": rec["dram_bytes_per_integer"] * integers if rec else None,
                         "kernel": {0: "k_sieve_log<search, u32 tile>", 1: "k_sieve<search, exact u64 tile>",
                                    2: "k_sieve_log<search, u16 tile>",
                                    3: "k_sieve_log<search, u8 tile>"}[ctx.tune()["tile_kind"]]
                                   + " (persistent shared-memory tile sieve, fused filter + warp-ballot compaction)",
                         "peak_source": f"{sms} SMs (queried) x 128 lanes/clk x {fmax:.0f} MHz max SM clock "
                                        f"({pk_src}) (issue roofline)",
                         "sms": sms,
                         "alg_ops_per_integer": ALG_OPS_PER_INT[tk], "sieve_ms_per_launch": ms_sieve,
                         "issue": issue,
                         "hbm_equivalent": {"achieved_gbs": sieve_rate * 8 / 1e9, "peak_gbs": pk["hbm_gbs"],
                                            "frac": sieve_rate * 8 / 1e9 / pk["hbm_gbs"],
                                            "note": f"8 B per integer vs {pk_src} copy bandwidth"}},
            "clocks": clocks,
            "device_loop_ms": loop_ms,
            "stats": st,
            "pairs_found": npairs,
        }
        if cpu:
            line["cpu_baseline"] = cpu
        line.update(extras)
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def full_range_2p32(ctx):
    """All pairs with n < 2^32 four ways: the CRT path, the device hash table
    over the filtered keys, Algorithm 2 (device radix sort of every key, about
    137 GB) and Algorithm 3 with the paper's chunks of 2^27."""
    out = {}
    once = ("algorithm3_chunks_2p27", "algorithm2_sorted")  # seconds, or 137 GB per call: run once
    for name, fn in (("crt_search", lambda: ctx.search(1, 1 << 32)),
                     ("hash_search", lambda: ctx.search_hash(1 << 32)),
                     ("algorithm2_sorted", lambda: ctx.search_sorted(1 << 32)),
                     ("algorithm3_chunks_2p27", lambda: ctx.search_chunked(1 << 32, 27))):
        try:
            if name not in once:
                fn()
            t0 = time.perf_counter()
            pairs = fn()
            dt = time.perf_counter() - t0
        except Exception as e:  # e.g. the 137 GB of Algorithm 2 not free on this device
            out[name] = {"error": str(e)}
            continue
        out[name] = {"seconds": dt, "pairs": len(pairs), "device_ms": ctx.stats()["ms_total"]}
    out["note"] = "paper: about one minute for n < 2^32 with Algorithm 3 on a 2021 consumer GPU"
    return out


def materialised_rad(ctx, torch, stream):
    """The HBM-writing counterpoint to the fused search: bnx_rad_segment (k_rad) writes
    the radical and the square part of each of the 2^31 integers
    [2^40, 2^40 + 2^31) to HBM (16 B per integer), CUDA-event timed."""
    lo, n = 1 << 40, 1 << 31
    rad = torch.empty(n, dtype=torch.int64, device="cuda")
    sq = torch.empty(n, dtype=torch.int64, device="cuda")
    ctx.rad_segment(lo, n, rad.data_ptr(), sq.data_ptr(), stream.cuda_stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ctx.rad_segment(lo, n, rad.data_ptr(), sq.data_ptr(), stream.cuda_stream)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    check = int(rad[0].item()) == 2 and int(sq[0].item()) == 1 << 39  # 2^40: radical 2
    del rad, sq
    torch.cuda.empty_cache()
    hbm = float(peaks()[0].get("hbm_gbs", 6800.0))
    gbs = 16 * n / (ms / 1e3) / 1e9
    return {"range": [lo, lo + n], "integers_per_s": n / (ms / 1e3), "ms": ms, "written_GBps": gbs,
            "hbm_frac": gbs / hbm, "first_value_ok": check,
            "note": "k_rad (u32 square-part tile) writing rad and the square part; the fused search writes neither"}


def serve_stream(B, ctx, args, throughput: float, saturate: bool = False, slice_len: int | None = None):
    """Seeded Poisson stream at 0.7x the batched throughput (or, saturated, every
    request at t = 0); p50/p99 latency and integers/s."""
    n = args.serve_requests
    mean_len = W.mean_serving_length()
    rate = 0.7 * throughput / mean_len
    reqs = W.serving_requests(n, rate_per_s=rate)
    if saturate:
        reqs = [W.Request(0.0, r.interval) for r in reqs]
    slice_len = slice_len or args.serve_slice
    B.bnx_server_start(ctx.h, max_active=args.serve_slots, slice_len=slice_len)
    lat = {}
    tickets = {}
    t0 = time.perf_counter()
    i = 0
    integers = sum(r.interval.length for r in reqs)
    try:
        while len(lat) < n:
            now = time.perf_counter() - t0
            while i < n and reqs[i].arrival_s <= now:
                iv = reqs[i].interval
                tickets[B.bnx_server_submit(ctx.h, iv.lo, iv.hi, iv.kinds, iv.id)] = i
                i += 1
            for t in list(tickets):
                r = B.bnx_server_poll(ctx.h, t)
                if r is not None:
                    lat[tickets.pop(t)] = r[1]
            if time.perf_counter() - t0 > args.serve_timeout:
                break
            time.sleep(0.001)
    finally:
        B.bnx_server_stop(ctx.h)
    span = time.perf_counter() - t0
    ls = sorted(lat.values())
    q = lambda p: ls[min(len(ls) - 1, int(math.ceil(p * len(ls))) - 1)] if ls else None
    return {"requests": n, "completed": len(ls), "rate_per_s": None if saturate else rate,
            "p50_s": q(0.50), "p99_s": q(0.99),
            "integers_per_s": integers / span, "span_s": span, "slots": args.serve_slots, "slice": slice_len,
            "note": ("all requests submitted at t = 0" if saturate else
                     "seeded Poisson arrivals at 0.7x batched throughput / E[len]") +
                    "; len log-uniform [2^20, 2^34], lo uniform [1, 1.4e12], kinds 1|2|3"}


def merged_tune(gpu_name: str, override: str | None) -> str | None:
    """The cached tuning for this GPU with the fields of `override` (JSON) on top."""
    base = json.loads(load_tune(gpu_name) or "{}")
    if override:
        base.update(json.loads(override))
    return json.dumps(base) if base else None


def profile_case(override: str | None = None, len_log2: int = 28):
    """One warm-up search and one search of [2^40, 2^40 + 2^len_log2): a single sieve
    launch over a window of the batched workload's magnitude (the small case for ncu;
    len_log2 = 32 gives a launch of about a millisecond, long enough for steady state)."""
    import torch

    from paper_2506_01099_gb300 import benelux as B

    ctx = B.Context(0, max_hi=MAX_HI, tune_json=merged_tune(torch.cuda.get_device_name(0), override))
    lo = 1 << 40
    ctx.search(lo, lo + (1 << 20))
    pairs = ctx.search(lo, lo + (1 << len_log2))
    print(json.dumps({"profile_case": [lo, lo + (1 << len_log2)], "pairs": pairs, "stats": ctx.stats()}))
    ctx.close()
    return 0


def profile_sorted(lg: int):
    """One Algorithm 2 search of all n < 2^lg (small case for ncu)."""
    from paper_2506_01099_gb300 import benelux as B

    ctx = B.Context(0, max_hi=MAX_HI)
    pairs = ctx.search_sorted(1 << lg)
    print(json.dumps({"profile_sorted": 1 << lg, "pairs": len(pairs), "stats": ctx.stats()}))
    ctx.close()
    return 0


def profile_rad(lg: int):
    """One warm-up and one bnx_rad_segment of 2^lg values at 2^40, rad and square part
    (the k_rad case for ncu)."""
    import torch

    from paper_2506_01099_gb300 import benelux as B

    ctx = B.Context(0, max_hi=MAX_HI)
    n = 1 << lg
    rad = torch.empty(n, dtype=torch.int64, device="cuda")
    sq = torch.empty(n, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        ctx.rad_segment(1 << 40, n, rad.data_ptr(), sq.data_ptr(), stream)
    torch.cuda.synchronize()
    print(json.dumps({"profile_rad": [1 << 40, (1 << 40) + n], "rad0": int(rad[0].item()), "sq0": int(sq[0].item())}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="timed batched steps only")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=2 ** 36)
    ap.add_argument("--ref-budget", type=float, default=2 ** 35)
    ap.add_argument("--serve-requests", type=int, default=1024)
    ap.add_argument("--serve-slots", type=int, default=64)
    ap.add_argument("--serve-slice", type=int, default=1 << 28)
    ap.add_argument("--serve-timeout", type=float, default=120.0)
    ap.add_argument("--tune", default=None, help="JSON of bnx_tune fields applied over the cached tuning")
    ap.add_argument("--profile-case", action="store_true",
                    help="one warm-up and one search of [2^40, 2^40 + 2^LEN) (small case for ncu), then exit")
    ap.add_argument("--profile-len-log2", type=int, default=28, metavar="LEN",
                    help="window length of --profile-case as a power of two (default 28)")
    ap.add_argument("--profile-sorted", type=int, default=0, metavar="LG",
                    help="one Algorithm 2 search of all n < 2^LG (small case for ncu), then exit")
    ap.add_argument("--profile-rad", type=int, default=0, metavar="LG",
                    help="radicals and square parts of 2^LG values at 2^40 (small case for ncu), then exit")
    args = ap.parse_args()
    if args.profile_sorted:
        return profile_sorted(args.profile_sorted)
    if args.profile_rad:
        return profile_rad(args.profile_rad)
    if args.profile_case:
        return profile_case(args.tune, args.profile_len_log2)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
