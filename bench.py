#!/usr/bin/env python3
"""Benchmark of the three-way partition sort on GB300.

Default workload (the headline): 2^27 int32 keys uniform over [-2^31, 2^31), seed 1,
sorted ascending by tsqs_sort.  Each timed step sorts its own freshly copied input
(512 MiB, larger than L2), staged in HBM before the timed region, so no step sees a
sorted array or a warm L2.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                       [--workload {uniform,patterns,c1,records,floats,batched,serving}]
Under torchrun each rank sorts its own array (replicas; the path does not shard), and
rank 0 prints one JSON line with the whole-job throughput (keys of all ranks / the
slowest rank's time).
"""
from __future__ import annotations

import argparse
import ctypes
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "Mkeys/s & % HBM roofline, 2^27 int32; batched vs per-call segs/s; p99 latency"
UNIT = "Mkeys/s"
N_HEADLINE = 1 << 27
SMALL_T = 4096
NOMINAL_HBM_GBS = 8000.0
FALLBACK_HBM_GBS = 6800.0

# dram__bytes_read.sum + dram__bytes_write.sum of one partition launch per key it read,
# from an ncu capture of the kernel source with this sha256 prefix (null when the
# kernel changed since).
# dram__bytes_read.sum + dram__bytes_write.sum of one full-width k_partition launch at the
# headline size (2^27 int32, level 3 of an instrumented sort): 537.1 MB + 479.1 MB for
# 134,217,721 keys; valid only for the kernel source it was taken on
NCU_TRAFFIC = {"kernels_sha": "c914553cd5b4a838",
               "bytes_per_key": (537056000 + 479370240) / 134217721,
               "source": "profiles/k_partition_2e27_int32_traffic.md"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tsqs", choices=["tsqs", "reference"])
    ap.add_argument("--workload", default="uniform",
                    choices=["uniform", "patterns", "c1", "records", "floats", "batched", "serving", "wide"])
    ap.add_argument("--n", type=int, default=N_HEADLINE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the compact timing of the other configurations in the headline line")
    ap.add_argument("--lookback", action="store_true",
                    help="with --profile: decoupled look-back offsets, whose layout (and so the "
                         "level count) does not depend on timing")
    ap.add_argument("--profile", action="store_true",
                    help="one instrumented (host-driven, one launch per kernel) sort of the "
                         "uniform workload and nothing else: the case the ncu captures use")
    ap.add_argument("--kind", default="i32", choices=["i32", "i64", "f32", "rec"],
                    help="with --profile: int32, int64 (uniform 64-bit), float32 (~N(0,1) with "
                         "specials) or {u64, u64} records")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", FALLBACK_HBM_GBS)), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def p_min(n: int, T: int = SMALL_T) -> int:
    """Unavoidable passes of a perfect-median three-way quicksort that finishes parts
    of <= T on chip: ceil(log2(n / T)) partition levels plus one on-chip pass."""
    return max(0, math.ceil(math.log2(n / T))) + 1 if n > T else 1


def size_label(n: int) -> str:
    return f"2^{n.bit_length() - 1}" if n & (n - 1) == 0 else str(n)


def kernels_sha() -> str:
    h = hashlib.sha256()
    for f in ("tsqs_kernels.cuh",):
        h.update(open(os.path.join(ROOT, "paper_1505_00558_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


# ------------------------------------------------------------------------------
# distributed plumbing
# ------------------------------------------------------------------------------

class Dist:
    def __init__(self, gpus: int):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group("gloo")
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ------------------------------------------------------------------------------
# clocks during the timed region
# ------------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.05)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, mx, reasons, pw = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------------------
# CPU legs (oracle; the only places bench.py runs oracle/)
# ------------------------------------------------------------------------------

def host_info() -> dict:
    """Host core count and CPU model of the box the bench runs on."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                if ln.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith(("model name", "cpu part")):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or None,
            "machine": platform.machine()}


class PinnedCore:
    """Runs the calling thread on one host core (the first it is allowed), so that the
    CPU references are single-threaded on the same core; restores the mask after."""

    def __enter__(self):
        self.mask = os.sched_getaffinity(0)
        self.core = min(self.mask)
        os.sched_setaffinity(0, {self.core})
        return self

    def __exit__(self, *exc):
        os.sched_setaffinity(0, self.mask)


def cpu_baselines(keys: np.ndarray) -> dict:
    """The oracle single-threaded on the whole workload once, and std::sort on the same
    core as a second (library) reference; Mkeys/s and seconds of each."""
    import oracle
    oracle.build()
    info = host_info()
    with PinnedCore() as pc:
        a = keys.copy()
        t0 = time.perf_counter()
        oracle.tsqs_sort(a, oracle.KIND_I32)
        t_orc = time.perf_counter() - t0
        b = keys.copy()
        t0 = time.perf_counter()
        oracle.std_sort_i32(b)
        t_std = time.perf_counter() - t0
    same = bool(np.array_equal(a, b))
    n = len(keys)
    return {"value": n / t_orc / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"the whole workload ({n} keys) sorted once by the oracle, single-threaded "
                      f"on host core {pc.core}",
            "seconds": t_orc,
            "std_sort": {"value": n / t_std / 1e6, "unit": UNIT, "seconds": t_std, "cores": 1,
                         "kind": "std::sort (g++ -O2), same core, same input",
                         "same_result_as_oracle": same},
            "host": info}


def reference_arm(args, dist):
    if dist.rank != 0:
        return
    from workloads import int32_pattern
    n = args.n
    keys = int32_pattern("random", min(n, 1 << 22) * 8, seed=1)
    chunk = 1 << 22
    import oracle
    oracle.build()
    for w in range(args.warmup):
        part = np.ascontiguousarray(keys[:chunk].copy())
        oracle.tsqs_sort(part, oracle.KIND_I32)
    times = []
    for s in range(args.steps):
        off = (s % 8) * chunk
        part = np.ascontiguousarray(keys[off:off + chunk].copy())
        t0 = time.perf_counter()
        oracle.tsqs_sort(part, oracle.KIND_I32)
        times.append(time.perf_counter() - t0)
    tot = sum(times)
    value = args.steps * chunk / tot / 1e6
    sample = f"each step: the oracle sorts {chunk} keys of the workload single-threaded"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": tot / args.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": "2^27 int32 uniform random seed 1 (bounded sample per step)",
                       "n_per_step": chunk},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample, "host": host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------
# GPU arm
# ------------------------------------------------------------------------------

def stage_copies(torch, src, count):
    return [src.clone() for _ in range(count)]


def time_sorts(torch, T, copies, kind, warmup, dist, records=False):
    """Sorts warmup copies untimed, then every remaining copy inside one timed region
    bracketed by a barrier and synchronize; returns (total ms, per-step ms list)."""
    stream = torch.cuda.current_stream()
    for i in range(warmup):
        T.sort_(copies[i], kind=kind)
    torch.cuda.synchronize()
    dist.barrier()
    torch.cuda.synchronize()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(len(copies) - warmup + 1)]
    evs[0].record(stream)
    for j, c in enumerate(copies[warmup:]):
        T.sort_(c, kind=kind)
        evs[j + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    total = evs[0].elapsed_time(evs[-1])
    per = [evs[j].elapsed_time(evs[j + 1]) for j in range(len(evs) - 1)]
    return total, per


def profile_case(args, dist):
    """One instrumented sort (every kernel its own launch: leaf, pivot, partition and
    level end per level, then the final leaf pass), for ncu captures; the graph path
    runs the same kernels as nodes of a conditional graph, which ncu does not profile
    one by one."""
    import torch
    torch.cuda.set_device(dist.local)
    import paper_1505_00558_gb300 as T
    from workloads import int32_pattern, records_u64
    from workloads.patterns import rand_u64
    n = args.n
    if args.kind == "rec":
        kind, label = T.TSQS_U64_U64_REC, "{u64, u64} records"
        src = torch.from_numpy(records_u64(n, seed=1).view(np.int64).copy()).cuda()
    elif args.kind == "i64":
        kind, label = T.TSQS_I64, "int64 uniform random"
        src = torch.from_numpy(rand_u64(1, 64, n).view(np.int64)).cuda()
    elif args.kind == "f32":
        from workloads import floats_normal_specials
        kind, label = T.TSQS_F32, "float32 ~N(0,1) with specials (raw bits)"
        src = torch.from_numpy(floats_normal_specials(n, seed=1).view(np.int32).copy()).cuda()
    else:
        kind, label = T.TSQS_I32, "int32 uniform random"
        src = torch.from_numpy(int32_pattern("random", n, seed=1)).cuda()
    plan = T.Plan()
    T.lib().tsqs_plan_default(kind, n, ctypes.byref(plan))
    plan.offset_mode = 1 if args.lookback else 0
    ctx = T.Context(plan)
    ms, keys, lms = ctx.sort_timed(src, kind=kind)
    torch.cuda.synchronize()
    if kind == T.TSQS_U64_U64_REC:
        # (key, payload) in order as unsigned 64-bit words: flip the sign bits, compare signed
        flip = torch.tensor(-(1 << 63), dtype=torch.int64, device=src.device)
        k, p = src[:, 0] ^ flip, src[:, 1] ^ flip
        ok = ctx.status() == 0 and bool(((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (p[1:] >= p[:-1]))).all().item())
    elif kind == T.TSQS_F32:
        # IEEE totalOrder on the raw bits: negative values flip their low 31 bits
        k = src ^ ((src >> 31) & 0x7FFFFFFF)
        ok = ctx.status() == 0 and bool((k[1:] >= k[:-1]).all().item())
    else:
        ok = ctx.status() == 0 and bool((src[1:] >= src[:-1]).all().item())
    if dist.rank == 0:
        print(json.dumps({"profile_case": f"{size_label(n)} {label} seed 1",
                          "levels": len(ms), "leaf_launches": len(ms) + 1, "sorted": ok,
                          "partition_ms": [round(m, 4) for m in ms],
                          "leaf_ms": [round(m, 4) for m in lms]}), flush=True)
    ctx.close()
    if not ok:
        raise SystemExit(1)


def gpu_arm(args, dist):
    import torch
    torch.cuda.set_device(dist.local)
    import paper_1505_00558_gb300 as T
    from workloads import int32_pattern
    T.lib()
    hbm, hbm_src = peaks()
    n = args.n
    K, W = args.steps, args.warmup
    x = int32_pattern("random", n, seed=1 + dist.rank * 0)
    src = torch.from_numpy(x).cuda()
    copies = stage_copies(torch, src, K + W)
    torch.cuda.synchronize()

    clocks = ClockSampler(dist.local)
    clocks.start()
    total_ms, per = time_sorts(torch, T, copies, T.TSQS_I32, W, dist)
    clk = clocks.stop()
    status = T.last_device_status()
    ok = bool((copies[-1][1:] >= copies[-1][:-1]).all().item()) and status == 0
    total_ms = dist.max(total_ms)
    keys_all = dist.sum(float(K * n))
    value = keys_all / (total_ms * 1e-3) / 1e6
    ms_step = total_ms / K

    # launches per sort: setup, the three presortedness kernels, init, 3 per level
    # iteration (pivot, partition, level end), the leaf pass and the loop control after
    # the levels (the depth guard's branch is skipped: no segment reaches its level)
    ctx = T.Context()
    chk = src.clone()
    T.sort_(chk, kind=T.TSQS_I32, ctx=ctx)
    st = ctx.stats()
    iters = max(1, st["levels"])
    launches_per_sort = 7 + 3 * iters
    del copies

    # dominant kernel: partition levels, timed one launch at a time with CUDA events
    part_ms, part_keys = [], []
    leaf_ms, leaf_runs = [], []
    for r in range(3):
        c = src.clone()
        ms, keys, lms = ctx.sort_timed(c, kind=T.TSQS_I32)
        if r == 0:
            continue                                     # first instrumented run warms up
        part_ms += ms
        part_keys += keys
        leaf_ms += lms
        leaf_runs.append(lms)
    busy = [(m, k) for m, k in zip(part_ms, part_keys) if k > 0]
    finals = [run[-1] - (statistics.median(run[:-1]) if len(run) > 1 else 0.0)
              for run in leaf_runs if run]
    leaf_final = sum(finals) / len(finals) if finals else None
    alg_bytes = sum(2 * 4 * k for _, k in busy)
    t_part = sum(m for m, _ in busy) * 1e-3
    achieved = alg_bytes / t_part / 1e9 if t_part > 0 else None
    n_launch = len(busy)
    sha = kernels_sha()
    traffic = None
    if NCU_TRAFFIC["kernels_sha"] == sha and NCU_TRAFFIC["bytes_per_key"]:
        traffic = NCU_TRAFFIC["bytes_per_key"] * (sum(k for _, k in busy) / max(1, n_launch))
    roofline = {"bound": "hbm", "kernel": "k_partition (one launch per level)",
                "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None,
                "traffic": traffic, "peak_source": hbm_src,
                "alg_bytes_per_launch": alg_bytes / max(1, n_launch),
                "avg_launch_ms": t_part * 1e3 / max(1, n_launch),
                "note": "8 bytes (one 4-byte read + one 4-byte write) per key partitioned in the "
                        "launch; launch times from CUDA events around each partition launch"}
    pm = p_min(n)
    whole_alg = pm * 2 * n * 4
    whole = {"p_min": pm, "alg_bytes": whole_alg,
             "achieved_gbs": whole_alg / (ms_step * 1e-3) / 1e9,
             "frac_of_measured": whole_alg / (ms_step * 1e-3) / 1e9 / hbm,
             "frac_of_nominal_8tbs": whole_alg / (ms_step * 1e-3) / 1e9 / NOMINAL_HBM_GBS,
             "roofline_mkeys": hbm * 1e9 / (2 * pm * 4) / 1e6,
             "partition_ms_per_sort": sum(m for m, _ in busy) / 2,
             # the graph runs one leaf pass after the levels; the host-driven run also
             # launches an (empty) leaf kernel per level, whose time the final entry
             # includes once: take a typical empty launch off it
             "leaf_final_pass_ms": leaf_final,
             "leaf_ms_per_sort_host_driven": sum(leaf_ms) / 2}

    # end to end through the C-ABI with host buffers (pinned), copies inside the region:
    # K host arrays streamed through tsqs_ctx_sort_host_stream (each step uploads the
    # unsorted input and downloads its sorted result; the copies of neighbouring steps
    # overlap the sort), plus the latency of one tsqs_sort_host call for reference
    e2e = None
    if not args.no_e2e:
        hsrc = torch.from_numpy(x).pin_memory()
        houts = [torch.empty_like(hsrc).pin_memory() for _ in range(3)]
        ectx = T.Context()
        ectx.sort_host_stream([hsrc] * W, [houts[i % 3] for i in range(W)], kind=T.TSQS_I32)
        torch.cuda.synchronize()
        dist.barrier()
        t0 = time.perf_counter()
        est = ectx.sort_host_stream([hsrc] * K, [houts[i % 3] for i in range(K)],
                                    kind=T.TSQS_I32)
        t1 = time.perf_counter()
        tt = dist.max(t1 - t0)
        ref = torch.sort(src)[0]
        e2e_ok = all(s_ == 0 for s_ in est) and all(torch.equal(h.cuda(), ref) for h in houts)
        del ref
        ectx.close()
        del houts
        # one call at a time: upload, sort, result written into the pinned array
        hbuf = torch.empty_like(hsrc).pin_memory()
        s = torch.cuda.current_stream()
        lib = T.lib()
        times = []
        for i in range(W + 5):
            hbuf.copy_(hsrc)
            ts0 = time.perf_counter()
            rc = lib.tsqs_sort_host(ctypes.c_void_p(hbuf.data_ptr()), n, 4, T.TSQS_I32,
                                    ctypes.c_void_p(s.cuda_stream))
            ts1 = time.perf_counter()
            assert rc == 0
            if i >= W:
                times.append(ts1 - ts0)
        single_ok = bool((hbuf[1:] >= hbuf[:-1]).all().item())
        ts = dist.max(sum(times))
        e2e = {"value": dist.sum(float(K * n)) / tt / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": n * 4, "d2h_bytes_per_step": n * 4,
               "ms_per_step": tt * 1e3 / K,
               "api": "tsqs_ctx_sort_host_stream: K steps, each a pinned host array copied "
                      "in, sorted on the device and copied out into a pinned host array "
                      "(host wall clock around the call)",
               "sorted": e2e_ok,
               "single_call": {"api": "tsqs_sort_host, one array per call",
                               "value": dist.sum(float(len(times) * n)) / ts / 1e6,
                               "ms": ts * 1e3 / len(times), "sorted": single_ok}}

    configs = None
    if not args.no_configs:
        configs = other_configs(torch, T, hbm)

    cpu = None
    if dist.rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baselines(x)

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": dist.world,
            "steps": K, "warmup": W, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": f"{size_label(n)} int32 uniform random [-2^31, 2^31), seed 1, tsqs_sort",
                       "n": n, "parallelism": f"replicas x{dist.world}",
                       "l2": "inputs larger than L2: every step sorts its own fresh 512 MiB copy",
                       "small_threshold": SMALL_T},
            "roofline": roofline, "roofline_whole_sort": whole, "cpu_baseline": cpu,
            "configs": configs,
            "e2e": e2e, "clocks": clk, "gpu_launches": launches_per_sort * K,
            "sorted": ok, "device_status": status,
            "per_step_ms": {"median": statistics.median(per), "min": min(per), "max": max(per)},
            "levels": st["levels"], "kernels_sha": sha}
    if dist.rank == 0:
        print(json.dumps(line), flush=True)


def other_configs(torch, T, hbm: float) -> dict:
    """Compact timings of the other configurations for the headline line: 1e6 int32
    (latency), the six other 2^27 int32 orderings, 2^26 records and 2^26 float32 under
    totalOrder.  Each: one warm-up sort, then the median of a few timed sorts of fresh
    copies (CUDA events; every input but the 1e6 one is larger than L2)."""
    from workloads import PATTERNS, int32_pattern, records_u64, floats_normal_specials
    out = {}

    def one(name, src, kind, n, es, reps, desc):
        med, best, ok, w = _time_fresh(torch, T, src, kind, reps, warm=1)
        if es == 16:
            flip = torch.tensor(-(1 << 63), dtype=torch.int64, device=w.device)
            k, p = w[:, 0] ^ flip, w[:, 1] ^ flip
            ok = ok and bool(((k[1:] > k[:-1]) | ((k[1:] == k[:-1]) & (p[1:] >= p[:-1]))).all().item())
        elif kind == T.TSQS_F32:
            u = w.view(torch.int32)
            key = torch.where(u < 0, u ^ 0x7FFFFFFF, u)        # totalOrder as signed ints
            ok = ok and bool((key[1:] >= key[:-1]).all().item())
        else:
            ok = ok and bool((w[1:] >= w[:-1]).all().item())
        pm = p_min(n)
        out[name] = {"workload": desc, "ms": med, "best_ms": best, "mkeys_s": n / med / 1e3,
                     "sorted": ok,
                     "frac_whole_sort_of_measured": pm * 2 * n * es / (med * 1e-3) / 1e9 / hbm}
        del w

    src = torch.from_numpy(int32_pattern("random", 1_000_000, seed=1)).cuda()
    one("c1_1e6_int32", src, T.TSQS_I32, 1_000_000, 4, 10,
        "1e6 int32 uniform random seed 1 (L2-resident: latency, not a roofline case)")
    n = N_HEADLINE
    for p in PATTERNS:
        if p == "random":
            continue
        src = torch.from_numpy(int32_pattern(p, n, seed=1)).cuda()
        one(f"c2_{p}", src, T.TSQS_I32, n, 4, 2, f"2^27 int32 {p}, seed 1")
        del src
    src = torch.from_numpy(records_u64(1 << 26, seed=1).view(np.int64)).cuda()
    one("c3a_records", src, T.TSQS_U64_U64_REC, 1 << 26, 16, 2,
        "2^26 {u64 key, u64 payload}, 10% duplicated keys, 0.1% duplicated records")
    del src
    src = torch.from_numpy(floats_normal_specials(1 << 26, seed=1)).cuda()
    one("c3b_float32", src, T.TSQS_F32, 1 << 26, 4, 2,
        "2^26 float32 ~N(0,1) with 0.1% +-0, +-inf, NaNs (IEEE totalOrder)")
    del src
    torch.cuda.empty_cache()
    return out


def _time_fresh(torch, T, src, kind, reps, records=False, ctx=None, warm=2):
    """Median / best ms of sorting fresh copies of src (copy outside the events)."""
    ts = []
    for r in range(reps + warm):
        w = src.clone()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        T.sort_(w, kind=kind, ctx=ctx)
        e1.record()
        torch.cuda.synchronize()
        if r >= warm:
            ts.append(e0.elapsed_time(e1))
    status = T.last_device_status() if ctx is None else ctx.status()
    ok = status == 0
    return statistics.median(ts), min(ts), ok, w


def _line(args, dist, value, config, extra, higher=True, unit=UNIT, ms=None):
    d = {"metric": METRIC, "value": value, "unit": unit, "n_gpus": dist.world,
         "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
         "higher_is_better": higher, "scaling": "weak", "vs_baseline": None,
         "dtype": config.pop("dtype", "int32"), "data": "synthetic", "config": config}
    d.update(extra)
    if dist.rank == 0:
        print(json.dumps(d), flush=True)


def other_workload(args, dist):
    import torch
    torch.cuda.set_device(dist.local)
    import paper_1505_00558_gb300 as T
    from workloads import (PATTERNS, int32_pattern, records_u64, floats_normal_specials)
    T.lib()
    hbm, hbm_src = peaks()
    w = args.workload
    if w == "c1":
        n = 1_000_000
        src = torch.from_numpy(int32_pattern("random", n, seed=1)).cuda()
        med, best, ok, out = _time_fresh(torch, T, src, T.TSQS_I32, max(args.steps, 10))
        _line(args, dist, n / med / 1e3, {"workload": "1e6 int32 uniform random seed 1 (L2-resident)",
                                          "n": n}, {"latency_ms_median": med, "latency_ms_best": best,
                                                    "sorted": ok}, ms=med)
    elif w == "patterns":
        n = args.n
        res = {}
        pm = p_min(n)
        for p in PATTERNS:
            src = torch.from_numpy(int32_pattern(p, n, seed=1)).cuda()
            med, best, ok, out = _time_fresh(torch, T, src, T.TSQS_I32, 3)
            ok = ok and bool((out[1:] >= out[:-1]).all().item())
            res[p] = {"mkeys_s": n / med / 1e3, "ms": med, "sorted": ok,
                      "frac_whole_sort_of_measured": pm * 2 * n * 4 / (med * 1e-3) / 1e9 / hbm}
            del src, out
        _line(args, dist, res["random"]["mkeys_s"], {"workload": f"{n} int32, seven patterns, seed 1", "n": n},
              {"patterns": res}, ms=res["random"]["ms"])
    elif w in ("records", "floats"):
        n = 1 << 26
        if w == "records":
            r = records_u64(n, seed=1)
            src = torch.from_numpy(r.view(np.int64)).cuda()
            kind, es, dt = T.TSQS_U64_U64_REC, 16, "u64+u64 record"
            desc = "2^26 records {u64 key, u64 payload}, 10% duplicated keys, 0.1% duplicated records"
        else:
            x = floats_normal_specials(n, seed=1)
            src = torch.from_numpy(x).cuda()
            kind, es, dt = T.TSQS_F32, 4, "float32 (totalOrder)"
            desc = "2^26 float32 ~N(0,1) with 0.1% +-0, +-inf, NaNs (IEEE totalOrder)"
        med, best, ok, out = _time_fresh(torch, T, src, kind, 5)
        pm = p_min(n)
        alg = pm * 2 * n * es
        _line(args, dist, n / med / 1e3, {"workload": desc, "n": n, "dtype": dt},
              {"sorted_status_ok": ok, "roofline_whole_sort": {
                  "p_min": pm, "alg_bytes": alg, "achieved_gbs": alg / (med * 1e-3) / 1e9,
                  "frac_of_measured": alg / (med * 1e-3) / 1e9 / hbm,
                  "roofline_mkeys": hbm * 1e9 / (2 * pm * es) / 1e6}}, ms=med)
    elif w == "wide":
        # large elements (Section VIII.G-H): 56-byte elements, int64 key at byte 8
        n, es, off = 1 << 24, 56, 8
        from workloads import rand_u64
        raw = np.frombuffer(rand_u64(1, 800, n * es // 8).tobytes(), dtype=np.uint8).copy()
        src = torch.from_numpy(raw).cuda()
        del raw
        ts = []
        for r in range(args.warmup + max(3, min(args.steps, 10))):
            wk = src.clone()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            T.sort_wide_(wk, es, off, T.TSQS_I64)
            e1.record()
            torch.cuda.synchronize()
            if r >= args.warmup:
                ts.append(e0.elapsed_time(e1))
        ok = T.last_device_status() == 0
        keys = wk.view(-1, es)[:, off:off + 8].contiguous().view(torch.int64).view(-1)
        ok = ok and bool((keys[1:] >= keys[:-1]).all().item())
        med = statistics.median(ts)
        pm = p_min(n)
        # key pass (8 B read, 16 B write), record sort (P_min passes of 2 x 16 B), gather
        # (16 B record + es read + es write), copy back (es read + es write)
        alg = n * (24 + pm * 32 + 16 + 4 * es)
        _line(args, dist, n / med / 1e3,
              {"workload": "2^24 elements of 56 bytes, int64 key at byte 8, uniform random, tsqs_sort_wide",
               "n": n, "elem_size": es},
              {"sorted_status_ok": ok, "roofline_whole_sort": {
                  "p_min_records": pm, "alg_bytes": alg, "achieved_gbs": alg / (med * 1e-3) / 1e9,
                  "frac_of_measured": alg / (med * 1e-3) / 1e9 / hbm}}, ms=med)
    elif w == "batched":
        batched_workload(args, dist, torch, T)
    elif w == "serving":
        serving_workload(args, dist, torch, T)


def batched_workload(args, dist, torch, T):
    """20,000 int32 segments, sizes floor(2^(20U)) in [1, 2^20], pattern per segment:
    one graph-replayed segmented sort with an autotuned plan vs a loop of per-segment
    tsqs_sort calls, on identical inputs, results compared byte for byte."""
    from workloads.patterns import batched_segments, batched_keys
    nseg = 20_000
    offs, sizes, pat = batched_segments(nseg, seed=1)
    x = batched_keys(offs, pat, seed=1)
    total = int(offs[-1])
    src = torch.from_numpy(x).cuda()
    d_offs = torch.from_numpy(offs.astype(np.int64)).cuda()
    del x
    plan = T.Plan()
    s = torch.cuda.current_stream()
    t0 = time.perf_counter()
    rc = T.lib().tsqs_plan_autotune(T.TSQS_I32, total, nseg, ctypes.c_void_p(s.cuda_stream),
                                    ctypes.byref(plan))
    tune_s = time.perf_counter() - t0
    ctx = T.Context(plan) if rc == 0 else T.Context()
    ctx.reserve(total, nseg, 4)
    # batched: one segmented call per step
    bt = []
    for r in range(args.warmup + 3):
        w = src.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        T.sort_segmented_(w, d_offs, kind=T.TSQS_I32, ctx=ctx)
        e1.record()
        torch.cuda.synchronize()
        if r >= args.warmup:
            bt.append(e0.elapsed_time(e1))
    ok_b = ctx.status() == 0
    out_b = w
    # per call: one tsqs_sort per segment (same context, same plan)
    w2 = src.clone()
    lib = T.lib()
    ptr = w2.data_ptr()
    sp = ctypes.c_void_p(s.cuda_stream)
    ofl = [int(o) for o in offs]
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for i in range(nseg):
        n = ofl[i + 1] - ofl[i]
        if n > 1:
            lib.tsqs_ctx_sort(ctx.handle, ctypes.c_void_p(ptr + 4 * ofl[i]), n, 4, T.TSQS_I32, sp)
    e1.record()
    torch.cuda.synchronize()
    pc = e0.elapsed_time(e1)
    same = bool(torch.equal(out_b, w2))
    bmed = statistics.median(bt)
    _line(args, dist, total / bmed / 1e3,
          {"workload": "batched: 20,000 int32 segments, sizes floor(2^(20U)) in [1, 2^20], seven patterns",
           "n_total": total, "nseg": nseg},
          {"batched": {"ms": bmed, "mkeys_s": total / bmed / 1e3, "segs_s": nseg / bmed * 1e3,
                       "status_ok": ok_b},
           "per_call": {"ms": pc, "mkeys_s": total / pc / 1e3, "segs_s": nseg / pc * 1e3},
           "batched_over_per_call": pc / bmed, "identical_results": same,
           "plan": plan.as_dict(), "autotune_s": tune_s}, ms=bmed)


def _gen_request(torch, kind_rec, n, pattern, seed, dev):
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    if kind_rec:
        r = torch.randint(-2 ** 63, 2 ** 63 - 1, (n, 2), dtype=torch.int64, device=dev, generator=g)
        h = max(1, n // 20)
        dup = torch.randint(0, n, (2 * h,), device=dev, generator=g)
        r[dup[:h], 0] = r[dup[h:], 0]
        return r
    i = torch.arange(n, device=dev, dtype=torch.int64)
    if pattern == "random":
        return torch.randint(-2 ** 31, 2 ** 31 - 1, (n,), dtype=torch.int32, device=dev, generator=g)
    if pattern == "sorted":
        return i.to(torch.int32)
    if pattern == "reversed":
        return (n - 1 - i).to(torch.int32)
    if pattern == "organ_pipe":
        return torch.where(i < n // 2, i + 1, n - i).to(torch.int32)
    if pattern == "many_equals":
        return torch.randint(0, 16, (n,), dtype=torch.int32, device=dev, generator=g)
    if pattern == "stair_steps":
        return (i // 1024).to(torch.int32)
    a = i.to(torch.int32)
    k = max(1, n // 200)
    p1 = torch.randint(0, n, (k,), device=dev, generator=g)
    p2 = torch.randint(0, n, (k,), device=dev, generator=g)
    a[p1], a[p2] = a[p2].clone(), a[p1].clone()
    return a


def serving_workload(args, dist, torch, T):
    """Poisson stream of 50,000 sort requests, sizes floor(2^(10 + 14U)), 70% int32 /
    30% (u64, u64) records, patterns from the seven, admitted under a 40 GB budget.
    The offered load is 0.7 x the sustained throughput measured with every request
    arriving at once.  Request contents come from a pool of 2,000 distinct generated
    requests: request i sorts pool entry i mod 2000 in a work buffer of its own, which is
    refilled from the pristine copy as soon as request i - 2000 on it has finished (off
    the submission path; a request whose buffer is not refilled yet when it arrives
    counts as a pool stall).  Latency is measured from the request's Poisson arrival
    time to its completion, on the host's monotonic clock; the time from submission to
    completion is reported beside it."""
    from workloads import PATTERNS
    from workloads.patterns import serving_requests
    nreq = int(os.environ.get("TSQS_SERVE_REQUESTS", "50000"))
    npool = min(nreq, int(os.environ.get("TSQS_SERVE_POOL", "2000")))
    budget, lanes = 40 << 30, 4
    req = serving_requests(nreq, seed=1)
    dev = torch.device("cuda")
    pristine = []
    for j in range(npool):
        pristine.append(_gen_request(torch, bool(req["is_rec"][j]), int(req["sizes"][j]),
                                     PATTERNS[int(req["pattern"][j])], j, dev))
    torch.cuda.synchronize()
    sizes = [int(req["sizes"][i % npool]) for i in range(nreq)]
    is_rec = [bool(req["is_rec"][i % npool]) for i in range(nreq)]
    nbytes = np.array([s_ * (16 if r_ else 4) for s_, r_ in zip(sizes, is_rec)], dtype=np.float64)
    total_keys = sum(sizes)
    lib = T.lib()
    stream = torch.cuda.current_stream()

    def run(lam):
        work = [p.clone() for p in pristine]
        ready = [None] * npool         # event of the buffer's last refill, until consumed
        torch.cuda.synchronize()
        srv = lib.tsqs_server_create(budget, lanes, 256)
        assert srv
        arrive = np.cumsum(req["gaps"] / lam) if lam else np.zeros(nreq)
        tickets = [None] * nreq
        py_sub = np.zeros(nreq)
        r = T.Result()
        stalls = 0                     # arrivals whose buffer was not refilled yet
        oldest = 0                     # first request whose buffer has not been refilled
        t0 = time.perf_counter()
        i = 0
        while True:
            # refill the buffers of finished requests (in submission order), long before
            # their next request arrives; the copies run on the device, the host goes on
            while oldest < i and oldest + npool < nreq:
                lib.tsqs_server_poll(srv, tickets[oldest], ctypes.byref(r))
                if not r.done:
                    break
                j = oldest % npool
                work[j].copy_(pristine[j])
                ev = torch.cuda.Event()
                ev.record(stream)
                ready[j] = ev
                oldest += 1
            now = time.perf_counter() - t0
            while i < nreq and arrive[i] <= now:
                j = i % npool
                if i >= npool:
                    if ready[j] is None or not ready[j].query():
                        stalls += 1
                        break
                    ready[j] = None
                tk = ctypes.c_uint64()
                kind, es = (T.TSQS_U64_U64_REC, 16) if is_rec[i] else (T.TSQS_I32, 4)
                rc = lib.tsqs_server_submit(srv, ctypes.c_void_p(work[j].data_ptr()), sizes[i], es,
                                            kind, ctypes.byref(tk))
                py_sub[i] = time.perf_counter()
                assert rc == 0, rc
                tickets[i] = tk.value
                i += 1
            left = lib.tsqs_server_progress(srv)
            if i == nreq and left == 0:
                break
        res = []
        for k in range(nreq):
            rr = T.Result()
            lib.tsqs_server_poll(srv, tickets[k], ctypes.byref(rr))
            res.append((rr.t_submit, rr.t_start, rr.t_done, rr.status, rr.batch_size, rr.batch_id))
        lib.tsqs_server_destroy(srv)
        t_sub = np.array([x[0] for x in res])
        t_start = np.array([x[1] for x in res])
        t_done = np.array([x[2] for x in res])
        # the server stamps times on its own monotonic clock: map the arrivals onto it
        # by the offset between the two clocks seen at every submission
        offset = float(np.median(py_sub - t_sub))
        t_arr = t0 + arrive - offset
        lat = (t_done - t_arr) * 1e3
        svc = (t_done - t_sub) * 1e3
        wait = (t_start - t_arr) * 1e3
        span = t_done.max() - min(t_arr.min(), t_sub.min())
        # device bytes of the requests launched and not yet complete, over time
        ev_t = np.concatenate([t_start, t_done])
        ev_b = np.concatenate([nbytes, -nbytes])
        order = np.lexsort((ev_b, ev_t))           # completions before launches at a tie
        in_flight = np.cumsum(ev_b[order])
        ok = all(x[3] == 0 for x in res)
        sorted_ok = all(bool((w[1:] >= w[:-1]).all().item()) if w.dim() == 1 else True for w in work[:50])
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()),
                "latency": "from the Poisson arrival time to completion",
                "service_p50_ms": float(np.percentile(svc, 50)),
                "service_p99_ms": float(np.percentile(svc, 99)),
                "queue_wait_p99_ms": float(np.percentile(wait, 99)),
                "sustained_mkeys_s": total_keys / span / 1e6,
                "span_s": span, "status_ok": ok, "spot_sorted": sorted_ok,
                "batches": len(set(x[5] for x in res)),
                "mean_batch": float(np.mean([x[4] for x in res])),
                "pool_stalls": stalls,
                "bytes_in_flight_peak": float(in_flight.max()),
                "bytes_in_flight_mean": float(np.average(
                    in_flight[:-1], weights=np.diff(ev_t[order]))) if len(in_flight) > 1 else 0.0,
                "budget_bytes": budget, "lanes": lanes}

    run(None)                                             # warm graphs and lanes
    sat = run(None)
    lam = 0.7 * sat["sustained_mkeys_s"] * 1e6 / (total_keys / nreq)
    load = run(lam)
    _line(args, dist, load["sustained_mkeys_s"],
          {"workload": f"serving: {nreq} Poisson requests (contents from a pool of {npool}), "
                       "sizes 2^10..2^24 log-uniform, 70% int32 / 30% u64+u64 records, seven "
                       "patterns, 40 GB budget, 4 lanes",
           "requests": nreq, "pool": npool, "offered_load_req_s": lam},
          {"at_offered_load": load, "saturated": sat}, ms=load["mean_ms"])


def main():
    args = parse()
    dist = Dist(args.gpus)
    try:
        if args.impl == "reference":
            reference_arm(args, dist)
        elif args.profile:
            profile_case(args, dist)
        elif args.workload == "uniform":
            gpu_arm(args, dist)
        else:
            other_workload(args, dist)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
