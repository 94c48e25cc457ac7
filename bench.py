"""Benchmark: set-bwte BWT build throughput (Mbp/s) on synthetic reads.

A step builds the BWT of the whole workload from an empty index: one
``sbwt_append`` of every read, which runs Algorithm 1 of arXiv 1410.0562 over
all its blocks (ConstructSA, B_int, ComputeRanks, the g[SA_int] gather,
Insert) in the library's CUDA kernels.  Default workload: 1M x 100 bp reads
from a seeded 10 Mbp i.i.d. genome with 1% substitutions (uniform offsets and
strands), blocks of 2^24 suffixes, 32-bit indices -- a synthetic stand-in
shaped like the paper's short-read set.

``value`` is timed with CUDA events on the library's stream, inputs already in
HBM; between timed steps a 256 MB buffer is written to flush L2 (outside the
timed region).  ``e2e`` times the host-buffer C-ABI call: H2D of the reads
from pinned memory, the build, and the D2H of B.  ``--impl reference`` times
the CPU oracle (a plain single-threaded suffix sort by direct comparison) on a
bounded sample of the same workload.

Under torchrun (N > 1) each rank builds an independent index of its own read
set (replicas: the path has no exchange step), so per-GPU work is fixed.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import readgen  # noqa: E402

METRIC = "BWT build Mbp/s"
UNIT = "Mbp/s"
# What bounds the kernels that can take the largest share, from their ncu
# captures (profiles/): the HBM fraction alone understates how close they are.
LIMITERS = {
    "radix_downsweep": "shared-memory ranking and staging: 40% issue, 36% DRAM, 0.46 of the copy bandwidth "
                       "alone under ncu (profiles/radix_downsweep_short-1Mx100.md)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="short", choices=["short", "tiny", "serve", "wide"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form measurement")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-form measurement")
    ap.add_argument("--profile-steps", type=int, default=None,
                    help="steps run under per-kernel event timing (default: the timed steps)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_workload(name: str, rank: int, n_reads: int = 1_000_000):
    if name == "tiny":
        w = readgen.tiny()
    elif name == "wide":
        w = readgen.wide(n_reads=n_reads, seed_genome=0x14100562 + 7 + 1000 * rank,
                         seed_reads=0x05621410 + 7 + 1000 * rank)
    else:
        # every rank indexes its own read set (same shape, its own seeds)
        w = readgen.short(n_reads=n_reads, seed_genome=0x14100562 + 2 + 1000 * rank,
                          seed_reads=0x05621410 + 2 + 1000 * rank)
    return w


def max_over_ranks(x: float, dist=None, device="cuda") -> float:
    """The largest x over all ranks (the job takes as long as its slowest rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mbps(bases_per_rank: int, world: int, steps: int, total_ms: float) -> float:
    """Weak scaling: every rank builds its own index of bases_per_rank bases per
    step; the job's throughput is all ranks' bases over the slowest rank's time."""
    return bases_per_rank * world * steps / (total_ms / 1e3) / 1e6


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def load_traffic(kernel: str, alg_bytes: float):
    """DRAM bytes of a launch of `kernel` that moves `alg_bytes` algorithmic
    bytes, scaled by units from the committed ncu capture
    (profiles/ncu_traffic.json), if that capture was taken on the kernel's
    current source files; else None."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        import hashlib
        with open(path) as f:
            t = json.load(f)
        if t.get("kernel") != kernel:
            return None
        h = hashlib.sha256()
        for name in t["source_files"]:
            h.update(name.encode())
            with open(os.path.join(ROOT, "paper_1410_0562_gb300", "csrc", name), "rb") as fh:
                h.update(fh.read())
        if h.hexdigest()[:16] != t["source_sha"]:
            return None
        return alg_bytes / float(t["algorithmic_bytes_per_unit"]) * float(t["dram_bytes_per_unit"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = f"/tmp/sbwt_clocks_{os.getpid()}.csv"

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index),
                 "--query-gpu=clocks.sm,clocks.max.sm,clocks_event_reasons.hw_slowdown,"
                 "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
                 "clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 6:
                    continue
                try:
                    sm.append(float(parts[0]))
                    mx.append(float(parts[1]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[2:6]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        except OSError:
            return None
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def measure_serving(sb, idx, requests, rate_rps=None, seed=7):
    """Serves `requests` (list of (reads, offsets)) against the index: all at
    once when rate_rps is None (closed loop: the sustained rate), else with
    Poisson arrivals at rate_rps requests/s.  Returns latency percentiles,
    throughput over the serving window and the batches' sizes."""
    import threading
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate_rps, size=len(requests)) if rate_rps else np.zeros(len(requests))
    tickets = [None] * len(requests)
    sb.sbwt_serve_start(idx.handle, 0)
    t0 = time.perf_counter()

    def submitter():
        t = t0
        for i, (r, o) in enumerate(requests):
            t += gaps[i]
            delay = t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            tickets[i] = sb.sbwt_submit(idx.handle, r, o)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat = []
    for tk in tickets:
        rc, _, ms = sb.sbwt_wait(idx.handle, tk)
        assert rc == sb.SBWT_OK, rc
        lat.append(ms)
    t1 = time.perf_counter()
    sb.sbwt_serve_stop(idx.handle)
    bases = sum(int(o[-1]) for _, o in requests)
    return {"requests": len(requests), "bases": bases, "Mbps": bases / (t1 - t0) / 1e6,
            "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "offered_rps": rate_rps}


def serving_report(sb, fresh, requests):
    """Closed loop for the sustained rate, then Poisson arrivals at 0.5x and
    0.9x of it (in requests/s).  Each run serves a freshly built resident
    index (fresh() builds one), so every run starts from the same index
    size; each run reports the index's memory when it ends."""
    out = {}
    rates = [None, 0.5, 0.9]
    sustained_rps = None
    for f in rates:
        idx = fresh()
        rate = None if f is None else f * sustained_rps
        r = measure_serving(sb, idx, requests, rate_rps=rate, seed=7 if f is None else int(f * 100))
        hbm, host = sb.sbwt_memory(idx.handle)
        r["memory_after"] = {"hbm": hbm, "host": host}
        idx.close()
        if f is None:
            sustained_rps = r["requests"] / (r["bases"] / r["Mbps"] / 1e6)
            out["sustained"] = r
        else:
            out[f"load_{f}"] = r
    return out


def cpu_baseline(w, n_reads: int):
    """The oracle as it stands on a bounded sample: the first n_reads reads."""
    import oracle
    n_reads = min(n_reads, w.m)
    off = w.offsets[: n_reads + 1]
    reads = w.reads[: int(off[-1])]
    t = time.perf_counter()
    oracle.bwt(reads, off, w.alphabet)
    dt = time.perf_counter() - t
    return {"value": float(off[-1]) / dt / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"first {n_reads} reads ({int(off[-1])} bp) of the workload, full BWT by the oracle, "
                      f"{dt:.1f} s single-threaded"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = make_workload(args.workload, 0)
    n_reads = min(50_000, w.m)
    off = w.offsets[: n_reads + 1]
    reads = w.reads[: int(off[-1])]
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.bwt(reads, off, w.alphabet)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.bwt(reads, off, w.alphabet)
        times.append(time.perf_counter() - t)
    total = sum(times)
    value = float(off[-1]) * args.steps / total / 1e6
    sample = (f"each step: the oracle's full BWT of the first {n_reads} reads ({int(off[-1])} bp) of the "
              f"workload, single-threaded")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "sample_reads": n_reads, "block_suffixes": w.block_suffixes,
                   "index_bits": w.index_bits, "parallelism": "none (host cores)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import torch

    import paper_1410_0562_gb300 as sb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl", device_id=torch.device("cuda", local))
        dist = dist_mod
    if rank == 0:
        sb.build()
    if dist:
        dist.barrier()
    sb.load()

    w = make_workload(args.workload, rank)
    bases = w.bases
    stream = torch.cuda.Stream()
    idx = sb.SetBWT(w.alphabet, index_bits=w.index_bits, block_suffixes=w.block_suffixes,
                    stream=stream.cuda_stream, device=local)
    d_reads = torch.from_numpy(w.reads).to("cuda")
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).to("cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()

    def step():
        idx.reset()
        idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # one untimed step with every kernel timed: the per-kernel breakdown and
    # the dominant kernel
    sb.sbwt_reset_kernel_stats(idx.handle)
    sb.sbwt_set_profiling(idx.handle, True)
    step()
    breakdown = [s for s in sb.sbwt_get_kernel_stats(idx.handle) if not s["name"].startswith("host:")]
    dominant = max(breakdown, key=lambda s: s["ms"])["name"]

    # timed region: K steps, each bracketed by events on the library stream;
    # inside, only the dominant kernel carries events (for the roofline)
    sb.sbwt_set_profiling_only(idx.handle, dominant)
    sb.sbwt_reset_kernel_stats(idx.handle)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)  # L2 flush, outside the events
                ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
        torch.cuda.synchronize()
    ms_steps = [a.elapsed_time(b) for a, b in ev]
    all_stats = sb.sbwt_get_kernel_stats(idx.handle)
    stats = [s for s in all_stats if not s["name"].startswith("host:")]
    host_phases = {s["name"][5:]: s["ms"] / args.steps for s in all_stats if s["name"].startswith("host:")}
    sb.sbwt_set_profiling(idx.handle, False)
    total_ms = max_over_ranks(float(sum(ms_steps)), dist)
    if dist:
        dist.barrier()

    # the result is the one the oracle pins: spot-check it on this rank
    B = idx.bwt()
    assert len(B) == bases + w.m
    assert int(np.count_nonzero(B == ord("$"))) == w.m

    # end to end through the host-buffer C ABI: pinned H2D, build, D2H of B
    e2e = None
    if not args.no_e2e:
        h_reads = torch.from_numpy(w.reads).pin_memory()
        h_off = torch.from_numpy(w.offsets.astype(np.int64)).pin_memory()
        h_out = torch.empty(bases + w.m, dtype=torch.uint8).pin_memory()
        out_ptr = h_out.data_ptr()
        import ctypes

        def e2e_step():
            idx.reset()
            sb.sbwt_append(idx.handle, h_reads.data_ptr(), h_off.data_ptr(), w.m)
            got = ctypes.c_uint64()
            rc = sb.load().sbwt_get_bwt(idx.handle, ctypes.c_void_p(out_ptr), bases + w.m, ctypes.byref(got))
            assert rc == 0

        for _ in range(max(1, args.warmup)):
            e2e_step()
        torch.cuda.synchronize()
        e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                e_ev[k][0].record(stream)
            e2e_step()
            e_ev[k][1].record(stream)
        torch.cuda.synchronize()
        e_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in e_ev)), dist)
        e2e = {"value": whole_job_mbps(bases, world, args.steps, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(w.reads.nbytes + w.offsets.nbytes),
               "d2h_bytes_per_step": int(bases + w.m)}

    # the batched form on the same reads: block size from the autotuner and
    # the whole append replayed from a captured CUDA graph
    batched = None
    if not args.no_batched:
        idx_b = sb.SetBWT(w.alphabet, index_bits=w.index_bits, stream=stream.cuda_stream, device=local)
        best_M, tune = sb.sbwt_autotune_block_suffixes(idx_b.handle, d_reads.data_ptr(), d_off.data_ptr(), w.m,
                                                       [1 << 22, 1 << 23, 1 << 24, 1 << 25, 1 << 26, 1 << 27])
        sb.sbwt_set_graph_replay(idx_b.handle, True)
        sb.sbwt_set_profiling_only(idx_b.handle, dominant)

        def step_b():
            idx_b.reset()
            idx_b.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)

        # the index alternates between two dictionary buffers, so two graphs:
        # each is seen once eagerly, then captured; replays from then on
        for _ in range(max(4, args.warmup)):
            step_b()
        sb.sbwt_reset_kernel_stats(idx_b.handle)
        b_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                for _ in range(args.steps)]
        torch.cuda.synchronize()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xFF)
                b_ev[k][0].record(stream)
            step_b()
            b_ev[k][1].record(stream)
        torch.cuda.synchronize()
        b_ms = max_over_ranks(float(sum(a.elapsed_time(b) for a, b in b_ev)), dist)
        b_stats = [s for s in sb.sbwt_get_kernel_stats(idx_b.handle) if not s["name"].startswith("host:")]
        b_dom = next((s for s in b_stats if s["name"] == dominant), None)
        Bb = idx_b.bwt()
        assert np.array_equal(Bb, B), "batched form differs from the plain pipeline"
        batched = {"value": whole_job_mbps(bases, world, args.steps, b_ms), "unit": UNIT,
                   "ms_per_step": b_ms / args.steps, "block_suffixes": int(best_M), "graph_replay": True,
                   "autotune_ms": {str(k): round(v, 3) for k, v in tune.items()},
                   "gpu_launches": int(sum(s["launches"] for s in b_stats)),
                   "dominant_kernel_GBps": (b_dom["bytes"] / (b_dom["ms"] / 1e3) / 1e9
                                            if b_dom and b_dom["ms"] > 0 else None)}
        idx_b.close()

    # the served form: requests of 10k..200k reads (U[100,150] bp) from the
    # same genome arriving at an index that holds the whole workload
    served = None
    if not args.no_serving and args.workload == "short":
        g = readgen.genome(10_000_000, 0x14100562 + 2 + 1000 * rank)
        rs = np.random.default_rng(99 + rank)
        sizes = np.exp(rs.uniform(np.log(10_000), np.log(200_000), size=24)).astype(np.int64)
        requests = [readgen.sampled_reads(g, int(mm), rs.integers(100, 151, size=int(mm)), 0.01, 500 + i)
                    for i, mm in enumerate(sizes)]
        def fresh():
            ix = sb.SetBWT(b"ACGT", block_suffixes=w.block_suffixes, index_bits=w.index_bits,
                           stream=stream.cuda_stream, device=local)
            ix.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)
            return ix

        served = serving_report(sb, fresh, requests)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    value = whole_job_mbps(bases, world, args.steps, total_ms)
    dom = next(s for s in stats if s["name"] == dominant)
    peak, peak_kind = load_peaks()
    achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9 if dom["ms"] > 0 else 0.0
    per_launch = dom["bytes"] / max(dom["launches"], 1)
    traffic = load_traffic(dom["name"], per_launch)
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": dom["bytes"] / max(dom["launches"], 1),
                "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1)}
    if dom["name"] in LIMITERS:
        roofline["limiter"] = LIMITERS[dom["name"]]
    kernels = {s["name"]: {"launches": s["launches"], "ms_per_step": s["ms"],
                           "GBps": (s["bytes"] / (s["ms"] / 1e3) / 1e9) if s["ms"] > 0 else None}
               for s in sorted(breakdown, key=lambda s: -s["ms"])}
    launches = int(sum(s["launches"] for s in stats))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": w.name, "reads": w.m, "bases": bases, "block_suffixes": w.block_suffixes,
                   "index_bits": w.index_bits, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "l2": "flushed between timed steps (256 MB write, outside the timed region)",
                   "step": "reset + one append of every read (all blocks of Algorithm 1)"},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": launches,
        "batched": batched,
        "served": served,
        "kernels": kernels,  # one untimed step with every kernel timed
        "host_ms_per_step": host_phases,
    }
    clocks = clk.summary()
    if clocks:
        line["clocks"] = clocks
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline(w, 200_000 if args.workload in ("short", "wide") else w.m)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def run_serve_workload(args):
    """The serving workload: a resident index of 20M x 100 bp reads (2 Gbp)
    under an 8 GB HBM budget, then append requests of 10k..1M reads arriving
    all at once (sustained rate) and as Poisson streams at 0.5x and 0.9x of
    it.  A second, smaller index under a 512 MB budget keeps its dictionaries
    in the pinned host tier and serves the same way."""
    import torch

    import paper_1410_0562_gb300 as sb
    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    sb.build()
    sb.load()
    t = time.perf_counter()
    resident, requests = readgen.serving()
    gen_s = time.perf_counter() - t
    stream = torch.cuda.Stream()
    idx = sb.SetBWT(b"ACGT", hbm_budget=8 << 30, index_bits=64, block_suffixes=1 << 25,
                    stream=stream.cuda_stream, device=local)
    d_reads = torch.from_numpy(resident.reads).to("cuda")
    d_off = torch.from_numpy(resident.offsets.astype(np.int64)).to("cuda")
    torch.cuda.synchronize()
    t = time.perf_counter()
    idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), resident.m)
    build_s = time.perf_counter() - t
    hbm, host = sb.sbwt_memory(idx.handle)
    n, m = idx.size()
    idx.close()

    def fresh():
        ix = sb.SetBWT(b"ACGT", hbm_budget=8 << 30, index_bits=64, block_suffixes=1 << 25,
                       stream=stream.cuda_stream, device=local)
        ix.append_device(d_reads.data_ptr(), d_off.data_ptr(), resident.m)
        return ix

    report = serving_report(sb, fresh, requests)
    del d_reads, d_off
    torch.cuda.empty_cache()

    # host tier: dictionaries in pinned host memory under a tight budget
    small = readgen.Workload("resident-2Mx100", resident.reads[: int(resident.offsets[2_000_000])],
                             resident.offsets[: 2_000_001], 1 << 21, 64, (0, 2_000_000))
    idx2 = sb.SetBWT(b"ACGT", hbm_budget=512 << 20, index_bits=64, block_suffixes=1 << 21,
                     stream=stream.cuda_stream, device=local)
    t = time.perf_counter()
    idx2.append(small.reads, small.offsets)
    build2_s = time.perf_counter() - t
    hbm2, host2 = sb.sbwt_memory(idx2.handle)
    small_reqs = [r for r in requests if len(r[1]) - 1 <= 100_000][:12]
    report2 = {"sustained": measure_serving(sb, idx2, small_reqs)}
    idx2.close()
    line = {
        "metric": "append throughput, served (Mbp/s); p50/p99 append latency", "unit": UNIT,
        "value": report["sustained"]["Mbps"], "higher_is_better": True, "n_gpus": 1, "data": "synthetic",
        "dtype": "u64",
        "config": {"workload": resident.name, "requests": len(requests), "hbm_budget": 8 << 30,
                   "block_suffixes": 1 << 25},
        "resident_build_s": build_s, "resident_build_Mbps": resident.bases / build_s / 1e6,
        "generation_s": gen_s, "resident_rows": n, "resident_reads": m,
        "memory_after_build": {"hbm": hbm, "host": host},
        "serving": report,
        "host_tier": {"resident": small.name, "hbm_budget": 512 << 20, "build_s": build2_s,
                      "memory": {"hbm": hbm2, "host": host2}, "serving": report2},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve":
        return run_serve_workload(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
