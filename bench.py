"""Benchmark: set-bwte BWT build throughput (Mbp/s) on synthetic reads.

A step builds the BWT of the whole workload from an empty index: one
``sbwt_append`` of every read, which runs Algorithm 1 of arXiv 1410.0562 over
all its blocks (ConstructSA, B_int, ComputeRanks, the g[SA_int] gather,
Insert) in the library's CUDA kernels.  Headline workload (``value``): 1M x
100 bp reads from a seeded 10 Mbp i.i.d. genome with 1% substitutions
(uniform offsets and strands), blocks of 2^24 suffixes, 32-bit indices -- a
synthetic stand-in shaped like the paper's short-read set.

``value`` is timed with CUDA events on the library's stream, inputs already in
HBM; between timed steps a 256 MB buffer is written to flush L2 (outside the
timed region).  ``e2e`` times the host-buffer C-ABI call: H2D of the reads
from pinned memory, the build, and the D2H of B.  The same line carries the
other workloads as keys, each timed the same way:

* ``batched``: 2M reads of U[50, 250] bp from a 50 Mbp genome, 64-bit
  indices: the plain per-block pipeline (every step of every block in turn
  on one stream, blocks of 2^24, occurrence sampling 64, eager launches)
  against the batched form (block size, sampling and tile shapes from the autotuner,
  block sorts overlapping the ranking and Insert of earlier blocks, every
  append one CUDA-graph launch), with per-kernel fractions of the HBM peak;
* ``long``: 20k log-normal long reads (mean 10 kbp, 10% errors) from a 100 Mbp
  genome, plain and batched;
* ``served``: a resident index of 20M x 100 bp reads (2 Gbp) under an 8 GB HBM
  budget, then 48 append requests of 10k-1M reads served closed-loop and as
  Poisson streams at 0.5x and 0.9x of the sustained rate (p50/p99 latency),
  a profiled append against the DRAM-resident dictionary, and a 2M-read index
  served from the pinned host tier under a 512 MB budget.

``--impl reference`` times the CPU oracle (a plain single-threaded suffix sort
by direct comparison) on a bounded sample of the same workload.

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
    "radix_downsweep": "shared-memory ranking and staging: 40% issue, 37% DRAM, 0.46 of the copy bandwidth "
                       "alone under ncu, DRAM traffic 0.94 x algorithmic (profiles/radix_downsweep_short-1Mx100.md)",
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="short", choices=["short", "tiny", "wide"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched workload and form")
    ap.add_argument("--no-long", action="store_true", help="skip the long-read workload")
    ap.add_argument("--no-serving", action="store_true", help="skip the served workload")
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


def serving_report(sb, fresh, requests, check=None):
    """Closed loop for the sustained rate, then Poisson arrivals at 0.5x and
    0.9x of it (in requests/s).  Each run serves a freshly built resident
    index (fresh() builds one), so every run starts from the same index
    size; each run reports the index's memory when it ends.  check(idx), if
    given, runs on the closed loop's index after its timing (its result is
    reported under "result_checks")."""
    out = {}
    rates = [None, 0.5, 0.9]
    sustained_rps = None
    for f in rates:
        idx = fresh()
        rate = None if f is None else f * sustained_rps
        r = measure_serving(sb, idx, requests, rate_rps=rate, seed=7 if f is None else int(f * 100))
        hbm, host = sb.sbwt_memory(idx.handle)
        r["memory_after"] = {"hbm": hbm, "host": host}
        if f is None and check is not None:
            r["result_checks"] = check(idx)
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


class Timer:
    """Builds from device-resident reads, timed with CUDA events on the
    library stream; L2 is flushed (a 256 MB write) before every timed step,
    outside the events."""

    def __init__(self, torch, stream, flush):
        self.torch, self.stream, self.flush = torch, stream, flush

    def steps(self, step, k: int, warmup: int):
        torch = self.torch
        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(k)]
        for i in range(k):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(i & 0xFF)
                ev[i][0].record(self.stream)
            step()
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]


def kernel_table(stats, peak):
    """Per-kernel time, launches, algorithmic GB/s and fraction of the HBM peak."""
    out = {}
    for s in sorted((s for s in stats if not s["name"].startswith("host:")), key=lambda s: -s["ms"]):
        gbps = s["bytes"] / (s["ms"] / 1e3) / 1e9 if s["ms"] > 0 else None
        out[s["name"]] = {"launches": s["launches"], "ms_per_step": round(s["ms"], 4),
                          "GBps": round(gbps, 1) if gbps else None, "frac": round(gbps / peak, 3) if gbps else None}
    return out


def profiled_step(sb, idx, step):
    """One untimed step with every kernel bracketed by events."""
    sb.sbwt_reset_kernel_stats(idx.handle)
    sb.sbwt_set_profiling(idx.handle, True)
    step()
    stats = sb.sbwt_get_kernel_stats(idx.handle)
    sb.sbwt_set_profiling(idx.handle, False)
    sb.sbwt_reset_kernel_stats(idx.handle)
    return stats


def host_counts(stats):
    return {s["name"][5:]: s["launches"] for s in stats if s["name"].startswith("host:graph")}


def symbol_counts(B, chunk: int = 1 << 26):
    """Occurrences of each byte value in B, counted a chunk at a time (a
    bincount of the whole array would widen it to 8-byte integers)."""
    counts = np.zeros(256, np.int64)
    for a in range(0, B.size, chunk):
        counts += np.bincount(B[a:a + chunk], minlength=256)
    return counts


def lf_walks(B, parts, k: int = 32, seed: int = 11, block: int = 4096):
    """Walks k sampled reads backwards through B by the LF mapping and
    counts those that spell their read.  Row r (r < m) is read r's
    terminator suffix; from there LF(i) = C[c] + rank(c, i), c = B[i], gives
    the row of the suffix one symbol longer, and the walk ends at the row
    whose B symbol is a terminator (the whole read).  rank comes from symbol
    counts at every `block` rows.  parts: (reads, offsets) pairs in read-id
    order.  Returns (walks that spelled their read, walks)."""
    n = B.size
    counts = symbol_counts(B)
    C = np.concatenate([[0], np.cumsum(counts)[:-1]])
    nb = n // block
    occ = {}
    step = (1 << 26) // block * block  # rows per chunk (whole blocks)
    for c in np.nonzero(counts)[0]:
        per = np.empty(nb, np.int64)
        for a in range(0, nb * block, step):
            z = min(nb * block, a + step)
            per[a // block:z // block] = (B[a:z].reshape(-1, block) == c).sum(axis=1, dtype=np.int64)
        occ[int(c)] = np.concatenate([[0], np.cumsum(per)])
    sizes = [len(o) - 1 for _, o in parts]
    starts = np.cumsum([0] + sizes)
    m = int(starts[-1])
    picks = np.random.default_rng(seed).choice(m, size=min(k, m), replace=False)
    good = 0
    for r in picks:
        pi = int(np.searchsorted(starts, r, side="right")) - 1
        reads, offs = parts[pi]
        j = int(r - starts[pi])
        want = reads[int(offs[j]):int(offs[j + 1])]
        i, out = int(r), []
        for _ in range(want.size + 1):
            c = int(B[i])
            if c == ord("$"):
                break
            out.append(c)
            b = i // block
            i = int(C[c] + occ[c][b] + np.count_nonzero(B[b * block:i] == c))
        good += bytes(out[::-1]) == want.tobytes()
    return good, len(picks)


def result_checks(B, parts):
    """Whole-B checks of an index built from `parts` ((reads, offsets) in
    read-id order): its length, the symbol multiset, the terminator rows
    (row r holds the last symbol of read r) and LF walks of sampled reads."""
    m = sum(len(o) - 1 for _, o in parts)
    bases = sum(int(o[-1]) for _, o in parts)
    expect = np.zeros(256, np.int64)
    lasts = []
    for reads, offs in parts:
        expect += symbol_counts(reads)
        lens = np.diff(offs.astype(np.int64))
        lasts.append(np.where(lens > 0, reads[np.maximum(offs[1:].astype(np.int64) - 1, 0)], ord("$")))
    expect[ord("$")] += m
    good, walks = lf_walks(B, parts)
    return {"length_ok": bool(B.size == bases + m),
            "multiset_ok": bool(np.array_equal(symbol_counts(B), expect)),
            "terminator_rows_ok": bool(np.array_equal(B[:m], np.concatenate(lasts).astype(np.uint8))),
            "lf_walks_ok": f"{good}/{walks}"}


def check_b(B, w):
    """Cheap checks of a benchmarked B that tie the number to a correct
    result (result_checks); any failure stops the run."""
    r = result_checks(B, [(w.reads, w.offsets)])
    assert r["length_ok"], "length differs"
    assert r["multiset_ok"], "symbol multiset differs from the reads"
    assert r["terminator_rows_ok"], "terminator rows differ"
    good, walks = map(int, r["lf_walks_ok"].split("/"))
    assert good == walks, f"LF walks of sampled reads: {r['lf_walks_ok']} spell their read"


def measure_forms(sb, torch, timer, w, local, args, peak, plain_M, candidates, stream, dist=None):
    """The plain per-block pipeline (Algorithm 1's loop: every step of every
    block in turn on one stream, eager launches, blocks of plain_M suffixes,
    occurrence sampling 64) and the batched form (block size and occurrence
    sampling from the autotuner, each block's suffix sort overlapping the
    previous blocks' ranking and Insert, every append one CUDA-graph launch)
    on the same device-resident reads; both must give the same B."""
    d_reads = torch.from_numpy(w.reads).to("cuda")
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).to("cuda")
    out = {"workload": w.name, "reads": w.m, "bases": w.bases, "index_bits": w.index_bits}
    idx = sb.SetBWT(w.alphabet, index_bits=w.index_bits, block_suffixes=plain_M, stream=stream.cuda_stream,
                    device=local)
    sb.sbwt_set_block_overlap(idx.handle, False)

    def step():
        idx.reset()
        idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)

    ms = timer.steps(step, args.steps, args.warmup)
    tot = max_over_ranks(sum(ms), dist)
    kern = kernel_table(profiled_step(sb, idx, step), peak)
    B = idx.bwt()
    check_b(B, w)
    idx.close()
    out["plain"] = {"value": whole_job_mbps(w.bases, 1, args.steps, tot), "unit": UNIT,
                    "ms_per_step": tot / args.steps, "block_suffixes": plain_M, "occ_sampling": 64,
                    "block_overlap": False, "graph_replay": False, "kernels": kern}
    if args.no_batched:
        return out
    idx_b = sb.SetBWT(w.alphabet, index_bits=w.index_bits, stream=stream.cuda_stream, device=local)
    best_M, best_s, tune = sb.sbwt_autotune(idx_b.handle, d_reads.data_ptr(), d_off.data_ptr(), w.m, candidates,
                                            [64, 128, 256])
    best_tiles, tune_tiles = sb.sbwt_autotune_tile_shapes(idx_b.handle, d_reads.data_ptr(), d_off.data_ptr(), w.m)
    sb.sbwt_set_graph_replay(idx_b.handle, True)

    def step_b():
        idx_b.reset()
        idx_b.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)

    sb.sbwt_reset_kernel_stats(idx_b.handle)
    ms_b = timer.steps(step_b, args.steps, args.warmup)
    graphs = host_counts(sb.sbwt_get_kernel_stats(idx_b.handle))
    tot_b = max_over_ranks(sum(ms_b), dist)
    kern_b = kernel_table(profiled_step(sb, idx_b, step_b), peak)
    Bb = idx_b.bwt()
    assert np.array_equal(Bb, B), "batched form differs from the plain pipeline"
    idx_b.close()
    out["batched"] = {"value": whole_job_mbps(w.bases, 1, args.steps, tot_b), "unit": UNIT,
                      "ms_per_step": tot_b / args.steps, "block_suffixes": int(best_M), "occ_sampling": int(best_s),
                      "block_overlap": True, "graph_replay": True, "graph_counts": graphs,
                      "autotune_ms": {f"{k[0]}/{k[1]}": round(v, 3) for k, v in tune.items()},
                      "tile_shapes": {"insert_threads": best_tiles[0], "rank_segment": best_tiles[1]},
                      "autotune_tiles_ms": {f"{k[0]}/{k[1]}": round(v, 3) for k, v in tune_tiles.items()},
                      "kernels": kern_b}
    out["batched_over_plain"] = out["batched"]["value"] / out["plain"]["value"]
    del d_reads, d_off
    return out


def host_link_table(tier_k, h2d, d2h, rnd):
    """The host tier's kernels against the host link (GB/s rates measured on
    the same device): ComputeRanks' block reads all cross the link as random
    32-byte reads.  The staging kernel reads each old block of a chunk over
    the link and writes it to HBM (its counted bytes are both); Insert then
    writes the chunk's output blocks back over the link.  So the link
    carries the output dictionary once in each direction, half the staging
    kernel's counted bytes: staging is held against the H2D rate, Insert's
    write-back against the D2H rate."""
    tiered = {}
    k = tier_k.get("compute_ranks")
    if k and k["GBps"]:
        tiered["compute_ranks"] = {"GBps": k["GBps"], "ms": k["ms_per_step"], "link_GBps": k["GBps"],
                                   "frac_of_link": round(k["GBps"] / rnd, 3), "link_roofline": "random 32-byte reads"}
    st, mg = tier_k.get("insert_stage"), tier_k.get("insert_merge")
    if st and st["GBps"]:
        link_bytes = st["GBps"] * 1e9 * st["ms_per_step"] / 1e3 / 2
        tiered["link_bytes_per_direction"] = int(link_bytes)
        for name, k, rate, roof in (("insert_stage", st, h2d, "H2D copy (old blocks read over the link)"),
                                    ("insert_merge", mg, d2h, "D2H copy (output blocks written over the link)")):
            if k and k["ms_per_step"] > 0:
                lg = link_bytes / (k["ms_per_step"] / 1e3) / 1e9
                tiered[name] = {"GBps": k["GBps"], "ms": k["ms_per_step"], "link_GBps": round(lg, 1),
                                "frac_of_link": round(lg / rate, 3), "link_roofline": roof}
    return tiered


def measure_served(sb, torch, w_res, requests, local, stream, peak):
    """The serving workload: a resident index of the 20M x 100 bp reads
    under an 8 GB HBM budget, then the append requests served closed-loop
    (sustained rate) and as Poisson streams at 0.5x and 0.9x of it; a
    profiled append of the largest request shows ComputeRanks and Insert
    against the DRAM-resident dictionary; a 2M-read index under a 512 MB
    budget serves from the pinned host tier."""
    d_reads = torch.from_numpy(w_res.reads).to("cuda")
    d_off = torch.from_numpy(w_res.offsets.astype(np.int64)).to("cuda")

    def fresh(budget=8 << 30):
        ix = sb.SetBWT(b"ACGT", hbm_budget=budget, index_bits=64, block_suffixes=1 << 25,
                       stream=stream.cuda_stream, device=local)
        ix.append_device(d_reads.data_ptr(), d_off.data_ptr(), w_res.m)
        return ix

    fresh().close()  # sizes the buffers once
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ix = sb.SetBWT(b"ACGT", hbm_budget=8 << 30, index_bits=64, block_suffixes=1 << 25,
                   stream=stream.cuda_stream, device=local)
    with torch.cuda.stream(stream):
        e0.record(stream)
    ix.append_device(d_reads.data_ptr(), d_off.data_ptr(), w_res.m)
    e1.record(stream)
    torch.cuda.synchronize()
    build_ms = e0.elapsed_time(e1)
    hbm, host = sb.sbwt_memory(ix.handle)
    n_rows, _ = ix.size()
    # one profiled append of the largest request into the resident index
    # (sorts not overlapped: each event pair holds one kernel's own run)
    big = max(requests, key=lambda r: len(r[1]))
    sb.sbwt_set_block_overlap(ix.handle, False)
    sb.sbwt_reset_kernel_stats(ix.handle)
    sb.sbwt_set_profiling(ix.handle, True)
    ix.append(*big)
    kern = kernel_table(sb.sbwt_get_kernel_stats(ix.handle), peak)
    ix.close()
    def served_check(ix):
        # the index holds the resident reads, then the requests' reads in
        # arrival order (one submitting thread); reported, not asserted
        try:
            return result_checks(ix.bwt(), [(w_res.reads, w_res.offsets)] + list(requests))
        except Exception as e:
            return {"error": f"{type(e).__name__}: {e}"}

    report = serving_report(sb, fresh, requests, check=served_check)
    out = {"workload": w_res.name, "resident_rows": n_rows, "resident_build_ms": build_ms,
           "resident_build_Mbps": w_res.bases / build_ms / 1e3, "memory_after_build": {"hbm": hbm, "host": host},
           "requests": len(requests), "request_bases": sum(int(o[-1]) for _, o in requests),
           "hbm_budget": 8 << 30, "serving": report,
           "largest_request_append": {"reads": len(big[1]) - 1, "bases": int(big[1][-1]), "kernels": kern}}
    ix_probe = sb.SetBWT(b"ACGT", stream=stream.cuda_stream, device=local)
    bw_all = sb.sbwt_measure_bandwidth(ix_probe.handle)
    ix_probe.close()
    out["bandwidth"] = bw_all
    cr = kern.get("compute_ranks")
    if cr and cr["GBps"]:
        # ComputeRanks reads one random 32-byte sector per LF step: its
        # roofline on a DRAM-resident dictionary is random-read bandwidth
        out["largest_request_append"]["compute_ranks_frac_of_hbm_random_reads"] = round(
            cr["GBps"] / bw_all["hbm_random_32B_GBps"], 3)
    del d_reads, d_off
    torch.cuda.empty_cache()
    # host tier: a 2M-read resident index whose one dictionary lives in
    # pinned host memory under a 512 MB budget, rewritten in place by Insert;
    # its kernels against the host link measured on the same device
    bw = bw_all
    h2d, d2h, rnd = bw["h2d_GBps"], bw["d2h_GBps"], bw["host_random_32B_GBps"]
    m2 = 2_000_000
    small_reads = w_res.reads[: int(w_res.offsets[m2])]
    small_off = w_res.offsets[: m2 + 1]
    ix2 = sb.SetBWT(b"ACGT", hbm_budget=512 << 20, index_bits=64, block_suffixes=1 << 21,
                    stream=stream.cuda_stream, device=local)
    t = time.perf_counter()
    ix2.append(small_reads, small_off)
    build2 = time.perf_counter() - t
    hbm2, host2 = sb.sbwt_memory(ix2.handle)
    n2, _ = ix2.size()
    small_reqs = [r for r in requests if len(r[1]) - 1 <= 100_000][:12]
    sb.sbwt_reset_kernel_stats(ix2.handle)
    sb.sbwt_set_block_overlap(ix2.handle, False)
    sb.sbwt_set_profiling(ix2.handle, True)
    ix2.append(*small_reqs[0])  # one profiled tiered append
    tier_k = kernel_table(sb.sbwt_get_kernel_stats(ix2.handle), peak)
    sb.sbwt_set_profiling(ix2.handle, False)
    sb.sbwt_set_block_overlap(ix2.handle, True)
    rep2 = measure_serving(sb, ix2, small_reqs[1:])
    ix2.close()
    link = bw
    tiered = host_link_table(tier_k, h2d, d2h, rnd)
    out["host_tier"] = {"resident_reads": m2, "hbm_budget": 512 << 20, "build_s": build2,
                        "build_Mbps": int(small_off[-1]) / build2 / 1e6, "memory": {"hbm": hbm2, "host": host2},
                        "host_bits_per_row": 8.0 * host2 / n2, "host_link": link, "tiered_kernels": tiered,
                        "serving": rep2}
    return out


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
    peak, peak_kind = load_peaks()

    w = make_workload(args.workload, rank)
    bases = w.bases
    stream = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    timer = Timer(torch, stream, flush)
    idx = sb.SetBWT(w.alphabet, index_bits=w.index_bits, block_suffixes=w.block_suffixes,
                    stream=stream.cuda_stream, device=local)
    d_reads = torch.from_numpy(w.reads).to("cuda")
    d_off = torch.from_numpy(w.offsets.astype(np.int64)).to("cuda")
    torch.cuda.synchronize()

    def step():
        idx.reset()
        idx.append_device(d_reads.data_ptr(), d_off.data_ptr(), w.m)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    # one untimed step with every kernel timed and the blocks' sorts not
    # overlapped with the other steps, so each event pair holds one kernel's
    # own run: the per-kernel breakdown and the dominant kernel (with the
    # overlap, a kernel of the lower-priority stream also waits for SMs
    # inside its events)
    sb.sbwt_set_block_overlap(idx.handle, False)
    breakdown = [s for s in profiled_step(sb, idx, step) if not s["name"].startswith("host:")]
    sb.sbwt_set_block_overlap(idx.handle, True)
    dominant = max(breakdown, key=lambda s: s["ms"])["name"]

    # timed region: K steps, each bracketed by events on the library stream;
    # inside, only the dominant kernel carries events (for the roofline)
    sb.sbwt_set_profiling_only(idx.handle, dominant)
    sb.sbwt_reset_kernel_stats(idx.handle)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ms_steps = timer.steps(step, args.steps, 0)
    all_stats = sb.sbwt_get_kernel_stats(idx.handle)
    stats = [s for s in all_stats if not s["name"].startswith("host:")]
    host_phases = {s["name"][5:]: s["ms"] / args.steps for s in all_stats if s["name"].startswith("host:")}
    sb.sbwt_set_profiling(idx.handle, False)
    total_ms = max_over_ranks(float(sum(ms_steps)), dist)
    if dist:
        dist.barrier()

    # the result the oracle pins: cheap whole-B checks on this rank
    B = idx.bwt()
    check_b(B, w)

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

        e_ms = max_over_ranks(float(sum(timer.steps(e2e_step, args.steps, max(1, args.warmup)))), dist)
        assert np.array_equal(h_out.numpy(), B)
        e2e = {"value": whole_job_mbps(bases, world, args.steps, e_ms), "unit": UNIT,
               "h2d_bytes_per_step": int(w.reads.nbytes + w.offsets.nbytes),
               "d2h_bytes_per_step": int(bases + w.m)}
    idx.close()
    del d_reads, d_off

    # the other workloads: batched (2M reads of U[50,250] bp, plain pipeline
    # against the batched form), long reads, and the served form on a 2 Gbp
    # resident index
    cands = [1 << 22, 1 << 23, 1 << 24, 1 << 25, 1 << 26]
    batched = long_reads = served = None
    if args.workload == "short" and not args.no_batched:
        wb = readgen.batched(seed_genome=0x14100562 + 3 + 1000 * rank, seed_reads=0x05621410 + 3 + 1000 * rank)
        batched = measure_forms(sb, torch, timer, wb, local, args, peak, 1 << 24, cands, stream)
        if not args.no_cpu_baseline and world == 1:
            batched["cpu_baseline"] = cpu_baseline(wb, 100_000)
        del wb
    if args.workload == "short" and not args.no_long:
        wl = readgen.long(seed_genome=0x14100562 + 4 + 1000 * rank, seed_reads=0x05621410 + 4 + 1000 * rank)
        long_reads = measure_forms(sb, torch, timer, wl, local, args, peak, 1 << 25, cands + [1 << 27], stream)
        if not args.no_cpu_baseline and world == 1:
            long_reads["cpu_baseline"] = cpu_baseline(wl, 1_000)
        del wl
    if args.workload == "short" and not args.no_serving:
        t = time.perf_counter()
        res, reqs = readgen.serving(seed_genome=0x14100562 + 5 + 1000 * rank,
                                    seed_reads=0x05621410 + 5 + 1000 * rank)
        gen_s = time.perf_counter() - t
        served = measure_served(sb, torch, res, reqs, local, stream, peak)
        served["generation_s"] = gen_s
        if not args.no_cpu_baseline and world == 1:
            served["cpu_baseline"] = cpu_baseline(res, 100_000)
        del res, reqs

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    value = whole_job_mbps(bases, world, args.steps, total_ms)
    dom = next(s for s in stats if s["name"] == dominant)
    achieved = dom["bytes"] / (dom["ms"] / 1e3) / 1e9 if dom["ms"] > 0 else 0.0
    per_launch = dom["bytes"] / max(dom["launches"], 1)
    traffic = load_traffic(dom["name"], per_launch)
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": per_launch,
                "avg_launch_us": 1e3 * dom["ms"] / max(dom["launches"], 1)}
    if dom["name"] in LIMITERS:
        roofline["limiter"] = LIMITERS[dom["name"]]
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
        "kernels": kernel_table(breakdown, peak),  # one untimed step, every kernel timed, sorts not overlapped
        "host_ms_per_step": host_phases,
        "batched": batched,
        "long": long_reads,
        "served": served,
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


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
