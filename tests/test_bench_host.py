"""The host side of the benchmark, without a GPU: the whole-job throughput
formula, the traffic record's scaling and staleness check, the clock-sample
summary, and the reference arm (the oracle timed on the host) printing one
JSON line with the contract's keys."""
import argparse
import io
import json
import os
import shutil
from contextlib import redirect_stdout

import pytest

import bench


def test_whole_job_throughput_is_all_ranks_bases_over_the_slowest_time():
    # 100 Mbp per rank, 2 ranks, 5 steps in 1 s: 1000 Mbp/s
    assert bench.whole_job_mbps(100_000_000, 2, 5, 1000.0) == pytest.approx(1000.0)
    assert bench.max_over_ranks(3.5) == 3.5


def test_traffic_scales_by_units_and_names_its_kernel():
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    alg = 16.0 * 1_000_000  # a launch over 1M units
    t = bench.load_traffic(rec["kernel"], alg)
    if t is not None:
        assert t == pytest.approx(alg / rec["algorithmic_bytes_per_unit"] * rec["dram_bytes_per_unit"])
    assert bench.load_traffic("some_other_kernel", alg) is None


def test_traffic_is_null_once_the_kernel_source_changes(tmp_path, monkeypatch):
    with open(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json")) as f:
        rec = json.load(f)
    (tmp_path / "profiles").mkdir()
    csrc = tmp_path / "paper_1410_0562_gb300" / "csrc"
    csrc.mkdir(parents=True)
    shutil.copy(os.path.join(bench.ROOT, "profiles", "ncu_traffic.json"), tmp_path / "profiles")
    for name in rec["source_files"]:
        shutil.copy(os.path.join(bench.ROOT, "paper_1410_0562_gb300", "csrc", name), csrc / name)
    in_tree = bench.load_traffic(rec["kernel"], 16.0)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.load_traffic(rec["kernel"], 16.0) == in_tree  # an unedited copy reads as the tree does
    with open(csrc / rec["source_files"][0], "a") as f:
        f.write("\n// edited\n")
    assert bench.load_traffic(rec["kernel"], 16.0) is None


def test_clock_summary_reads_median_max_and_active_reasons(tmp_path):
    c = bench.Clocks(0)
    c.path = str(tmp_path / "clocks.csv")
    with open(c.path, "w") as f:
        f.write("1965, 2070, Not Active, Not Active, Not Active, Not Active\n")
        f.write("1980, 2070, Not Active, Not Active, Not Active, Active\n")
        f.write("[N/A], 2070, Not Active, Not Active, Not Active, Not Active\n")
        f.write("2010, 2070, Not Active, Not Active, Not Active, Not Active\n")
        f.write("short line\n")
    c.proc = object()  # as if nvidia-smi had been started
    s = c.summary()
    assert s == {"sm_mhz": 1980.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    c.proc = None
    assert c.summary() is None


def test_reference_arm_prints_one_contract_line():
    args = argparse.Namespace(impl="reference", gpus=1, steps=1, warmup=0, workload="tiny")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    lines = [ln for ln in buf.getvalue().splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["value"] > 0 and line["higher_is_better"] is True and line["vs_baseline"] is None
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": bench.UNIT, "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("tiny-1000x100")


def test_reference_arm_is_silent_on_other_ranks(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = argparse.Namespace(impl="reference", gpus=2, steps=1, warmup=0, workload="tiny")
    buf = io.StringIO()
    with redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""


def test_host_link_table_counts_the_bytes_that_cross_the_link():
    # kernel rows as kernel_table gives them (one tiered append)
    tier_k = {"compute_ranks": {"GBps": 90.0, "ms_per_step": 1.0},
              "insert_stage": {"GBps": 400.0, "ms_per_step": 1.0},  # 400 MB counted: 200 MB read + 200 MB written
              "insert_merge": {"GBps": 150.0, "ms_per_step": 2.0}}
    t = bench.host_link_table(tier_k, h2d=200.0, d2h=100.0, rnd=90.0)
    assert t["link_bytes_per_direction"] == 200_000_000
    assert t["compute_ranks"]["frac_of_link"] == pytest.approx(1.0)
    # staging: 200 MB over the link in 1 ms = 200 GB/s, all of the H2D rate
    assert t["insert_stage"]["link_GBps"] == pytest.approx(200.0)
    assert t["insert_stage"]["frac_of_link"] == pytest.approx(1.0)
    # Insert: the same 200 MB written back in 2 ms = 100 GB/s, all of D2H
    assert t["insert_merge"]["link_GBps"] == pytest.approx(100.0)
    assert t["insert_merge"]["frac_of_link"] == pytest.approx(1.0)
    # no staging kernel (the dictionary fits HBM): no link rows for Insert
    assert set(bench.host_link_table({"compute_ranks": tier_k["compute_ranks"]}, 200.0, 100.0, 90.0)) == \
        {"compute_ranks"}


def _parts_and_oracle_bwt():
    """A resident set and two requests (reads of mixed lengths, one empty),
    and B of their concatenation in that order, by the oracle."""
    import numpy as np

    import oracle
    import readgen
    rng = np.random.default_rng(3)
    parts = []
    for n_reads, seed in ((40, 1), (15, 2), (9, 3)):
        reads, off = readgen.uniform_reads(n_reads, 30, seed)
        lens = rng.integers(0, 31, size=n_reads)
        lens[0] = 0
        keep = np.concatenate([reads[int(off[j]):int(off[j]) + int(lens[j])] for j in range(n_reads)])
        parts.append((keep.astype(np.uint8), np.concatenate([[0], np.cumsum(lens)]).astype(np.uint64)))
    reads = np.concatenate([r for r, _ in parts])
    offs, base = [np.uint64(0)], 0
    for r, o in parts:
        offs.extend((o[1:] + np.uint64(base)).tolist())
        base += int(o[-1])
    oracle.build()
    return parts, oracle.bwt(reads, np.array(offs, np.uint64))


def test_result_checks_pass_on_the_oracle_bwt_and_lf_walks_catch_a_swap():
    import numpy as np
    parts, B = _parts_and_oracle_bwt()
    m = sum(len(o) - 1 for _, o in parts)
    r = bench.result_checks(B, parts)
    assert r["length_ok"] and r["multiset_ok"] and r["terminator_rows_ok"]
    assert r["lf_walks_ok"] == "32/32"
    assert bench.lf_walks(B, parts, k=m, block=16) == (m, m)  # several checkpoints
    # two rows past the terminator rows with different symbols swapped: the
    # multiset and the terminator rows still agree, the walks through them do not
    i = m + 5
    j = next(x for x in range(B.size - 1, m, -1) if B[x] != B[i])
    bad = B.copy()
    bad[i], bad[j] = B[j], B[i]
    r = bench.result_checks(bad, parts)
    assert r["multiset_ok"] and r["terminator_rows_ok"]
    good, walks = bench.lf_walks(bad, parts, k=m, block=16)
    assert walks == m and good < m
    # check_b stops the run on it (one part: the whole set as one workload)
    reads = np.concatenate([p[0] for p in parts])
    w = type("W", (), {})()
    w.reads, w.m, w.bases = reads, m, int(reads.size)
    offs = [0]
    for _, o in parts:
        offs.extend((o[1:].astype(np.int64) + offs[-1]).tolist())
    w.offsets = np.array(offs, np.uint64)
    bench.check_b(B, w)
    with pytest.raises(AssertionError):
        bench.check_b(np.concatenate([bad[:m], np.roll(bad[m:], 1)]), w)
