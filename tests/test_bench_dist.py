"""Multi-rank host logic of bench.py on CPU (gloo, world size 2).

The method shards into independent replicas (one per GPU, no data-path collective); the only
cross-rank steps are the barrier around the timed region, the max of the timed region and the sum
of the units processed.  These run here on gloo; the GPU launch uses the same functions on NCCL.
"""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r "timed" 10 + r ms and processed 100 (r + 1) triplets
        ms, units = bench.reduce_over_ranks(10.0 + rank, 100 * (rank + 1), "cpu")
        dist.barrier()
        with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
            json.dump({"ms": ms, "units": units}, f)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    for r in range(world):
        got = json.load(open(tmp_path / f"r{r}.json"))
        assert got["ms"] == 11.0  # slowest rank
        assert got["units"] == 300.0  # all ranks' units


def test_reduce_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(7.5, 42) == (7.5, 42.0)


def test_replica_inputs_differ_per_rank():
    """Weak scaling: each rank's replica is an independent seed of the same workload recipe."""
    sys.path.insert(0, ROOT)
    import md_inputs
    a, b = md_inputs.fcc_system(500, 0.8, 1.0, 0.05, md_inputs.config_seed(2, 0)), \
        md_inputs.fcc_system(500, 0.8, 1.0, 0.05, md_inputs.config_seed(2, 1))
    assert a.L == b.L and a.x.shape == b.x.shape
    assert not np.array_equal(a.x, b.x)


def test_reference_arm_other_ranks_exit_without_work():
    """Under torchrun only rank 0 runs the reference (oracle) arm; rank 1 prints nothing, exits 0."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    p = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=120)
    assert p.returncode == 0, p.stderr
    assert p.stdout.strip() == ""


def test_clock_summary_reads_both_sample_formats():
    """The clock sampler's lines (NVML or nvidia-smi CSV): median SM clock, maximum, and the throttle
    reasons that were active in any sample."""
    import bench
    lines = ["1995, 2070, , 0x4, Not Active, Not Active, Not Active, Active",
             "2070, 2070, 512.3, 0x0, Not Active, Not Active, Not Active, Not Active",
             "2070, 2070, 514.0, Not Active, Not Active, Not Active, Not Active, Not Active",
             "garbage"]
    c = bench.clock_summary(lines)
    assert c["sm_mhz"] == 2070.0 and c["sm_max_mhz"] == 2070.0
    assert c["reasons"] == ["sw_power_cap"] and c["samples"] == 3
    assert bench.clock_summary([])["sm_mhz"] is None


def test_profiled_traffic_counts_only_for_the_captured_source(tmp_path, monkeypatch):
    """roofline.traffic comes from a profile summary only while the kernel's source hash is the one
    recorded at capture; any later change to the source makes it stale (reported as null)."""
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "kernel.cu"
    src.write_text("__global__ void k() {}\n")
    prof = tmp_path / "profiles"
    prof.mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    monkeypatch.setattr(bench, "PROFILES", str(prof))
    monkeypatch.setattr(bench, "KERNEL_SOURCES", {"k": ["kernel.cu"]})
    assert bench.profiled_traffic("k") == (None, "no capture in profiles/")
    rec = {"kernel": "k", "dram_bytes_per_launch": 1234, "source_sha256": bench.source_hash("k")}
    (prof / "k_case.md").write_text("# k\n\ntraffic: " + json.dumps(rec) + "\n")
    assert bench.profiled_traffic("k") == (1234.0, "k_case.md")
    src.write_text("__global__ void k() { /* changed */ }\n")
    val, why = bench.profiled_traffic("k")
    assert val is None and why.startswith("stale")


def test_cpu_linked_cell_line_on_a_small_workload():
    """The bench's linked-cell CPU entry: its configuration keys, rates and a plausible triplet count
    per evaluation (averaged over the run; the exact count is pinned in tests/test_cpu_cells.py)."""
    sys.path.insert(0, ROOT)
    import bench
    import md_inputs
    import oracle
    w = md_inputs.small_fcc_1k()
    line = bench.cpu_linked_cell(w)
    assert line["cores"] >= 1 and set(line) >= {"kind", "cores", "cpu_model", "fcc1k", "fcc100k"}
    for key in ("fcc1k", "fcc100k"):
        r = line[key]
        assert r["n"] == 1000 and r["triplets_per_s"] > 0 and r["rrespa_steps_per_s"] > 0
        assert 0 < r["lj_share"] < 1 and 0 < r["atm_share"] < 1 and r["atm_only_triplets_per_s"] > 0
    _, _, _, cnt = oracle.atm_brute(w.x, w.L, w.nu, w.rc3)
    assert abs(line["fcc1k"]["triplets_per_eval"] - cnt) < 0.05 * cnt  # the lattice start relaxes: a few %
