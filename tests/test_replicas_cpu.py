"""The benchmark's multi-process path on CPU (gloo, two ranks).

The path shards by replica: every rank runs its own copy of the workload on its own
GPU with no collective on the data path; the job's clock is the slowest rank's timed
region and its throughput counts every rank's sources.  These tests run the
aggregation across two gloo processes, and check that the reference arm prints only
on rank 0; and the benchmark's roofline arithmetic (host logic, no GPU).
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [12.5, 20.0][rank]                      # the second replica is slower
    slowest = bench.max_over_ranks(ms, world)
    value = bench.whole_job_value(200, world, slowest)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ms": slowest, "value": value}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_value(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    got = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for g in got:
        assert g["ms"] == 20.0                   # every rank sees the slowest replica's time
        assert g["value"] == pytest.approx(200 * 2 / 20.0e-3)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1) == 7.5
    assert bench.whole_job_value(200, 1, 40.0) == pytest.approx(5000.0)


def test_reference_arm_prints_on_rank_zero_only(tmp_path):
    # rank 1 of a two-rank reference run does no work and prints nothing; rank 0 prints one
    # JSON line (a tiny workload keeps the oracle's sample short)
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--workload", "small"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
    env.update(RANK="0", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0", "--workload", "small"],
                       capture_output=True, text=True, env=env, cwd=ROOT, timeout=300)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2


def test_roofline_arithmetic_and_traffic_validity():
    # the ALU roofline is the shorter of the FP32 and MUFU times for the stated op counts;
    # the DRAM figure is the captured bytes over the measured time; the captured bytes are
    # reported only while the kernel's sources hash to the captured version
    sys.path.insert(0, ROOT)
    import bench
    peaks = {"fp32_fma_per_s": 3.0e13, "fp32x2_fma_per_s": 4.0e13, "mufu_rsqrt_per_s": 5.0e12,
             "mufu_sin_per_s": 6.0e12}
    r = bench.roofline_one("fit", 2.0, 1.0e10, 0.0, peaks)
    t_fp32 = 6.0 * 1.0e10 / 4.0e13
    t_mufu = 1.0 * 1.0e10 / 5.0e12
    assert r["limiting_unit"] == "mufu" and r["frac"] == pytest.approx(max(t_fp32, t_mufu) / 2.0e-3)
    assert r["achieved"] == pytest.approx(1.0e10 / 2.0e-3 / 1e9)
    r5 = bench.roofline_one("fit", 2.0, 1.0e10, 0.0, peaks, fp32=30.0)
    assert r5["limiting_unit"] == "fp32" and r5["frac"] == pytest.approx(30.0 * 1.0e10 / 4.0e13 / 2.0e-3)
    for (name, workload), (files, digest, nbytes) in bench.TRAFFIC.items():
        assert bench.traffic_of(name, workload) in (None, nbytes)
        assert bench.traffic_of(name, "another workload") is None
        if bench.source_hash(files) == digest:
            assert bench.traffic_of(name, workload) == nbytes
            rw = bench.roofline_one(name, 2.0, 1.0e10, 0.0, peaks, workload=workload)
            assert rw["traffic"] == nbytes
            if bench.hbm_peak_gbs():
                assert rw["dram_gb_s"] == pytest.approx(nbytes / 2.0e-3 / 1e9)
