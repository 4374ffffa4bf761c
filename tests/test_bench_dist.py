"""The benchmark's multi-GPU path on CPU: two gloo ranks.

Characters are independent, so every rank evaluates its own batch (same
skeletons and clips, its own times and blend weights) and the only
cross-rank operation is the maximum of the timings.  These checks run the
rank logic of bench.py with the gloo backend."""
import os

import numpy as np
import pytest


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w = bench.rank_workload(rank)
    t = 1.0 + rank  # stand-in for a rank's measured milliseconds
    m = bench.aggregate_max(t, world)
    bench.barrier(world)
    q.put((rank, m, float(w["time"][0]), len(w["char_type"]), [len(x["parents"]) for x in w["types"]]))
    dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + (os.getpid() % 2000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, m0, t0, n0, s0), (r1, m1, t1, n1, s1) = res
    assert m0 == m1 == 2.0          # the max over ranks reaches every rank
    assert n0 == n1 and s0 == s1    # same workload shape on every rank (weak scaling)
    assert t0 != t1                 # independent batches


def test_single_rank_helpers():
    import bench
    assert bench.aggregate_max(3.5, 1) == 3.5
    w = bench.rank_workload(0)
    assert bench.frame_algorithmic_bytes(w) > 48 * 2_000_000
    assert len(bench.kernel_source_hash()) == 16


def test_roofline_helpers():
    """The nominal-peak fractions sit beside every HBM roofline object, and
    the frame's touched bytes count 228 B per joint."""
    import bench
    r = {"roofline": {"unit": "GB/s", "achieved": 790.0},
         "fwd_bwd": {"roofline": {"unit": "GB/s", "achieved": 395.0}},
         "other": {"roofline": {"unit": "TFLOP/s", "achieved": 1.0}}}
    bench.add_nominal_fractions(r)
    assert r["roofline"]["frac_of_nominal"] == 0.1
    assert r["fwd_bwd"]["roofline"]["frac_of_nominal"] == 0.05
    assert "frac_of_nominal" not in r["other"]["roofline"]
    w = bench.rank_workload(0)
    joints = sum(len(w["types"][t]["parents"]) for t in w["char_type"])
    assert bench.frame_touched_bytes(w) == joints * 228


def test_source_hash_ignores_comments_only(tmp_path, monkeypatch):
    """The stored ncu traffic is keyed by a hash of the frame kernel's
    sources that a comment edit leaves alone and a code edit changes."""
    import shutil
    import bench
    src = os.path.join(bench.ROOT, "paper_2505_06703_gb300", "csrc")
    dst = tmp_path / "paper_2505_06703_gb300" / "csrc"
    shutil.copytree(src, dst)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    h0 = bench.kernel_source_hash()
    f = dst / "k_scan_qt.cu"
    text = f.read_text()
    f.write_text(text.replace("#include <cuda_runtime.h>", "#include <cuda_runtime.h>  // a comment\n/* and a block */", 1))
    assert bench.kernel_source_hash() == h0
    f.write_text(text.replace("const int cs2 = 2 * n + 1;", "const int cs2 = 2 * n + 2;", 1))
    assert bench.kernel_source_hash() != h0


def test_oracle_on_all_cores_helper():
    """The all-cores CPU baseline: spawned processes each time their share of
    the frame's characters from one start signal; the CPU model is named."""
    import bench
    dt, n = bench.oracle_all_cores(reps=1, warm=1, workers=2)
    assert n == 2 and dt > 0
    assert bench.host_cores() >= 1
    assert bench.cpu_model()


def test_reference_arm_line():
    """bench.py --impl reference: the oracle on the host cores prints the
    contract's line (impl, metric, value, unit, cpu_baseline, e2e)."""
    import argparse
    import bench
    r = bench.run_reference(argparse.Namespace(steps=2, warmup=1))
    assert r["impl"] == "reference" and r["metric"] == bench.METRIC and r["unit"] == bench.UNIT
    assert r["value"] > 0 and r["higher_is_better"] is True and r["steps"] == 2 and r["warmup"] == 1
    cb = r["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == r["value"] and cb["sample"]
    assert r["e2e"] == {"value": r["value"], "unit": r["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
