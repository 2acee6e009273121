"""The multi-rank benchmark path on CPU: two gloo ranks, no GPU.

Under torchrun every rank integrates its own independent cluster (seed =
rank) with no data-path collective; the only cross-rank operations are the
barrier around the timed region and the all-reduce MAX of its duration.
These tests run exactly those operations of bench.py on world size 2.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from paper_1411_5234_gb300 import inputs
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    dist.barrier()
    local_ms = 100.0 + 50.0 * rank                 # rank 1 is the slow one
    worst = bench.reduce_max(local_ms, dist, device="cpu")
    value = bench.job_rate(3 * 1024 * 1024, world, worst * 1e-3)
    cl = bench.make_cluster(512, seed=rank)        # the rank's own cluster
    np.save(os.path.join(out_dir, f"r{rank}.npy"),
            np.array([worst, value, cl.pos[0, 0], cl.mass.sum()]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_timing():
    torch = pytest.importorskip("torch")
    import tempfile
    import torch.multiprocessing as mp
    with tempfile.TemporaryDirectory() as d:
        mp.start_processes(_rank_main, args=(2, _free_port(), d), nprocs=2, join=True,
                           start_method="spawn")
        r0, r1 = (np.load(os.path.join(d, f"r{k}.npy")) for k in (0, 1))
    assert r0[0] == r1[0] == 150.0                  # max over ranks
    assert r0[1] == r1[1] == pytest.approx(2 * 3 * 1024 * 1024 / 0.150)
    assert r0[2] != r1[2]                           # independent clusters per rank
    assert r0[3] == pytest.approx(1.0) and r1[3] == pytest.approx(1.0)


def test_single_rank_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(42.0) == 42.0
    assert bench.job_rate(10, 4, 2.0) == 20.0


def test_bench_traffic_follows_the_kernel_source(tmp_path):
    """roofline.traffic is the committed ncu figure only while the kernel
    source it was measured on is unchanged."""
    sys.path.insert(0, ROOT)
    import bench
    import re
    sha = bench.kernel_source_sha(bench.KERNEL_FILES)
    assert sha == bench.kernel_source_sha(bench.KERNEL_FILES)
    text = open(os.path.join(ROOT, "profiles", "force_mixed_n1048576.md")).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha256:\s*([0-9a-f]+)", text)
    assert m is not None and float(m.group(1)) > 0
    got = bench.traffic_from_profile(bench.KERNEL_FILES)
    assert got == (float(m.group(1)) if m.group(2) == sha else None)
    other = tmp_path / "changed_kernel.cuh"
    other.write_text("// a different kernel source\n")
    assert bench.traffic_from_profile(bench.KERNEL_FILES + [str(other)]) is None


def test_random_vectors_are_seeded_and_bounded():
    sys.path.insert(0, ROOT)
    from paper_1411_5234_gb300 import inputs
    a = inputs.random_vectors(4000, 2.0, seed=3, lo=0.5)
    b = inputs.random_vectors(4000, 2.0, seed=3, lo=0.5)
    c = inputs.random_vectors(4000, 2.0, seed=4, lo=0.5)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    r = np.linalg.norm(a, axis=1)
    assert r.min() >= 0.5 and r.max() < 2.0
    assert np.abs(a.mean(0)).max() < 0.1          # isotropic directions


def test_reference_arm_json_line():
    """bench.py --impl reference (the oracle on the host cores) prints one
    JSON line with the contract's keys."""
    import json
    import subprocess
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "1", "--n", "2048"],
                       capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"]
    assert "workload" in line["config"]
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    e2e = line["e2e"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0
    assert e2e["value"] == line["value"] and e2e["unit"] == line["unit"]
