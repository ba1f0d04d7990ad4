"""The multi-rank (replicas) path of the benchmark on CPU: world-size-2 gloo
process groups and a torchrun launch of the reference arm."""
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


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = bench.rank_env()
    slowest = bench.max_over_ranks(10.0 + 7.5 * rank)       # per-rank step times (ms)
    value = bench.replica_value(1000.0, slowest, w)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"rank": r, "world": w, "local": lr, "slowest": slowest, "value": value}, f)


def test_max_over_ranks_and_replica_value(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert (d["rank"], d["world"], d["local"]) == (r, 2, r)
        assert d["slowest"] == 17.5                  # both ranks see the slowest rank's time
        assert d["value"] == pytest.approx(2 * 1000.0 / 17.5e-3)   # all ranks' units / that time


def test_single_process_defaults(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.rank_env() == (0, 1, 0)
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.replica_value(500.0, 2.0, 1) == pytest.approx(250000.0)


def test_reference_arm_under_torchrun():
    """Two ranks: rank 0 alone times the oracle and prints one JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3",
           "--particles", "4096", "--cpu-sample", "256"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_cpu_baseline_thread_count():
    """The one-core CPU sample sets the oracle's OpenMP runtime to one thread,
    reports it, and the caller restores the previous count; the sample counts
    the interactions it timed."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2006_16560_gb300 import inputs
    d = inputs.plummer(4096, 3)
    v_all, _, thr_all, si_all = bench.cpu_oracle_sample(d["pos"], d["mass"], 256)
    prev = bench._omp_threads(1)
    try:
        v1, _, thr1, si1 = bench.cpu_oracle_sample(d["pos"], d["mass"], 256)
    finally:
        bench._omp_threads(prev)
    assert thr1 == 1 and bench._omp_threads() == prev == thr_all
    assert v1 > 0 and v_all > 0 and si1 == si_all > 0       # same sample (seed), same work
