"""The multi-rank (replica) host logic of bench.py, on CPU: two gloo ranks.

Every rank runs the same workload; the timing of the run is its slowest rank (an all-reduce MAX), and the
throughput counts the units of all ranks.  The reference arm runs on rank 0 only; the other ranks exit at once."""
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
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        bench.barrier()
        # rank r took (r + 1) ms for the first quantity and (10 - r) ms for the second
        got = bench.max_over_ranks([rank + 1.0, 10.0 - rank])
        rate = bench.whole_job_rate(1000, world, got[0] * 1e-3)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as fh:
            json.dump({"max": got, "rate": rate}, fh)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for r in range(2):
        with open(tmp_path / f"rank{r}.json") as fh:
            d = json.load(fh)
        assert d["max"] == [2.0, 10.0]
        assert d["rate"] == pytest.approx(2 * 1000 / 2e-3)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([3.0, 4.5]) == [3.0, 4.5]
    assert bench.whole_job_rate(10, 1, 2.0) == 5.0


def _reference_arm(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0", "--ref-block", "1", "--gpus", "2"], capture_output=True, text=True,
                          env=env, cwd=ROOT, timeout=600)


def test_reference_arm_runs_on_rank_zero_only():
    r1 = _reference_arm(1)
    assert r1.returncode == 0 and r1.stdout.strip() == ""
    r0 = _reference_arm(0)
    assert r0.returncode == 0, r0.stderr[-2000:]
    line = json.loads(r0.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["n_gpus"] == 2
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0
