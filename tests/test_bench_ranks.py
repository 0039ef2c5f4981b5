"""Host-side multi-rank logic of bench.py on CPU (gloo, world size 2): replicas, max-over-ranks
time, whole-job throughput; and the reference arm's rank behaviour."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_max, value = bench.combine_ranks(100.0 + 50.0 * rank, 1000, 4)
    q.put((rank, ms_max, value))
    dist.barrier()
    dist.destroy_process_group()


def test_combine_ranks_gloo_two_ranks():
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, ms_max, value in res:
        assert ms_max == 150.0
        assert abs(value - 2 * 1000 * 4 / 0.150) < 1e-6


def test_combine_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    ms, v = bench.combine_ranks(200.0, 10, 2)
    assert ms == 200.0 and abs(v - 100.0) < 1e-9


@pytest.mark.parametrize("rank", [0, 1])
def test_reference_arm_ranks(rank):
    env = dict(os.environ, RANK=str(rank), WORLD_SIZE="2", LOCAL_RANK=str(rank))
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "8",
                        "--steps", "1", "--warmup", "0", "--cpu-targets", "2", "--gpus", "2"],
                       capture_output=True, text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stderr
    if rank == 1:
        assert r.stdout.strip() == ""
    else:
        line = json.loads(r.stdout.strip().splitlines()[-1])
        assert line["impl"] == "reference" and line["value"] > 0
        assert line["cpu_baseline"]["kind"] == "oracle"
        assert line["e2e"]["h2d_bytes_per_step"] == 0
