"""The N > 1 bench path on CPU: two gloo ranks (replicas only, no data-path collective).
Checks the barrier, the max-over-ranks time and the sum-over-ranks work used for the
whole-job value, and that each replica builds the same seeded input."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import graphgen as gg
    bench.barrier(world)
    t = bench.max_over_ranks(1.0 + rank, world)
    w = bench.sum_over_ranks(10.0 * (rank + 1), world)
    g = gg.rmat(8)
    digest = int(g.colidx.to(torch.int64).sum()) + 31 * g.E
    digests = [None] * world
    dist.all_gather_object(digests, digest)
    out[rank] = (t, w, len(set(digests)))
    dist.destroy_process_group()


def test_two_gloo_ranks_reduce_like_bench():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        t, w, ndig = res[r]
        assert t == 2.0          # max over ranks of 1.0, 2.0
        assert w == 30.0         # 10 + 20
        assert ndig == 1         # identical seeded replicas


def test_reference_arm_runs_on_cpu():
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--scale", "12",
                        "--steps", "2", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_under_torchrun_prints_one_line():
    """Launched like the scaling run (two ranks): rank 0 alone times the oracle and prints the one
    JSON line; the other rank exits 0 without work."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
                        os.path.join(root, "bench.py"), "--impl", "reference", "--scale", "10", "--steps", "2",
                        "--warmup", "1", "--gpus", "2"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
