"""Multi-rank (replica) path of bench.py on CPU with gloo, world size 2.

Each rank advances its own seeded ensemble (instances shard by rank, no data-path
collective); the job time is the slowest rank's and the work is the sum over ranks.
"""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", init_method="env://")
    t, pts = bench.reduce_ranks(10.0 + rank, 1000 * (rank + 1), True)
    # each rank's seeded ensemble differs (seed 2506 + rank)
    from paper_2506_16045_gb300 import inputs as I
    ens = I.ensemble_1d(count=4, seed=2506 + rank)
    q.put((rank, t, pts, [c.n for c in ens], float(ens[0].params["a"])))
    dist.barrier()
    dist.destroy_process_group()


def test_reduce_ranks_gloo_world2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    for rank, t, pts, ns, a in out:
        assert t == 11.0                 # max over ranks
        assert pts == 3000.0             # sum over ranks
    assert out[0][4] != out[1][4]        # different instances per rank


def test_reference_arm_non_zero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="1", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--steps", "1", "--warmup", "0"], env=env, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""
