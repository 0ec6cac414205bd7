"""Multi-rank (replica) path on CPU with gloo, world size 2: disjoint env
ranges per rank, the slowest rank's time, and whole-job throughput."""
import os

import numpy as np
import torch.multiprocessing as mp

from paper_2412_13211_b300 import replicas, scenes


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    start, end = replicas.env_range(8, rank)
    sc, _ = scenes.make_config(2, num_envs=end - start, env_start=start)
    t = 1.0 + rank                        # rank 1 is the slow one
    worst = replicas.slowest(t)
    out[rank] = (start, end, worst, float(sc.pos[:, 0].sum()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_envs_and_slowest_time():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + os.getpid() % 1000
        ctx_procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
        for p in ctx_procs:
            p.start()
        for p in ctx_procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:2] == (0, 8) and res[1][:2] == (8, 16)
    assert res[0][2] == res[1][2] == 2.0
    assert res[0][3] != res[1][3]         # different envs per rank
    assert replicas.job_throughput(8, 10, 2.0, 2) == 80.0


def test_single_process_slowest_is_identity():
    assert replicas.slowest(3.5) == 3.5
    assert replicas.env_range(4096, 3) == (3 * 4096, 4 * 4096)
    sc_a, _ = scenes.make_config(2, num_envs=2, env_start=0)
    sc_b, _ = scenes.make_config(2, num_envs=4, env_start=0)
    np.testing.assert_array_equal(sc_a.pos, sc_b.pos[:sc_a.num_bodies])
