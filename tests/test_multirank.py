"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path shards by views with no data-path collective: rank r renders views
r V .. r V + V - 1, the job's step time is the slowest rank's, and the units
(rays, samples) of all ranks are summed.  This runs the same helpers the GPU
benchmark uses, over a gloo process group.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, q) -> None:
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from paper_2310_01881_gb300 import scenes as S
        cfg = S.CONFIGS["c1"]
        _, o, d = bench.workload(cfg, rank, views=2, px=8)
        w_env, r_env, _ = bench._dist()
        bench.barrier()
        t_max = bench.max_over_ranks(1.0 + 2.0 * rank, device="cpu")
        n_sum = bench.sum_over_ranks(float(len(o) + rank), device="cpu")
        q.put((rank, w_env, r_env, o, d, t_max, n_sum))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_views_and_reduce():
    import multiprocessing as mpl
    ctx = mpl.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        r, *rest = q.get(timeout=120)
        out[r] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    from paper_2310_01881_gb300 import scenes as S
    cfg = S.CONFIGS["c1"]
    for r in range(2):
        w_env, r_env, o, d, t_max, n_sum = out[r]
        assert (w_env, r_env) == (2, r)
        ref = [S.view_rays(cfg, 0, 2 * r + v, 8, 8) for v in range(2)]
        np.testing.assert_array_equal(o, np.concatenate([x[0] for x in ref]))
        np.testing.assert_array_equal(d, np.concatenate([x[1] for x in ref]))
        assert t_max == 3.0                                  # the slowest rank
        assert n_sum == float(len(out[0][2]) + len(out[1][2]) + 1)
    assert not np.array_equal(out[0][2], out[1][2])         # different views per rank
