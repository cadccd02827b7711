"""Multi-rank host logic on CPU with two gloo ranks.

Each rank traces its shard of the photon ids (first_photon_id = the shard's
start) -- here with the CPU oracle, the GPU path's host logic being the same
-- and the gathered result equals one run over all ids; the max/sum
reductions the benchmark uses agree across ranks.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, n, out_dir):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import oracle
    import workloads as W
    from paper_1508_07803_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    scene, b = W.lst_workload(n // 5, seed=4)
    lo, cnt = shard.shard(b.n, rank, world)
    part = W.Bundle(np.ascontiguousarray(b.origins[:, lo:lo + cnt]), np.ascontiguousarray(b.dirs[:, lo:lo + cnt]),
                    b.wavelengths[lo:lo + cnt].copy())
    r = oracle.trace(scene, part, seed=9, first_photon_id=lo, n_threads=1)
    parts = [None] * world  # shards differ in size: gather them as objects
    dist.all_gather_object(parts, (r["status"].astype(np.int64), np.ascontiguousarray(r["hit"])))
    bounces = float(r["bounces"].astype(np.int64).sum())
    total = shard.all_reduce_scalar(bounces, "sum")
    slowest = shard.all_reduce_scalar(float(rank + 1), "max")
    if rank == 0:
        np.savez(os.path.join(out_dir, "gathered.npz"), status=np.concatenate([p[0] for p in parts]),
                 hit=np.concatenate([p[1] for p in parts], axis=1), total=total, slowest=slowest)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_reproduce_a_single_run(tmp_path):
    import oracle
    import workloads as W
    from paper_1508_07803_gb300 import shard
    n, world = 2_005, 2
    mp.start_processes(_worker, args=(world, _free_port(), n, str(tmp_path)), nprocs=world, start_method="spawn")
    got = np.load(tmp_path / "gathered.npz")
    scene, b = W.lst_workload(n // 5, seed=4)
    ref = oracle.trace(scene, b, seed=9, n_threads=2)
    assert np.array_equal(got["status"], ref["status"].astype(np.int64))
    assert np.array_equal(got["hit"], ref["hit"])
    assert float(got["total"]) == float(ref["bounces"].astype(np.int64).sum())
    assert float(got["slowest"]) == world
    # the shard ranges are disjoint and cover every photon
    spans = [shard.shard(b.n, r, 3) for r in range(3)]
    assert spans[0][0] == 0 and sum(c for _, c in spans) == b.n
    assert all(spans[k][0] + spans[k][1] == spans[k + 1][0] for k in range(2))
    assert shard.replica_first_id(3, 1000) == 3000
