"""Multi-process path on the CPU: two gloo ranks each rank a shard of the
kernels (here with the oracle standing in for the per-GPU ranking) and the
gathered answers equal the unsharded answer; shards partition the kernels."""
import os
import socket
import sys

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2301_03636_gb300 import sharding
from paper_2301_03636_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, result_path):
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    widths = (32, 16, 16, 1)
    off = W.make_segments(97, 1, 30, 8)
    desc = W.make_descriptors(int(off[-1]), 8)
    p = W.make_weights(widths, 8, "he", 0.1)
    k_lo, k_hi, r_lo, r_hi, loc = sharding.shard_segments(off, rank, world)
    f, st = oracle.extract_features(desc[r_lo:r_hi], 32)
    mu, sg = np.zeros(32), np.full(32, 4.0)
    y = oracle.mlp_forward(f, widths, p, mu, sg, st)
    best, _ = oracle.select_best(y, loc)
    sizes = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(sizes, torch.tensor([len(best)]))
    mx = int(max(s.item() for s in sizes))
    buf = torch.full((mx,), -9, dtype=torch.int32)
    buf[:len(best)] = torch.from_numpy(best)
    gathered = [torch.zeros(mx, dtype=torch.int32) for _ in range(world)]
    dist.all_gather(gathered, buf)
    if rank == 0:
        allb = np.concatenate([g[:int(s.item())].numpy() for g, s in zip(gathered, sizes)])
        f, st = oracle.extract_features(desc, 32)
        ref, _ = oracle.select_best(oracle.mlp_forward(f, widths, p, mu, sg, st), off)
        np.save(result_path, np.stack([allb, ref]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_sharded_ranking(tmp_path):
    out = str(tmp_path / "res.npy")
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    allb, ref = np.load(out)
    assert np.array_equal(allb, ref)


def test_shards_partition_kernels():
    off = W.make_segments(1000, 4, 64, 2)
    for world in (1, 2, 3, 8):
        ks, rows = [], 0
        for r in range(world):
            k_lo, k_hi, r_lo, r_hi, loc = sharding.shard_segments(off, r, world)
            ks.extend(range(k_lo, k_hi))
            assert loc[0] == 0 and loc[-1] == r_hi - r_lo
            rows += r_hi - r_lo
        assert ks == list(range(1000)) and rows == off[-1]
    # balanced by rows within one kernel's size
    sizes = [sharding.shard_segments(off, r, 4)[3] - sharding.shard_segments(off, r, 4)[2] for r in range(4)]
    assert max(sizes) - min(sizes) <= 2 * 64


def test_bench_job_is_sharded_by_the_library():
    """bench.py's multi-GPU job: `world` seeded batches split by
    sharding.shard_segments; rank r gets batch r whole, and one rank alone gets
    the single-GPU workload."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2301_03636_gb300 import workloads as W
    off1 = bench.WL.offsets()
    n1 = int(off1[-1])
    off, desc, n_g = bench.global_job_shard(1, 0)
    assert n_g == n1 and np.array_equal(off, off1)
    assert np.array_equal(desc, W.make_descriptors(n1, bench.WL.seed))
    for r in range(3):
        off, desc, n_g = bench.global_job_shard(3, r)
        assert n_g == 3 * n1 and np.array_equal(off, off1)
        assert np.array_equal(desc, W.make_descriptors(n1, bench.WL.seed + 1000 * r))
