"""Multi-rank sharding on CPU (gloo, world size 2): the partition balances
pixels, every pair is scored exactly once, and the gathered scores equal a
single-process run.  Per-rank scoring uses the FP64 oracle (CPU), standing in
for each rank's GPU."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2101_06354_gb300 import shard


def test_partition_balances_and_covers():
    sizes = [(1080, 1920)] * 5 + [(360, 640)] * 11 + [(2160, 3840)] * 2 + [(177, 203)]
    for world in (1, 2, 3, 4, 8):
        parts = shard.partition(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i][0] * sizes[i][1] for i in p) for p in parts]
        biggest = max(h * w for h, w in sizes)
        assert max(loads) - min(loads) <= biggest
    assert shard.partition(sizes, 2) == shard.partition(sizes, 2)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_2101_06354_gb300 import synth

    xs, ys = synth.ragged_pairs_u8(sizes)
    mine = shard.partition(sizes, world)[rank]
    local = torch.tensor([oracle.ssim(xs[i].numpy(), ys[i].numpy())[0] for i in mine], dtype=torch.float64)
    full = shard.gather_scores(local, mine, len(sizes))
    if rank == 0:
        np.save(out_path, full.numpy())
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_gather_equals_single_process(tmp_path):
    sizes = [(40, 52), (33, 33), (64, 20), (25, 90), (48, 48), (17, 31), (80, 40)]
    out = str(tmp_path / "scores.npy")
    mp.start_processes(_worker, args=(2, _free_port(), sizes, out), nprocs=2, join=True, start_method="spawn")
    got = np.load(out)
    import oracle
    from paper_2101_06354_gb300 import synth

    xs, ys = synth.ragged_pairs_u8(sizes)
    ref = np.array([oracle.ssim(x.numpy(), y.numpy())[0] for x, y in zip(xs, ys)])
    assert not np.isnan(got).any()
    np.testing.assert_array_equal(got, ref)
