"""Multi-rank host logic on CPU (gloo, world size 2): token shards cover the
batch exactly once, per-rank products concatenate to the unsharded result bit
for bit (the oracle stands in for each rank's GPU), and the timing reduction
is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import synth
from paper_2505_07329_b300.dist import shard_range, weak_scaling_range

Q = synth.Q60


@pytest.mark.parametrize("total,world", [(10, 2), (11, 2), (1, 2), (0, 3), (4096, 8), (7, 7)])
def test_shards_cover_every_token_once(total, world):
    seen = []
    for r in range(world):
        t0, t1 = shard_range(total, r, world)
        assert 0 <= t1 - t0 <= total // world + 1
        seen += list(range(t0, t1))
    assert seen == list(range(total))


def test_weak_scaling_ranges_are_disjoint():
    assert [weak_scaling_range(5, r) for r in range(3)] == [(0, 5), (5, 10), (10, 15)]


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, outdir):
    import torch.distributed as dist

    import oracle
    from paper_2505_07329_b300.dist import max_over_ranks
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        N, d_in, d_out, T = 64, 150, 9, 11
        W = synth.weights(d_out, d_in, seed=5)
        L = synth.blocks(d_in, N)
        A = synth.uniform_words((T, L, N), Q, 6)
        B = synth.uniform_words((T, L, N), Q, 7)
        t0, t1 = shard_range(T, rank, world)
        a, b = oracle.lwedot_all(W, A[t0:t1], B[t0:t1], Q)  # this rank's shard, no data collective
        np.save(os.path.join(outdir, f"a{rank}.npy"), a)
        np.save(os.path.join(outdir, f"b{rank}.npy"), b)
        m = max_over_ranks(10.0 * (rank + 1))
        np.save(os.path.join(outdir, f"m{rank}.npy"), np.array([m]))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_sharded_products_equal_the_unsharded_result(tmp_path, orc):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    a = np.concatenate([np.load(tmp_path / f"a{r}.npy") for r in range(world)])
    b = np.concatenate([np.load(tmp_path / f"b{r}.npy") for r in range(world)])
    N, d_in, d_out, T = 64, 150, 9, 11
    W = synth.weights(d_out, d_in, seed=5)
    L = synth.blocks(d_in, N)
    ea, eb = orc.lwedot_all(W, synth.uniform_words((T, L, N), Q, 6), synth.uniform_words((T, L, N), Q, 7), Q)
    assert np.array_equal(a, ea) and np.array_equal(b, eb)
    for r in range(world):
        assert float(np.load(tmp_path / f"m{r}.npy")[0]) == 20.0
