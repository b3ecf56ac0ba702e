"""Multi-rank path on the CPU: two gloo ranks shard a grid and the shards,
evaluated independently (here by the FP64 oracle), reproduce the full grid;
the job time is the maximum over ranks."""
import os

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1007_1658_gb300 import shard


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    from paper_1007_1658_gb300 import synth
    c = synth.plain_1k()
    f0, df, nf, k = shard.strong_block(c.f0, c.df, 301, rank, world)
    P = oracle.periodogram(c.t, c.X, f0, df, nf)
    t_job = shard.max_over_ranks(1.0 + rank, dist)
    wf0, wdf, wnf = shard.weak_block(c.f0, c.df, 150, rank, world)
    Pw = oracle.periodogram(c.t, c.X, wf0, wdf, wnf)
    np.save(out + "/strong_%d.npy" % rank, P)
    np.save(out + "/weak_%d.npy" % rank, Pw)
    np.save(out + "/time_%d.npy" % rank, np.array([t_job, k]))
    dist.destroy_process_group()


def test_two_gloo_ranks_tile_the_grid(tmp_path):
    import oracle
    from paper_1007_1658_gb300 import synth
    world, port = 2, 29500 + (os.getpid() % 1000)
    mp.spawn(_rank, args=(world, port, str(tmp_path)), nprocs=world, join=True)
    c = synth.plain_1k()
    full = oracle.periodogram(c.t, c.X, c.f0, c.df, 301)
    strong = np.concatenate([np.load(tmp_path / ("strong_%d.npy" % r)) for r in range(world)])
    assert np.allclose(strong, full, rtol=1e-10, atol=1e-12)  # block origins round differently
    weak = np.concatenate([np.load(tmp_path / ("weak_%d.npy" % r)) for r in range(world)])
    assert np.allclose(weak, oracle.periodogram(c.t, c.X, c.f0, c.df, 300), rtol=1e-12, atol=1e-12)
    for r in range(world):
        t_job, k = np.load(tmp_path / ("time_%d.npy" % r))
        assert t_job == 2.0  # max over ranks of 1 + rank
    assert shard.strong_block(0.0, 1.0, 301, 1, 2)[3] == 151


def test_blocks_reject_bad_rank():
    with pytest.raises(ValueError):
        shard.weak_block(0.1, 0.1, 10, 2, 2)
