"""Sharding relabellings across two ranks (gloo, CPU): the merged maxima and
counts equal a single-process run. Per-rank compute is the FP64 oracle here
(no GPU); the sharding and merge logic is what the GPU ranks use."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1703_01506_gb300 import shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    import oracle
    from paper_1703_01506_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n, n1, v, P = 16, 8, 300, 101
    X = synth.gaussian_mean_shift(n, v, seed=3)
    perms = synth.perms_pcg32(n, P, seed=1)
    a, b = shard.shard_rows(P, world, rank)
    r = oracle.naive(X, n1, perms[a:b])
    mx = shard.merge_maxnull(torch.tensor(r.maxnull), P)
    am = shard.merge_maxnull(torch.tensor(r.argmax.astype(np.int32)), P)
    ct = shard.merge_counts(torch.tensor(r.counts.astype(np.int32)))
    if rank == 0:
        np.save(os.path.join(out_dir, "mx.npy"), mx.numpy())
        np.save(os.path.join(out_dir, "am.npy"), am.numpy())
        np.save(os.path.join(out_dir, "ct.npy"), ct.numpy())
    dist.destroy_process_group()


def test_shard_rows_cover_exactly():
    for P in (1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            rows = [shard.shard_rows(P, world, r) for r in range(world)]
            assert rows[0][0] == 0 and rows[-1][1] == P
            assert all(rows[i][1] == rows[i + 1][0] for i in range(world - 1))


def test_two_rank_gloo_merge_equals_single(tmp_path):
    import oracle
    from paper_1703_01506_gb300 import synth
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    n, n1, v, P = 16, 8, 300, 101
    X = synth.gaussian_mean_shift(n, v, seed=3)
    perms = synth.perms_pcg32(n, P, seed=1)
    ref = oracle.naive(X, n1, perms)
    np.testing.assert_array_equal(np.load(tmp_path / "mx.npy"), ref.maxnull)
    np.testing.assert_array_equal(np.load(tmp_path / "am.npy"), ref.argmax.astype(np.int32))
    np.testing.assert_array_equal(np.load(tmp_path / "ct.npy"), ref.counts.astype(np.int64))
