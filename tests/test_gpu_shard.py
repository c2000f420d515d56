"""One study sharded over two ranks through the library: each rank runs
pt_prepare + pt_maxnull_naive_ex on its rows (shard_rows) and the ranks merge
with the helpers the benchmark uses (gloo here, on host copies). Both ranks
share cuda:0; their kernels are independent (no rank waits on another's
kernels), only the host-side merge exchanges data. The merged maxima, argmax
and counts must equal one call over all rows and the FP64 oracle."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu

N, N1, V, P = 48, 24, 4001, 1001


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch
    import torch.distributed as dist

    from paper_1703_01506_gb300 import binding as B
    from paper_1703_01506_gb300 import shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    torch.cuda.set_device(0)
    X = torch.as_tensor(synth.gaussian_mean_shift(N, V, seed=8)).cuda()
    perms = synth.perms_pcg32(N, P, seed=8)
    a, b = shard.shard_rows(P, world, rank)
    ctx = B.pt_prepare(X, N1)
    mx, am, ct = B.maxnull_naive(ctx, torch.as_tensor(perms[a:b]).cuda(), precision=2)
    ctx.close()
    mx = shard.merge_maxnull(mx.cpu(), P)
    am = shard.merge_maxnull(am.cpu(), P)
    ct = shard.merge_counts(ct.cpu())
    if rank == 0:
        np.save(os.path.join(out_dir, "mx.npy"), mx.numpy())
        np.save(os.path.join(out_dir, "am.npy"), am.numpy())
        np.save(os.path.join(out_dir, "ct.npy"), ct.numpy())
    dist.destroy_process_group()


def test_two_rank_shard_merge_through_library(cuda_lib, tmp_path):
    import torch
    B = cuda_lib
    mp.start_processes(_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    Xh = synth.gaussian_mean_shift(N, V, seed=8)
    perms = synth.perms_pcg32(N, P, seed=8)
    ctx = B.pt_prepare(torch.as_tensor(Xh).cuda(), N1)
    mx1, am1, ct1 = B.maxnull_naive(ctx, torch.as_tensor(perms).cuda(), precision=2)
    ctx.close()
    mx, am, ct = (np.load(tmp_path / f) for f in ("mx.npy", "am.npy", "ct.npy"))
    np.testing.assert_array_equal(mx, mx1.cpu().numpy())     # bit-identical to one call
    np.testing.assert_array_equal(am, am1.cpu().numpy())
    np.testing.assert_array_equal(ct, ct1.cpu().numpy().astype(np.int64))
    ref = oracle.naive(Xh, N1, perms, tie_rel=2.0 * (N + 4) * 2.0 ** -24)
    same = am == ref.argmax
    near = (ref.u_of(ref.maxnull) - ref.u_of(ref.second)) <= 2 * np.max(ref.tau)
    assert np.all(same | near)
    err = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7)
    assert np.all(np.abs(ct - ref.counts.astype(np.int64)) <= ref.near.astype(np.int64))
