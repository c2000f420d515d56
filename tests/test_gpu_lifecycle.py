"""Context lifetime: pt_destroy returns at once, with the context's work still
queued, and its workspaces are handed to a later context only after that work
has finished (an event recorded on its stream at destroy).

Each round prepares a study, queues the NaivePT call and destroys the context
straight away, alternating between two streams, so later contexts ask the
cache for blocks while earlier work may still run. A block handed out too
early would be overwritten under a running kernel and change its outputs; all
rounds must give the same maxima, argmax and counts, equal to the FP64
oracle's (maxima to FP32 output rounding where the argmax agrees).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu


def test_destroy_with_work_in_flight(cuda_lib):
    B = cuda_lib
    n, n1, v, P = 48, 24, 20000, 3000
    X = synth.gaussian_mean_shift(n, v, seed=21)
    perms = synth.perms_pcg32(n, P, seed=22)
    Xd = torch.as_tensor(X).cuda()
    pd = torch.as_tensor(perms).cuda()
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    opts = B.naive_opts(3)
    outs = []
    for r in range(8):
        st = streams[r % 2]
        with torch.cuda.stream(st):
            mx = torch.empty(P, dtype=torch.float32, device="cuda")
            am = torch.empty(P, dtype=torch.int32, device="cuda")
            ct = torch.empty(v, dtype=torch.int32, device="cuda")
            ctx = B.pt_prepare(Xd, n1, stream=st)
            B.pt_maxnull_naive_ex(ctx, pd, opts, mx, am, ct)
            ctx.close()  # no wait: the call above may still be running
            outs.append((mx, am, ct))
    torch.cuda.synchronize()
    first = [t.cpu().numpy() for t in outs[0]]
    for mx, am, ct in outs[1:]:
        np.testing.assert_array_equal(mx.cpu().numpy(), first[0])
        np.testing.assert_array_equal(am.cpu().numpy(), first[1])
        np.testing.assert_array_equal(ct.cpu().numpy(), first[2])
    ref = oracle.naive(X, n1, perms)
    same = first[1] == ref.argmax
    assert np.mean(same) > 0.99
    err = np.abs(first[0].astype(np.float64) - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7), float(err[same].max())


def test_release_cached_memory_after_deferred_destroy(cuda_lib):
    """pt_release_cached_memory waits for the held-back blocks' work, frees
    them, and later contexts allocate afresh and still compute correctly."""
    B = cuda_lib
    n, n1, v, P = 30, 15, 5000, 500
    X = synth.gaussian_mean_shift(n, v, seed=5)
    perms = synth.perms_pcg32(n, P, seed=6)
    Xd = torch.as_tensor(X).cuda()
    pd = torch.as_tensor(perms).cuda()
    ctx = B.pt_prepare(Xd, n1)
    mx, am, _ = B.maxnull_naive(ctx, pd, precision=3, counts=False, sync=False)
    ctx.close()
    B.pt_release_cached_memory()
    ctx = B.pt_prepare(Xd, n1)
    mx2, am2, _ = B.maxnull_naive(ctx, pd, precision=3, counts=False)
    ctx.close()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(mx.cpu().numpy(), mx2.cpu().numpy())
    np.testing.assert_array_equal(am.cpu().numpy(), am2.cpu().numpy())
