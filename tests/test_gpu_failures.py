"""Failure handling on the GPU without a GPU fault: a device-side wait that
runs out of time (an mbarrier phase nothing completes, short limit) is
reported as PT_ERR_TIMEOUT by pt_sync and leaves the context usable; an
injected host-side allocation failure is reported as PT_ERR_NOMEM and the
library recovers once allocations succeed again."""
import time

import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

from test_gpu_naive import check, tie_rel

pytestmark = pytest.mark.gpu


def _problem(n=30, n1=15, v=800, P=200, seed=4):
    X = synth.gaussian_mean_shift(n, v, seed=seed)
    perms = synth.perms_pcg32(n, P, seed=seed)
    return X, n1, perms


def _parity(B, ctx, X, n1, perms):
    pd = torch.as_tensor(perms).cuda()
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=2)
    ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(2, X.shape[0]))
    check(ref, (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
                ct.cpu().numpy().astype(np.int64)), 2, "after failure")


def test_bounded_wait_times_out_and_context_survives(cuda_lib):
    B = cuda_lib
    X, n1, perms = _problem()
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    t0 = time.perf_counter()
    B.pt_selftest_bounded_wait(ctx, 50)
    with pytest.raises(B.PtError) as e:
        B.pt_sync(ctx)
    dt = time.perf_counter() - t0
    assert e.value.status == B.PT_ERR_TIMEOUT
    assert 0.04 < dt < 1.5, dt  # gave up after about its limit
    B.pt_sync(ctx)  # the status was cleared
    _parity(B, ctx, X, n1, perms)
    with pytest.raises(B.PtError):
        B.pt_selftest_bounded_wait(ctx, 0)  # limit out of range: rejected on the host
    ctx.close()


def test_injected_allocation_failure(cuda_lib):
    B = cuda_lib
    X, n1, perms = _problem()
    Xd = torch.as_tensor(X).cuda()
    try:
        B.pt_debug_fail_allocations(0)
        with pytest.raises(B.PtError) as e:
            B.pt_prepare(Xd, n1)
        assert e.value.status == B.PT_ERR_NOMEM
        B.pt_debug_fail_allocations(-1)
        ctx = B.pt_prepare(Xd, n1)
        _parity(B, ctx, X, n1, perms)
        # a larger call needs new workspaces: they fail, then succeed once allowed
        big = synth.perms_pcg32(X.shape[0], 5000, seed=9)
        pd = torch.as_tensor(big).cuda()
        B.pt_debug_fail_allocations(0)
        with pytest.raises(B.PtError) as e:
            B.maxnull_naive(ctx, pd, precision=2)
        assert e.value.status == B.PT_ERR_NOMEM
    finally:
        B.pt_debug_fail_allocations(-1)
    B.pt_sync(ctx)
    _parity(B, ctx, X, n1, big)
    ctx.close()
