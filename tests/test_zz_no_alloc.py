"""The allocation-free NaivePT entry point against the regular one.

pt_maxnull_naive_noalloc serves callers that cannot call cudaMalloc (code
inside another runtime's memory pool or a host callback, or under a fixed
memory budget after start-up); its buffers live in one static device array.
It must give what pt_prepare + pt_maxnull_naive (FP32 path) give, within the
tolerances of the other GPU tests, on consecutive calls that reuse the array.
This file is collected last on purpose.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu


def _regular(B, Xd, n1, pd, two_sided):
    ctx = B.pt_prepare(Xd, n1)
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=B.PT_PREC_FP32, two_sided=two_sided)
    ctx.close()
    return mx, am, ct


def _noalloc(B, Xd, n1, pd, two_sided):
    P, v = pd.shape[0], Xd.shape[1]
    mx = torch.full((P,), float("nan"), dtype=torch.float32, device="cuda")
    am = torch.full((P,), -7, dtype=torch.int32, device="cuda")
    ct = torch.full((v,), -7, dtype=torch.int32, device="cuda")
    B.pt_maxnull_naive_noalloc(Xd, n1, pd, mx, am, ct, two_sided=two_sided)
    return mx, am, ct


def _compare(ref_or, a, b):
    """a = regular entry point, b = allocation-free one."""
    mxa, ama, cta = (t.cpu().numpy().astype(np.float64) for t in a)
    mxb, amb, ctb = (t.cpu().numpy().astype(np.float64) for t in b)
    same = ama == amb
    near = (ref_or.u_of(ref_or.maxnull) - ref_or.u_of(ref_or.second)) <= 2 * np.max(ref_or.tau)
    assert np.all(same | near)
    err = np.abs(mxa - mxb) / np.maximum(np.abs(mxa), 1.0)
    assert np.all(err[same] <= 1e-5)
    assert np.all(np.abs(cta - ctb) <= ref_or.near.astype(np.float64))


@pytest.mark.parametrize("two_sided", [False, True])
def test_noalloc_matches_regular_on_two_calls(cuda_lib, two_sided):
    B = cuda_lib
    cases = [(40, 17, 3001, 700, 21), (20, 10, 2000, 1000, 1)]  # second call reuses the array
    for n, n1, v, P, seed in cases:
        X = synth.gaussian_mean_shift(n, v, seed=seed)
        X[:, 5] = 0.25  # a voxel without a t statistic
        perms = synth.perms_pcg32(n, P, seed=seed)
        Xd = torch.as_tensor(X).cuda()
        pd = torch.as_tensor(perms).cuda()
        ref = oracle.naive(X, n1, perms, two_sided=two_sided, tie_rel=2.0 * (n + 4) * 2.0 ** -24)
        a = _regular(B, Xd, n1, pd, two_sided)
        b = _noalloc(B, Xd, n1, pd, two_sided)
        _compare(ref, a, b)
        assert int(b[2][5].item()) == 0


def test_noalloc_rejects_oversize_and_bad_rows(cuda_lib):
    B = cuda_lib
    n, n1 = 100, 50
    X = torch.zeros((n, 400_000), dtype=torch.float32, device="cuda")  # needs > 64 MiB
    perms = torch.as_tensor(synth.perms_pcg32(n, 10, seed=1)).cuda()
    mx = torch.empty(10, dtype=torch.float32, device="cuda")
    am = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_naive_noalloc(X, n1, perms, mx, am)
    assert e.value.status == B.PT_ERR_INVALID and "static limit" in str(e.value)
    Xs = torch.as_tensor(synth.gaussian_mean_shift(n, 500, seed=3)).cuda()
    bad = perms.clone()
    bad[2, 0] = bad[2, 1]
    with pytest.raises(B.PtError):
        B.pt_maxnull_naive_noalloc(Xs, n1, bad, mx, am)
    B.pt_maxnull_naive_noalloc(Xs, n1, perms, mx, am)  # still usable
