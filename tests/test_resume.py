"""Chunked NaivePT with checkpoints: the checkpoint file logic on the host, and
(GPU) an interrupted and resumed run against one call."""
import numpy as np
import pytest
import torch

from paper_1703_01506_gb300 import synth


class _Opts:
    def __init__(self, precision=2, two_sided=0):
        self.precision, self.two_sided = precision, two_sided


def test_checkpoint_round_trip_and_refusals(tmp_path):
    from paper_1703_01506_gb300 import resume as R
    perms = synth.perms_pcg32(30, 200, seed=5)
    d = R.problem_digest(perms, 1000, _Opts())
    assert d != R.problem_digest(perms[:199], 1000, _Opts())
    assert d != R.problem_digest(perms, 1001, _Opts())
    assert d != R.problem_digest(perms, 1000, _Opts(two_sided=1))
    other = perms.copy()
    other[3, [0, 1]] = other[3, [1, 0]]
    assert d != R.problem_digest(other, 1000, _Opts())
    path = str(tmp_path / "ck.npz")
    assert R.load_state(path, d, 200, 1000) is None
    mx = np.arange(200, dtype=np.float32)
    am = np.arange(200, dtype=np.int32)
    ct = np.arange(1000, dtype=np.uint32)
    R.save_state(path, d, 128, mx, am, ct)
    rows, mx2, am2, ct2 = R.load_state(path, d, 200, 1000)
    assert rows == 128
    np.testing.assert_array_equal(mx2, mx)
    np.testing.assert_array_equal(am2, am)
    np.testing.assert_array_equal(ct2, ct)
    with pytest.raises(ValueError):
        R.load_state(path, R.problem_digest(other, 1000, _Opts()), 200, 1000)
    with pytest.raises(ValueError):
        R.load_state(path, d, 300, 1000)  # sizes do not match the saved arrays


@pytest.mark.gpu
@pytest.mark.parametrize("precision", [0, 2])
def test_interrupted_run_resumes_to_the_one_call_result(cuda_lib, tmp_path, precision):
    from paper_1703_01506_gb300 import resume as R
    B = cuda_lib
    n, n1, v, P = 60, 30, 3001, 1000
    X = synth.gaussian_mean_shift(n, v, seed=7)
    perms = synth.perms_pcg32(n, P, seed=7)
    perms[17] = np.arange(n)  # an observed-set row: counted exactly in every chunk
    dev = torch.device("cuda:0")
    ctx = B.pt_prepare(torch.as_tensor(X).to(dev), n1)
    pd = torch.as_tensor(perms).to(dev)
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=precision)
    one = (mx.cpu().numpy(), am.cpu().numpy(), ct.cpu().numpy().astype(np.uint32))
    path = str(tmp_path / "run.npz")
    assert R.maxnull_naive_resumable(ctx, pd, 300, path, precision=precision,
                                     max_chunks=2) is None
    rows, _, _, _ = R.load_state(path, R.problem_digest(pd, v, B.naive_opts(precision)), P, v)
    assert rows == 600
    got = R.maxnull_naive_resumable(ctx, pd, 300, path, precision=precision)
    for a, b in zip(one, got):
        np.testing.assert_array_equal(a, b)
    # a checkpoint of another problem is refused
    with pytest.raises(ValueError):
        R.maxnull_naive_resumable(ctx, pd[:999].contiguous(), 300, path, precision=precision)
    ctx.close()


@pytest.mark.gpu
def test_accumulated_counts_single_and_batched(cuda_lib):
    """accumulate_counts adds a call's exceedances to the counts already in the
    buffer (single-study and batched calls); without it the buffer is replaced."""
    B = cuda_lib
    dev = torch.device("cuda:0")
    shapes = [(40, 20, 1500, 300), (130, 65, 900, 257)]
    ctxs, perms, mxs, ams, cts, halves = [], [], [], [], [], []
    for k, (n, n1, v, P) in enumerate(shapes):
        X = synth.gaussian_mean_shift(n, v, seed=20 + k)
        c = B.pt_prepare(torch.as_tensor(X).to(dev), n1)
        p = torch.as_tensor(synth.perms_pcg32(n, P, seed=30 + k)).to(dev)
        ctxs.append(c)
        perms.append(p)
        mxs.append(torch.empty(P, dtype=torch.float32, device=dev))
        ams.append(torch.empty(P, dtype=torch.int32, device=dev))
        cts.append(torch.empty(v, dtype=torch.int32, device=dev))
        _, _, full = B.maxnull_naive(c, p, precision=2)
        halves.append(full.cpu().numpy())
    acc = B.naive_opts(2, accumulate_counts=True)
    for c, p, mx, am, ct, full in zip(ctxs, perms, mxs, ams, cts, halves):
        h = p.shape[0] // 2
        ct.zero_()
        B.pt_maxnull_naive_ex(c, p[:h].contiguous(), acc, mx[:h], am[:h], ct)
        B.pt_maxnull_naive_ex(c, p[h:].contiguous(), acc, mx[h:], am[h:], ct)
        B.pt_sync(c)
        np.testing.assert_array_equal(ct.cpu().numpy(), full)
    B.pt_maxnull_naive_batched(ctxs, perms, B.naive_opts(2), mxs, ams, cts)
    B.pt_sync(ctxs[0])
    for ct, full in zip(cts, halves):
        np.testing.assert_array_equal(ct.cpu().numpy(), full)
    B.pt_maxnull_naive_batched(ctxs, perms, acc, mxs, ams, cts)
    B.pt_sync(ctxs[0])
    for ct, full in zip(cts, halves):
        np.testing.assert_array_equal(ct.cpu().numpy(), 2 * full)
    for c in ctxs:
        c.close()
