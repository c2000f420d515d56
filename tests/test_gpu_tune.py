"""Autotuner of the fused tensor-core kernel (through the C ABI): every
configuration it may record leaves the outputs bit-identical to the default's,
the tuned call still matches the FP64 oracle, and the batched call plans with
the tuned entries."""
import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

from test_gpu_naive import check, tie_rel

pytestmark = pytest.mark.gpu

# (n, n1, v, P): one shape per voxel tile (256, 128, 64), ragged v and P
SHAPES = [(100, 50, 3001, 1000), (37, 15, 1007, 300), (200, 100, 1500, 700),
          (300, 150, 1001, 300)]


def outputs(B, ctx, pd, opts):
    dev = pd.device
    P = pd.shape[0]
    mx = torch.empty(P, dtype=torch.float32, device=dev)
    am = torch.empty(P, dtype=torch.int32, device=dev)
    ct = torch.empty(B.pt_num_voxels(ctx), dtype=torch.int32, device=dev)
    B.pt_maxnull_naive_ex(ctx, pd, opts, mx, am, ct)
    B.pt_sync(ctx)
    return mx.cpu().numpy(), am.cpu().numpy(), ct.cpu().numpy()


def same(a, b):
    return all(np.array_equal(x, y) for x, y in zip(a, b))


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("two_sided", [False, True])
@pytest.mark.parametrize("n,n1,v,P", SHAPES)
def test_configurations_leave_outputs_unchanged(cuda_lib, precision, two_sided, n, n1, v, P):
    B = cuda_lib
    B.pt_tune_clear()
    dev = torch.device("cuda:0")
    X = synth.gaussian_mean_shift(n, v, seed=n + v)
    perms = synth.perms_pcg32(n, P, seed=3)
    ctx = B.pt_prepare(torch.as_tensor(X).to(dev), n1)
    pd = torch.as_tensor(perms).to(dev)
    opts = B.naive_opts(precision, two_sided)
    V = B.pt_num_valid_voxels(ctx)
    base = outputs(B, ctx, pd, opts)
    found, d = B.pt_tune_lookup(n, precision, int(two_sided), V, P)
    assert found == 0
    tried = 0
    for kps in (1, 2, 4, 8):
        for stages in (2, 3, 4, 8):
            for items in (1, 3, 8):
                try:
                    B.pt_tune_set(n, precision, int(two_sided), V, P, d.voxel_tile, stages, kps,
                                  items)
                except B.PtError:
                    continue  # does not fit this n
                assert B.pt_tune_lookup(n, precision, int(two_sided), V, P)[0] == 1
                got = outputs(B, ctx, pd, opts)
                assert same(base, got), (n, kps, stages, items)
                tried += 1
    assert tried >= 12
    B.pt_tune_clear()
    cfg, ms = B.pt_autotune_naive(ctx, pd, opts)
    assert ms > 0.0 and cfg.voxel_tile == d.voxel_tile
    found, rec = B.pt_tune_lookup(n, precision, int(two_sided), V, P)
    assert found == 1 and rec.as_tuple() == cfg.as_tuple()
    assert same(base, outputs(B, ctx, pd, opts))
    ref = oracle.naive(X, n1, perms, two_sided=two_sided, tie_rel=tie_rel(precision, n))
    got = outputs(B, ctx, pd, opts)
    check(ref, tuple(np.asarray(a, dtype=np.float64 if i == 0 else np.int64)
                     for i, a in enumerate(got)), precision, "tuned n=%d" % n)
    ctx.close()
    B.pt_tune_clear()


def test_batched_plans_with_tuned_entries(cuda_lib):
    B = cuda_lib
    B.pt_tune_clear()
    dev = torch.device("cuda:0")
    shapes = [(100, 50, 2500, 600), (200, 100, 1300, 500), (300, 150, 900, 400)]
    ctxs, perms, mx, am, ct = [], [], [], [], []
    for k, (n, n1, v, P) in enumerate(shapes):
        X = synth.gaussian_mean_shift(n, v, seed=50 + k)
        ctxs.append(B.pt_prepare(torch.as_tensor(X).to(dev), n1))
        perms.append(torch.as_tensor(synth.perms_pcg32(n, P, seed=60 + k)).to(dev))
        mx.append(torch.empty(P, dtype=torch.float32, device=dev))
        am.append(torch.empty(P, dtype=torch.int32, device=dev))
        ct.append(torch.empty(v, dtype=torch.int32, device=dev))
    opts = B.naive_opts(2)

    def run():
        B.pt_maxnull_naive_batched(ctxs, perms, opts, mx, am, ct)
        B.pt_sync(ctxs[0])
        return [(m.cpu().numpy(), a.cpu().numpy(), c.cpu().numpy()) for m, a, c in zip(mx, am, ct)]

    before = run()
    singles = [outputs(B, c, p, opts) for c, p in zip(ctxs, perms)]
    B.pt_autotune_naive_batched(ctxs, perms, opts)
    for (n, _, _, P), c in zip(shapes, ctxs):
        assert B.pt_tune_lookup(n, 2, 0, B.pt_num_valid_voxels(c), P)[0] == 1
    after = run()
    again = run()  # graph replay
    for b, a, g, s in zip(before, after, again, singles):
        assert same(b, a) and same(a, g) and same(a, s)
    for c in ctxs:
        c.close()
    B.pt_tune_clear()


def test_autotune_rejects_bad_input(cuda_lib):
    B = cuda_lib
    dev = torch.device("cuda:0")
    n, n1, v, P = 40, 20, 600, 200
    X = synth.gaussian_mean_shift(n, v, seed=9)
    ctx = B.pt_prepare(torch.as_tensor(X).to(dev), n1)
    perms = synth.perms_pcg32(n, P, seed=9)
    pd = torch.as_tensor(perms).to(dev)
    with pytest.raises(B.PtError) as e:
        B.pt_autotune_naive(ctx, pd, B.naive_opts(0))  # FP32 has no tensor-core launch
    assert e.value.status == B.PT_ERR_INVALID
    bad = perms.copy()
    bad[7, 3] = bad[7, 4]  # not a permutation
    with pytest.raises(B.PtError) as e:
        B.pt_autotune_naive(ctx, torch.as_tensor(bad).to(dev), B.naive_opts(2))
    assert e.value.status == B.PT_ERR_INVALID
    assert B.pt_tune_lookup(n, 2, 0, v, P)[0] == 0  # nothing recorded
    # the context stays usable
    got = outputs(B, ctx, pd, B.naive_opts(2))
    ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(2, n))
    check(ref, (got[0].astype(np.float64), got[1].astype(np.int64), got[2].astype(np.int64)), 2,
          "after bad tune")
    ctx.close()
