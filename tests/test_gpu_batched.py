"""pt_maxnull_naive_batched: several studies of different n (hence different
tensor-core tile classes), v and P in one call, against the FP64 oracle and
against one pt_maxnull_naive_ex call per study; graph replay after the
relabelling rows change in place."""
import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

from test_gpu_naive import check, tie_rel

pytestmark = pytest.mark.gpu

# (n, n1, v, P): n_pad 16 .. 400 spans the 256-, 128- and 64-voxel tiles of
# both BF16 modes; v and P ragged against the 128-row blocks and voxel tiles.
STUDIES = [(20, 10, 2000, 1000), (3, 1, 129, 5), (150, 70, 1500, 300), (37, 15, 1007, 257),
           (400, 200, 600, 130), (200, 100, 700, 260)]


def _make(B, studies, seed0=0):
    dev = torch.device("cuda:0")
    out = []
    for k, (n, n1, v, P) in enumerate(studies):
        X = synth.two_group_gaussian(n1, n - n1, v, frac=0.02, effect=1.0, seed=seed0 + 11 * k + n)
        perms = synth.perms_pcg32(n, P, seed=seed0 + 3 + k)
        ctx = B.pt_prepare(torch.as_tensor(X).to(dev).contiguous(), n1)
        out.append(dict(X=X, n1=n1, perms=perms, ctx=ctx,
                        pd=torch.as_tensor(perms).to(dev).contiguous(),
                        mx=torch.empty(P, dtype=torch.float32, device=dev),
                        am=torch.empty(P, dtype=torch.int32, device=dev),
                        ct=torch.empty(v, dtype=torch.int32, device=dev)))
    return out


def _run_batched(B, ss, precision, two_sided=False):
    opts = B.pt_naive_opts(precision, int(two_sided))
    B.pt_maxnull_naive_batched([s["ctx"] for s in ss], [s["pd"] for s in ss], opts,
                               [s["mx"] for s in ss], [s["am"] for s in ss],
                               [s["ct"] for s in ss])
    B.pt_sync(ss[0]["ctx"])
    for s in ss:
        B.pt_sync(s["ctx"])
    return [(s["mx"].cpu().numpy().astype(np.float64), s["am"].cpu().numpy().astype(np.int64),
             s["ct"].cpu().numpy().astype(np.int64)) for s in ss]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("two_sided", [False, True])
def test_batched_matches_oracle_and_single(cuda_lib, precision, two_sided):
    B = cuda_lib
    ss = _make(B, STUDIES)
    got = _run_batched(B, ss, precision, two_sided)
    for (n, n1, v, P), s, g in zip(STUDIES, ss, got):
        ref = oracle.naive(s["X"], n1, s["perms"], two_sided=two_sided,
                           tie_rel=tie_rel(precision, n))
        check(ref, g, precision, ("batched", n, v, P))
        mx, am, ct = B.maxnull_naive(s["ctx"], s["pd"], precision=precision,
                                     two_sided=two_sided)
        # same arithmetic per (relabelling, voxel); max and counts are order-free
        assert np.array_equal(g[0], mx.cpu().numpy().astype(np.float64)), (n, v, P)
        assert np.array_equal(g[1], am.cpu().numpy().astype(np.int64)), (n, v, P)
        assert np.array_equal(g[2], ct.cpu().numpy().astype(np.int64)), (n, v, P)
    for s in ss:
        s["ctx"].close()


def test_batched_graph_replay_sees_new_rows(cuda_lib):
    """Second call with the same buffers replays the captured graph; rows
    rewritten in place between the calls are read by the replay."""
    B = cuda_lib
    studies = STUDIES[:4]
    ss = _make(B, studies, seed0=50)
    _run_batched(B, ss, 2)
    l0 = B.pt_kernel_launch_count()
    for k, s in enumerate(ss):
        n = s["X"].shape[0]
        s["perms"] = synth.perms_pcg32(n, s["pd"].shape[0], seed=900 + k)
        s["pd"].copy_(torch.as_tensor(s["perms"]))
    got = _run_batched(B, ss, 2)
    assert B.pt_kernel_launch_count() > l0  # replayed kernels are counted
    for (n, n1, v, P), s, g in zip(studies, ss, got):
        ref = oracle.naive(s["X"], n1, s["perms"], tie_rel=tie_rel(2, n))
        check(ref, g, 2, ("replay", n, v, P))
    for s in ss:
        s["ctx"].close()


def test_batched_study_without_valid_voxels(cuda_lib):
    """A study whose voxels are all constant takes no tensor-core work and
    reports what the single-study call reports."""
    B = cuda_lib
    dev = torch.device("cuda:0")
    ss = _make(B, STUDIES[:2], seed0=70)
    n, n1, v, P = 12, 6, 300, 40
    Xc = np.full((n, v), 2.5, dtype=np.float32)
    perms = synth.perms_pcg32(n, P, seed=4)
    ss.append(dict(X=Xc, n1=n1, perms=perms,
                   ctx=B.pt_prepare(torch.as_tensor(Xc).to(dev), n1),
                   pd=torch.as_tensor(perms).to(dev).contiguous(),
                   mx=torch.empty(P, dtype=torch.float32, device=dev),
                   am=torch.empty(P, dtype=torch.int32, device=dev),
                   ct=torch.empty(v, dtype=torch.int32, device=dev)))
    got = _run_batched(B, ss, 2)
    mx, am, ct = B.maxnull_naive(ss[2]["ctx"], ss[2]["pd"], precision=2)
    assert np.array_equal(got[2][1], am.cpu().numpy()) and np.all(got[2][1] == -1)
    assert np.array_equal(got[2][0], mx.cpu().numpy().astype(np.float64))
    assert np.all(got[2][2] == 0)
    for (nn, nn1, vv, PP), s, g in zip(STUDIES[:2], ss[:2], got[:2]):
        ref = oracle.naive(s["X"], nn1, s["perms"], tie_rel=tie_rel(2, nn))
        check(ref, g, 2, ("with-empty", nn, vv, PP))
    for s in ss:
        s["ctx"].close()


def test_batched_bad_arguments(cuda_lib):
    B = cuda_lib
    ss = _make(B, STUDIES[:2], seed0=90)
    ctxs = [s["ctx"] for s in ss]
    args = ([s["pd"] for s in ss], None, [s["mx"] for s in ss], [s["am"] for s in ss])
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_naive_batched(ctxs, args[0], B.pt_naive_opts(0, 0), *args[2:])
    assert e.value.status == B.PT_ERR_UNSUPPORTED
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_naive_batched([ctxs[0], ctxs[0]], args[0], B.pt_naive_opts(2, 0), *args[2:])
    assert e.value.status == B.PT_ERR_INVALID
    # the contexts stay usable
    got = _run_batched(B, ss, 2)
    for (n, n1, v, P), s, g in zip(STUDIES[:2], ss, got):
        ref = oracle.naive(s["X"], n1, s["perms"], tie_rel=tie_rel(2, n))
        check(ref, g, 2, ("after-error", n, v, P))
    for s in ss:
        s["ctx"].close()
