"""Cluster-level summaries on the GPU (pt_cluster_maxnull, pt_cluster_observed)
against the oracle (oracle/cluster.py: FP64 rows of T, scipy's component
labelling).

The GPU decides t >= tau as u >= u(tau) on its FP32-class u, so a voxel whose
t lies within rounding of tau may fall on either side. The largest cluster is
monotone in the threshold, so the GPU's value must lie between the oracle's at
tau + delta and tau - delta (delta = 1e-4, far above the rounding); away from
such voxels the two are equal. The observed map is checked where no voxel
lies within delta of tau: labels and sizes equal, voxel by voxel.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import cluster as C
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu
DELTA = 1e-4


def field(n=30, dims=(16, 18, 15), seed=6):
    X, mask = synth.brain_field(n, n // 2, grid=dims, center=tuple(d // 2 for d in dims),
                                semi_axes=(6.5, 7.5, 6.0), fwhm=4.0, effect=0.9,
                                effect_radius=3.0, seed=seed)
    return X.numpy(), mask.numpy().astype(bool), dims


@pytest.mark.parametrize("conn", [6, 18, 26])
@pytest.mark.parametrize("precision", [0, 2, 3])
def test_cluster_maxnull_matches_oracle(cuda_lib, conn, precision):
    B = cuda_lib
    X, mask, dims = field()
    n, n1 = X.shape[0], X.shape[0] // 2
    perms = synth.perms_pcg32(n, 300, seed=4)
    perms[7] = np.arange(n, dtype=np.int32)  # the observed labelling as one row
    Xm = X[:, mask]
    X[:, np.flatnonzero(mask)[5]] = 0.5       # a constant mask voxel (no statistic)
    Xm = X[:, mask]
    tau = 2.0
    hi = C.cluster_max_sizes(Xm, n1, perms, mask, dims, tau - DELTA, conn)
    lo = C.cluster_max_sizes(Xm, n1, perms, mask, dims, tau + DELTA, conn)
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1, torch.as_tensor(mask.astype(np.uint8)).cuda())
    got = B.pt_cluster_maxnull(ctx, torch.as_tensor(perms).cuda(), tau, dims, conn, precision)
    B.pt_sync(ctx)
    got = got.cpu().numpy().astype(np.int64)
    assert np.all((lo <= got) & (got <= hi)), np.flatnonzero((got < lo) | (got > hi))[:10]
    assert np.mean(lo == hi) > 0.9 and np.all(got[lo == hi] == lo[lo == hi])
    assert got.max() > 5   # the threshold leaves real clusters
    ctx.close()


def test_cluster_extremes_and_batches(cuda_lib):
    """A threshold above every t gives 0; one below every t gives the largest
    connected part of the mask; the relabellings of a ~40k-voxel mask take two
    batches (a batch holds about 2^28 / v relabellings), and the rows on both
    sides of the batch boundary match the oracle."""
    B = cuda_lib
    dims = (48, 56, 48)
    X, mask = synth.brain_field(20, 10, grid=dims, center=(24, 28, 24), semi_axes=(20, 24, 20),
                                fwhm=5.0, seed=8)
    X, mask = X.numpy(), mask.numpy().astype(bool)
    n, n1 = 20, 10
    v = int(mask.sum())
    batch = (2 ** 28 // v) // 128 * 128
    P = batch + 600
    assert batch < P
    perms = synth.perms_pcg32(n, P, seed=9)
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1, torch.as_tensor(mask.astype(np.uint8)).cuda())
    pd = torch.as_tensor(perms).cuda()
    _, sizes = C.label_volume(mask.reshape(dims), 6)
    got = B.pt_cluster_maxnull(ctx, pd, -1e6, dims, 6, 3).cpu().numpy()
    assert np.all(got == sizes.max())
    got = B.pt_cluster_maxnull(ctx, pd, 1e6, dims, 6, 3).cpu().numpy()
    assert np.all(got == 0)
    rows = np.arange(batch - 100, batch + 100)
    Xm = X[:, mask]
    hi = C.cluster_max_sizes(Xm, n1, perms[rows], mask, dims, 2.5 - DELTA, 18)
    lo = C.cluster_max_sizes(Xm, n1, perms[rows], mask, dims, 2.5 + DELTA, 18)
    got = B.pt_cluster_maxnull(ctx, pd, 2.5, dims, 18, 0).cpu().numpy()[rows]
    assert np.all((lo <= got) & (got <= hi))
    assert got.max() > 5
    with pytest.raises(B.PtError):
        B.pt_cluster_maxnull(ctx, pd, 2.5, (48, 56, 47), 6, 3)   # wrong grid
    with pytest.raises(B.PtError):
        B.pt_cluster_maxnull(ctx, pd, 2.5, dims, 8, 3)           # bad connectivity
    ctx.close()


@pytest.mark.parametrize("conn", [6, 26])
def test_cluster_observed_table(cuda_lib, conn):
    B = cuda_lib
    X, mask, dims = field(seed=10)
    n, n1 = X.shape[0], X.shape[0] // 2
    Xm = X[:, mask]
    t = oracle.t_rows(Xm, n1, np.arange(n, dtype=np.int32)[None, :])[0]
    srt = np.sort(t)
    k = np.searchsorted(srt, 1.8)   # a threshold in the widest gap near 1.8
    gaps = srt[k - 20:k + 20][1:] - srt[k - 20:k + 20][:-1]
    g = int(np.argmax(gaps))
    tau = 0.5 * (srt[k - 20 + g] + srt[k - 19 + g])
    assert np.min(np.abs(t - tau)) > DELTA
    want_label, want_size = C.cluster_table(t, mask, dims, tau, conn)
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1, torch.as_tensor(mask.astype(np.uint8)).cuda())
    label, size = B.pt_cluster_observed(ctx, tau, dims, conn)
    B.pt_sync(ctx)
    np.testing.assert_array_equal(label.cpu().numpy(), want_label)
    np.testing.assert_array_equal(size.cpu().numpy(), want_size)
    assert want_size.max() > 5
    ctx.close()
