"""Rows of T (pt_t_rows) against the FP64 oracle, element by element.

The GPU forms u = L . Xn (unit-norm centred data, FP32 accumulation; FP32
CUDA cores or BF16 pieces on the tensor cores) and t = sqrt(k(n-2)) u /
sqrt(1 - k u^2) in FP32; the oracle computes Eq. 5 per entry in FP64. These
are RapidPT's training-row kernels (T_ex).

Tolerances:
* FP32, BF16x3 and FP16x2 (FP32-class; FP16x2 keeps ~22 bits of each
  value): |t_gpu - t| <= 1e-5 max(|t|, 1) (1e-5 relative, absolute floor
  1e-5 near t = 0).
* BF16x2 keeps 16 bits of each data value, so its u carries up to
  tau_j = (2^-17 + (n+4) 2^-24) ||Xn_j||_1 of error; through the map that is
  |dt/du| tau_j = sqrt(k(n-2)) (1 - k u^2)^(-3/2) tau_j, plus FP32 rounding of t.
Voxels without a statistic are NaN.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import rapid as R
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu


def gpu_rows(B, X, n1, perms, precision, mask=None):
    Xd = torch.as_tensor(np.ascontiguousarray(X)).cuda()
    md = None if mask is None else torch.as_tensor(mask.astype(np.uint8)).cuda()
    ctx = B.pt_prepare(Xd, n1, md)
    pd = torch.as_tensor(perms).cuda()
    T = B.pt_t_rows(ctx, pd, precision)
    B.pt_sync(ctx)
    out = T.cpu().numpy().astype(np.float64)
    ctx.close()
    return out


def check_rows(X, n1, perms, T, precision):
    n = X.shape[0]
    ref = oracle.t_rows(X, n1, perms)               # FP64, NaN-free where defined
    valid = R.valid_voxels(X)
    assert np.all(np.isnan(T[:, ~valid]))
    ref, T = ref[:, valid], T[:, valid]
    err = np.abs(T - ref)
    if precision in (0, 2, 3):
        bound = 1e-5 * np.maximum(np.abs(ref), 1.0)
    else:
        k = 1.0 / n1 + 1.0 / (n - n1)
        Xd = X[:, valid].astype(np.float64)
        Xc = Xd - Xd.mean(axis=0)
        l1 = np.abs(Xc).sum(axis=0) / np.sqrt((Xc * Xc).sum(axis=0))
        tau = (2.0 ** -17 + (n + 4) * 2.0 ** -24) * l1
        u = ref / np.sqrt(k * (n - 2) + k * ref * ref)
        dtdu = np.sqrt(k * (n - 2)) / (1.0 - k * u * u) ** 1.5
        bound = dtdu * tau[None, :] + 1e-6 * np.maximum(np.abs(ref), 1.0)
    worst = float(np.max(err / bound))
    assert worst <= 1.0, (precision, worst, float(np.max(err)))
    return float(np.max(err / np.maximum(np.abs(ref), 1.0)))


@pytest.mark.parametrize("precision", [0, 1, 2, 3])
@pytest.mark.parametrize("n,n1,v,P", [(20, 10, 2000, 300), (37, 15, 3001, 257),
                                      (100, 50, 1500, 130), (200, 100, 700, 129)])
def test_t_rows_match_oracle(cuda_lib, precision, n, n1, v, P):
    B = cuda_lib
    X = synth.gaussian_mean_shift(n, v, seed=n + v)
    X[:, 3] = np.float32(0.75)                       # no statistic: NaN row entries
    perms = synth.perms_pcg32(n, P, seed=5)
    T = gpu_rows(B, X, n1, perms, precision)
    rel = check_rows(X, n1, perms, T, precision)
    print("n=%d v=%d P=%d precision=%d: max |dt|/max(|t|,1) = %.3g" % (n, v, P, precision, rel))


@pytest.mark.parametrize("precision", [0, 2, 3])
def test_t_rows_masked_brain_field(cuda_lib, precision):
    """A masked smoothed field in [0, 1] (gray-matter-like values): rows come
    back in masked order."""
    B = cuda_lib
    n, n1, P = 60, 30, 200
    X, mask = synth.brain_field(n, n1, grid=(24, 28, 24), center=(12, 14, 12),
                                semi_axes=(9, 11, 9), fwhm=6.0, effect=0.3, seed=4)
    X, mask = X.numpy(), mask.numpy().astype(bool)
    perms = synth.perms_pcg32(n, P, seed=9)
    T = gpu_rows(B, X, n1, perms, precision, mask=mask)
    check_rows(X[:, mask], n1, perms, T, precision)


def test_t_rows_agree_with_rapid_training_maxima(cuda_lib):
    """The rows' maxima are the training maxima RapidPT reports (the FP64
    winner statistic) to FP32 rounding of t."""
    B = cuda_lib
    n, n1, v, P = 40, 20, 2500, 300
    X = synth.gaussian_mean_shift(n, v, seed=2)
    perms = synth.perms_pcg32(n, P, seed=2)
    T = gpu_rows(B, X, n1, perms, 2)
    ref = oracle.naive(X, n1, perms)
    np.testing.assert_allclose(np.nanmax(T, axis=1), ref.maxnull, rtol=1e-5, atol=1e-5)
