"""One-way F max-null on the GPU (pt_maxnull_anova) against the FP64 oracle
(oracle/anova.py), element by element.

The kernels form B = SS_between / SS_total from the g - 1 group sums u_h of
the unit-norm centred voxel (FP32 class), take the row maximum of B and the
counts B >= B_obs, and recompute the winner's F in FP64. Tolerances:
* maxima within FP32 output rounding (2.5e-7 relative) where the argmax agrees;
* argmax equal unless the oracle's best and runner-up are within the band;
* counts equal except entries whose B lies within the band of B_obs.
The band: each u_h carries at most tie_rel * ||Xn_j||_1 of error (the
two-sample path's bound), and |u_h| / n_h <= 1, so
B moves by at most 4 g tie_rel ||Xn_j||_1 (+ FP32 rounding of B).
"""
import numpy as np
import pytest
import torch

from oracle import anova as A
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu


def tie_rel(precision, n):
    eps24 = 2.0 ** -24
    if precision == 1:
        return 2.0 * (2.0 ** -17 + (n + 4) * eps24)
    if precision == 3:
        return 2.0 * (2.0 ** -22 + (n + 4) * eps24)
    return 2.0 * (n + 4) * eps24


def run(B, X, sizes, perms, precision, mask=None):
    ctx = B.pt_prepare(torch.as_tensor(np.ascontiguousarray(X)).cuda(), sizes[0],
                       None if mask is None else torch.as_tensor(mask.astype(np.uint8)).cuda())
    mx, am, ct = B.pt_maxnull_anova(ctx, torch.as_tensor(perms).cuda(), sizes, precision)
    B.pt_sync(ctx)
    out = (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
           ct.cpu().numpy().astype(np.int64))
    ctx.close()
    return out


def check(X, sizes, perms, got, precision):
    n, g = X.shape[0], len(sizes)
    ref = A.anova(X, sizes, perms)
    mx, am, ct = got
    Xd = X.astype(np.float64)
    Xc = Xd - Xd.mean(axis=0)
    with np.errstate(invalid="ignore", divide="ignore"):
        l1 = np.abs(Xc).sum(axis=0) / np.sqrt((Xc * Xc).sum(axis=0))
    band = 4.0 * g * tie_rel(precision, n) * np.nan_to_num(l1) + 4e-7
    same = am == ref.argmax
    Bbest = A.b_of_f(ref.maxnull, n, g)
    Bsec = A.b_of_f(ref.second, n, g)
    near = (Bbest - Bsec) <= 2.0 * band.max()
    assert np.all(same | near), np.flatnonzero(~same & ~near)[:10]
    err = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7), float(err[same].max())
    Bij = A.b_of_f(ref.F, n, g)
    Bo = A.b_of_f(ref.F_obs, n, g)
    with np.errstate(invalid="ignore"):
        nearc = (np.abs(Bij - Bo[None, :]) <= 2.0 * band[None, :]).sum(axis=0)
    assert np.all(np.abs(ct - ref.counts) <= nearc)
    return ref


@pytest.mark.parametrize("precision", [0, 2, 3])
@pytest.mark.parametrize("sizes,v,P", [([8, 8, 8], 2000, 300), ([10, 12, 15], 3001, 257),
                                       ([5, 6, 7, 9], 1500, 200), ([3, 4, 2, 5, 6, 3], 1000, 150)])
def test_anova_matches_oracle(cuda_lib, precision, sizes, v, P):
    n = sum(sizes)
    X = synth.gaussian_mean_shift(n, v, seed=n + v)
    X[:, 4] = np.float32(0.3)                      # no statistic there
    perms = synth.perms_pcg32(n, P, seed=3)
    perms[9] = np.arange(n, dtype=np.int32)        # the observed labelling as a row
    got = run(cuda_lib, X, sizes, perms, precision)
    ref = check(X, sizes, perms, got, precision)
    assert got[2][4] == 0


@pytest.mark.parametrize("sizes,precision", [([90, 80, 80], 3), ([140, 140, 140], 3),
                                              ([100, 100, 100], 2), ([60, 70, 60, 60, 50], 3)])
def test_anova_large_n_tiles(cuda_lib, sizes, precision):
    """Large n: the fused F mode on the 128-, 96- and 64-voxel tiles (FP16x2 at
    n = 250 and 420, BF16x3 at n = 300) and with four rows per relabelling."""
    n = sum(sizes)
    v, P = 1301, 140
    X = synth.gaussian_mean_shift(n, v, seed=n)
    perms = synth.perms_pcg32(n, P, seed=7)
    perms[5] = np.arange(n, dtype=np.int32)
    got = run(cuda_lib, X, sizes, perms, precision)
    check(X, sizes, perms, got, precision)


def test_anova_two_groups_is_t_squared(cuda_lib):
    """g = 2: the maximum of F is the square of the two-sided t maximum (both
    recomputed in FP64 at the same winning voxel)."""
    B = cuda_lib
    n, n1, v, P = 30, 12, 2500, 400
    X = synth.gaussian_mean_shift(n, v, seed=5)
    perms = synth.perms_pcg32(n, P, seed=6)
    mx, am, _ = run(B, X, [n1, n - n1], perms, 3)
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    tm, ta, _ = B.maxnull_naive(ctx, torch.as_tensor(perms).cuda(), precision=3, two_sided=True)
    ctx.close()
    tm = tm.cpu().numpy().astype(np.float64)
    same = ta.cpu().numpy() == am
    assert np.mean(same) > 0.99
    np.testing.assert_allclose(mx[same], tm[same] ** 2, rtol=1e-6)


def test_anova_masked_field_and_bad_rows(cuda_lib):
    B = cuda_lib
    sizes = [9, 9, 12]
    n = sum(sizes)
    X, mask = synth.brain_field(n, 9, grid=(14, 16, 13), center=(7, 8, 6), semi_axes=(6, 7, 5),
                                fwhm=3.0, effect=0.6, effect_radius=3.0, seed=2)
    X, mask = X.numpy(), mask.numpy().astype(bool)
    perms = synth.perms_pcg32(n, 260, seed=2)
    got = run(B, X, sizes, perms, 3, mask)
    check(X[:, mask], sizes, perms, got, 3)
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), 9, torch.as_tensor(mask.astype(np.uint8)).cuda())
    bad = perms.copy()
    bad[3, 0] = bad[3, 1]
    B.pt_maxnull_anova(ctx, torch.as_tensor(bad).cuda(), sizes, 3)
    with pytest.raises(B.PtError):
        B.pt_sync(ctx)
    with pytest.raises(B.PtError):
        B.pt_maxnull_anova(ctx, torch.as_tensor(perms).cuda(), [9, 9, 11], 3)   # sizes != n
    mx, _, _ = B.pt_maxnull_anova(ctx, torch.as_tensor(perms).cuda(), sizes, 3)  # still usable
    assert torch.isfinite(mx).all()
    ctx.close()
