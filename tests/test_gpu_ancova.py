"""F of a g-group factor with nuisance covariates on the GPU (pt_maxnull_anova
on a context from pt_prepare_glm) against the FP64 oracle (oracle/ancova.py),
element by element.

The kernels form, per relabelling, M^-1 = (E^T (I - Q Q^T) E)^-1 in FP64, the
g - 1 group sums u = E^T r^ of each voxel's unit-norm residual on [1, Z] from
the tensor-core contraction (BF16 pieces of r^), and B = u^T M^-1 u; the row
maximum and the counts B >= B_obs are taken on B, and the winner's F is
recomputed in FP64. Tolerances:
* maxima to FP32 output rounding (2.5e-7 relative) where the argmax agrees;
* argmax equal unless the oracle's best and runner-up lie within the band;
* counts equal except entries whose B lies within the band of B_obs.
The band of an entry: each u_h carries at most tau = tie_rel ||r^||_1 of
error (the two-sample path's bound for the same pieces), so B moves by at most
2 sum_h |(M^-1 u)_h| tau (+ FP32 rounding of B), computed here in FP64.
"""
import numpy as np
import pytest
import torch

from oracle import ancova as AC
from oracle import glm as G
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu


def tie_rel(precision, n):
    eps24 = 2.0 ** -24
    if precision == 1:
        return 2.0 * (2.0 ** -17 + (n + 4) * eps24)
    return 2.0 * (n + 4) * eps24


def bands(X, sizes, Z, perms, precision):
    """Per entry: B in FP64 and its band (P x v), from the unit residual r^."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    C = G.design_base(Z, n)
    Qb, _ = np.linalg.qr(C)
    R = X - Qb @ (Qb.T @ X)
    nr = np.sqrt((R * R).sum(axis=0))
    with np.errstate(invalid="ignore", divide="ignore"):
        Rh = R / nr
    tau = tie_rel(precision, n) * np.abs(Rh).sum(axis=0)
    Bm = np.empty((len(perms), v))
    band = np.empty((len(perms), v))
    for i, row in enumerate(perms):
        E = AC._indicators(row, sizes)
        M = E.T @ E - (Qb.T @ E).T @ (Qb.T @ E)
        Mi = np.linalg.inv(M)
        U = E.T @ Rh
        W = Mi @ U
        Bm[i] = (U * W).sum(axis=0)
        band[i] = 2.0 * np.abs(W).sum(axis=0) * tau + 1e-6
    return Bm, band


def run(B, X, sizes, Z, perms, precision, mask=None):
    md = None if mask is None else torch.as_tensor(mask.astype(np.uint8)).cuda()
    ctx = B.pt_prepare_glm(torch.as_tensor(np.ascontiguousarray(X)).cuda(), sizes[0], Z, md)
    mx, am, ct = B.pt_maxnull_anova(ctx, torch.as_tensor(perms).cuda(), sizes, precision)
    B.pt_sync(ctx)
    out = (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
           ct.cpu().numpy().astype(np.int64))
    ctx.close()
    return out


def check(X, sizes, Z, perms, got, precision):
    ref = AC.ancova(X, sizes, Z, perms)
    mx, am, ct = got
    Bm, band = bands(X, sizes, Z, perms, precision)
    Bo, band_o = bands(X, sizes, Z, np.arange(X.shape[0])[None, :], precision)
    n = X.shape[0]
    same = am == ref.argmax
    Bbest = AC.b_of_f(ref.maxnull, n, sizes, Z)
    Bsec = AC.b_of_f(ref.second, n, sizes, Z)
    near = (Bbest - Bsec) <= 2.0 * np.nanmax(band, axis=1)
    assert np.all(same | near), np.flatnonzero(~same & ~near)[:10]
    err = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7), float(err[same].max())
    with np.errstate(invalid="ignore"):
        nearc = (np.abs(Bm - Bo) <= band + band_o).sum(axis=0)
    assert np.all(np.abs(ct - ref.counts) <= nearc)
    return ref


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("sizes,q,v,P", [([8, 9, 10], 2, 2000, 300), ([6, 7, 5, 9], 1, 3001, 257),
                                         ([12, 13], 3, 1500, 200),
                                         ([100, 100, 100], 2, 1001, 120)])
def test_ancova_matches_oracle(cuda_lib, precision, sizes, q, v, P):
    n = sum(sizes)
    X = synth.gaussian_mean_shift(n, v, seed=n + v + q)
    rng = np.random.default_rng(n + q)
    Z = rng.standard_normal((n, q))
    X = (X + 0.7 * (Z[:, :1] @ np.ones((1, v)))).astype(np.float32)
    X[:, 4] = np.float32(0.3)                              # no statistic there
    perms = synth.perms_pcg32(n, P, seed=3)
    perms[9] = np.arange(n, dtype=np.int32)                # the observed labelling
    got = run(cuda_lib, X, sizes, Z, perms, precision)
    check(X, sizes, Z, perms, got, precision)
    assert got[2][4] == 0


def test_ancova_two_groups_is_adjusted_t_squared(cuda_lib):
    """g = 2: the maximum of F is the square of the two-sided covariate-adjusted
    t maximum at the same winning voxel (both recomputed in FP64)."""
    B = cuda_lib
    n, n1, v, P = 30, 13, 2500, 300
    X = synth.gaussian_mean_shift(n, v, seed=21)
    Z = np.random.default_rng(22).standard_normal((n, 2))
    perms = synth.perms_pcg32(n, P, seed=23)
    mx, am, _ = run(B, X, [n1, n - n1], Z, perms, 2)
    ctx = B.pt_prepare_glm(torch.as_tensor(X).cuda(), n1, Z)
    tm, ta, _ = B.maxnull_naive(ctx, torch.as_tensor(perms).cuda(), precision=2, two_sided=True)
    ctx.close()
    tm = tm.cpu().numpy().astype(np.float64)
    same = ta.cpu().numpy() == am
    assert np.mean(same) > 0.99
    np.testing.assert_allclose(mx[same], tm[same] ** 2, rtol=1e-6)


def test_ancova_masked_field_bad_rows_and_collinear_groups(cuda_lib):
    B = cuda_lib
    sizes = [9, 9, 12]
    n = sum(sizes)
    X, mask = synth.brain_field(n, 9, grid=(14, 16, 13), center=(7, 8, 6), semi_axes=(6, 7, 5),
                                fwhm=3.0, effect=0.6, effect_radius=3.0, seed=2)
    X, mask = X.numpy(), mask.numpy().astype(bool)
    Z = np.random.default_rng(3).standard_normal((n, 1))
    perms = synth.perms_pcg32(n, 260, seed=2)
    got = run(B, X, sizes, Z, perms, 2, mask)
    check(X[:, mask], sizes, Z, perms, got, 2)
    md = torch.as_tensor(mask.astype(np.uint8)).cuda()
    ctx = B.pt_prepare_glm(torch.as_tensor(X).cuda(), 9, Z, md)
    bad = perms.copy()
    bad[3, 0] = bad[3, 1]
    B.pt_maxnull_anova(ctx, torch.as_tensor(bad).cuda(), sizes, 2)
    with pytest.raises(B.PtError):
        B.pt_sync(ctx)
    with pytest.raises(B.PtError):
        B.pt_maxnull_anova(ctx, torch.as_tensor(perms).cuda(), sizes, 0)   # FP32: unsupported
    mx, _, _ = B.pt_maxnull_anova(ctx, torch.as_tensor(perms).cuda(), sizes, 2)  # still usable
    assert torch.isfinite(mx).all()
    ctx.close()
    # a covariate equal to group 1's indicator under the identity: that row's
    # group columns are dependent on [1, Z], which the next pt_sync reports
    Zc = np.column_stack([Z, np.r_[np.ones(9), np.zeros(n - 9)]])
    ctx = B.pt_prepare_glm(torch.as_tensor(X).cuda(), 12, Zc[::-1].copy(), md)
    rows = np.vstack([perms[:5], np.arange(n - 1, -1, -1, dtype=np.int32)[None, :]])
    B.pt_maxnull_anova(ctx, torch.as_tensor(rows).cuda(), sizes, 2)
    with pytest.raises(B.PtError):
        B.pt_sync(ctx)
    ctx.close()
