"""GPU NaivePT with nuisance covariates (pt_prepare_glm, through the C ABI)
against the oracle's least-squares statistic (oracle/glm.py), element by
element: maxima (recomputed in FP64 on the GPU, so exact to FP32 output
rounding where the argmax agrees), argmax except at near-ties, counts except
at near-ties, the observed statistic; and the error paths."""
import numpy as np
import pytest
import torch

from oracle import glm
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu

EPS24 = 2.0 ** -24


def tie_rel(precision, n):
    if precision == 1:
        return 2.0 * (2.0 ** -17 + (n + 4) * EPS24)
    return 2.0 * (n + 4) * EPS24


def unit_residuals(X, Z):
    X = np.asarray(X, dtype=np.float64)
    C = glm.design_base(Z, X.shape[0])
    Q, _ = np.linalg.qr(C)
    R = X - Q @ (Q.T @ X)
    nrm = np.linalg.norm(R, axis=0)
    return R / np.where(nrm > 0, nrm, 1.0)


def run(B, X, Z, n1, perms, precision, two_sided):
    dev = torch.device("cuda:0")
    ctx = B.pt_prepare_glm(torch.as_tensor(X).to(dev), n1, Z)
    pd = torch.as_tensor(perms).to(dev)
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=precision, two_sided=two_sided)
    t_obs = torch.empty(B.pt_num_voxels(ctx), dtype=torch.float32, device=dev)
    B.pt_t_obs(ctx, t_obs)
    B.pt_sync(ctx)
    out = (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
           ct.cpu().numpy().astype(np.int64), t_obs.cpu().numpy().astype(np.float64))
    ctx.close()
    return out


def check(ref, got, X, Z, precision, two_sided, name):
    mx, am, ct, t_obs = got
    n = X.shape[0]
    P = mx.shape[0]
    rows = np.arange(P)
    # observed statistic
    ok = ~np.isnan(ref.t_obs)
    assert np.array_equal(np.isnan(t_obs), ~ok), name
    np.testing.assert_allclose(t_obs[ok], ref.t_obs[ok], rtol=2e-6, atol=1e-6, err_msg=name)
    # tie band on the contraction's scale u (group-1 share of the unit residual)
    Rn = unit_residuals(X, Z)
    tau = tie_rel(precision, n) * np.abs(Rn).sum(axis=0)
    band = 2.0 * float(tau.max())
    same = am == ref.argmax
    err = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7), (name, float(err[same].max()))
    gap = ref.u_of(ref.maxnull, rows) - ref.u_of(ref.second, rows)
    bad = ~same & ~(gap <= band)
    assert not bad.any(), (name, np.flatnonzero(bad)[:8])
    du = np.abs(ref.u_of(mx, rows) - ref.u_of(ref.maxnull, rows))
    assert np.all(du[~same] <= band), (name, du[~same])
    # counts: entries whose comparison the rounding can flip
    S = np.abs(ref.T) if two_sided else ref.T
    s_obs = np.abs(ref.t_obs) if two_sided else ref.t_obs
    u = ref.u_of(S, rows[:, None])                       # P x v
    f = np.sqrt(ref.a_obs / ref.a)[:, None]
    u_obs = s_obs / np.sqrt(ref.df + s_obs ** 2) * np.sqrt(ref.a_obs)  # w_obs sqrt(a_obs)
    z = u * f
    near = np.abs(z - u_obs[None, :]) <= (1.0 + f) * tau[None, :] + 2.0 ** -20 * np.abs(u_obs)
    near &= ~np.isnan(z)
    dc = np.abs(ct - ref.counts)
    badc = dc > near.sum(axis=0)
    assert not badc[ok].any(), (name, np.flatnonzero(badc)[:8], dc[badc][:8])
    assert np.all(ct[~ok] == 0), name


SHAPES = [  # (n, n1, v, P, q): one per voxel tile (256, 128, 64), ragged v and P, q = 0
    (40, 20, 1500, 300, 2), (37, 15, 1007, 300, 1), (24, 12, 513, 129, 0),
    (130, 65, 900, 257, 3), (300, 150, 700, 130, 2)]


@pytest.mark.parametrize("precision", [1, 2])
@pytest.mark.parametrize("two_sided", [False, True])
@pytest.mark.parametrize("n,n1,v,P,q", SHAPES)
def test_glm_parity(cuda_lib, precision, two_sided, n, n1, v, P, q):
    rng = np.random.default_rng(n * 7 + q)
    X = synth.two_group_gaussian(n1, n - n1, v, frac=0.03, effect=1.0, seed=n + v + q)
    Z = rng.standard_normal((n, q)) if q else None
    if q:
        X = X + (Z @ rng.uniform(0.5, 2.0, (q, v))).astype(np.float32)  # covariate effects
    X[:, 5] = 3.0  # a constant voxel: no statistic
    perms = synth.perms_pcg32(n, P, seed=q + 3)
    perms[P // 3] = np.arange(n)  # the observed group-1 set: counted exactly
    ref = glm.glm_naive(X, Z, n1, perms, two_sided=two_sided)
    got = run(cuda_lib, X, Z, n1, perms, precision, two_sided)
    check(ref, got, X, Z, precision, two_sided, "n=%d q=%d" % (n, q))


def test_glm_tuned_launch_leaves_outputs_unchanged(cuda_lib):
    B = cuda_lib
    n, n1, v, P, q = 130, 65, 2000, 700, 2
    rng = np.random.default_rng(1)
    X = synth.gaussian_mean_shift(n, v, seed=1)
    Z = rng.standard_normal((n, q))
    dev = torch.device("cuda:0")
    ctx = B.pt_prepare_glm(torch.as_tensor(X).to(dev), n1, Z)
    pd = torch.as_tensor(synth.perms_pcg32(n, P, seed=1)).to(dev)
    base = [t.cpu().numpy() for t in B.maxnull_naive(ctx, pd)]
    B.pt_tune_clear()
    B.pt_autotune_naive(ctx, pd, B.naive_opts(2))
    got = [t.cpu().numpy() for t in B.maxnull_naive(ctx, pd)]
    B.pt_tune_clear()
    for a, b in zip(base, got):
        np.testing.assert_array_equal(a, b)
    ctx.close()


def test_glm_errors(cuda_lib):
    B = cuda_lib
    dev = torch.device("cuda:0")
    n, n1, v = 30, 15, 400
    X = torch.as_tensor(synth.gaussian_mean_shift(n, v, seed=2)).to(dev)
    rng = np.random.default_rng(2)
    Z = rng.standard_normal((n, 2))
    with pytest.raises(B.PtError) as e:  # [1, Z] without full column rank
        B.pt_prepare_glm(X, n1, np.column_stack([Z, Z[:, 0]]))
    assert e.value.status == B.PT_ERR_INVALID
    Zn = Z.copy()
    Zn[3, 1] = np.nan
    with pytest.raises(B.PtError):
        B.pt_prepare_glm(X, n1, Zn)
    g = np.zeros((n, 1))
    g[:n1] = 1.0  # the observed group column itself
    with pytest.raises(B.PtError):
        B.pt_prepare_glm(X, n1, g)
    with pytest.raises(B.PtError):  # too many covariates for the degrees of freedom
        B.pt_prepare_glm(X[:5].contiguous(), 2, rng.standard_normal((5, 3)))
    # a covariate equal to another group-1 set: that relabelling has no statistic
    other = np.zeros((n, 1))
    other[n1:] = 1.0
    other[0] = 1.0
    other[n1] = 0.0
    ctx = B.pt_prepare_glm(X, n1, other)
    perms = synth.perms_pcg32(n, 50, seed=2)
    perms[7] = np.concatenate([np.flatnonzero(other[:, 0] == 1.0), np.flatnonzero(other[:, 0] == 0.0)])
    pd = torch.as_tensor(perms).to(dev)
    mx = torch.empty(50, dtype=torch.float32, device=dev)
    am = torch.empty(50, dtype=torch.int32, device=dev)
    B.pt_maxnull_naive_ex(ctx, pd, B.naive_opts(2), mx, am, None)
    with pytest.raises(B.PtError) as e:
        B.pt_sync(ctx)
    assert e.value.status == B.PT_ERR_INVALID
    # paths that run the plain statistic only
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_naive_ex(ctx, pd, B.naive_opts(0), mx, am, None)
    assert e.value.status == B.PT_ERR_UNSUPPORTED
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_rapid(ctx, pd, 3, 0.2, 10, B.rapid_opts(), mx)
    assert e.value.status == B.PT_ERR_UNSUPPORTED
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_naive_batched([ctx], [pd], B.naive_opts(2), [mx], [am])
    assert e.value.status == B.PT_ERR_UNSUPPORTED
    ctx.close()


def test_glm_masked_field_from_pinned_host_memory(cuda_lib):
    """A masked brain-shaped field with covariates, X and the mask read from
    page-locked host memory: outputs equal the device-memory run and match the
    oracle on the mask voxels (masked-order argmax and counts)."""
    B = cuda_lib
    n, n1, P, q = 28, 14, 300, 2
    X, mask = synth.brain_field(n, n1, grid=(20, 24, 20), center=(10, 12, 10),
                                semi_axes=(8, 10, 8), fwhm=4.0, effect=0.5, effect_radius=3.0,
                                seed=8, device="cpu")
    Z = np.random.default_rng(8).standard_normal((n, q))
    perms = synth.perms_pcg32(n, P, seed=8)
    pd = torch.as_tensor(perms).cuda()
    outs = []
    for host in (False, True):
        Xa = X.contiguous().pin_memory() if host else X.cuda()
        ma = mask.to(torch.uint8).contiguous()
        ma = ma.pin_memory() if host else ma.cuda()
        ctx = B.pt_prepare_glm(Xa, n1, Z, ma)
        mx, am, ct = B.maxnull_naive(ctx, pd, precision=2)
        t_obs = torch.empty(B.pt_num_voxels(ctx), dtype=torch.float32, device="cuda")
        B.pt_t_obs(ctx, t_obs)
        B.pt_sync(ctx)
        outs.append([t.cpu() for t in (mx, am, ct, t_obs)])
        ctx.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)
    Xm = X[:, mask.bool()].numpy()
    ref = glm.glm_naive(Xm, Z, n1, perms)
    mx, am, ct, t_obs = outs[1]
    check(ref, (mx.numpy().astype(np.float64), am.numpy().astype(np.int64),
                ct.numpy().astype(np.int64), t_obs.numpy().astype(np.float64)),
          Xm, Z, 2, False, "masked field")


@pytest.mark.parametrize("two_sided", [False, True])
def test_glm_fwer_pvalues_match_oracle(cuda_lib, two_sided):
    """FWER-corrected p-values (Sec. 2) from the covariate-adjusted max-null and
    t_obs (pt_fwer_pvalues) against the oracle's definition applied to the
    oracle's own max-null and t_obs."""
    import oracle
    B = cuda_lib
    n, n1, v, P, q = 36, 18, 1200, 400, 3
    rng = np.random.default_rng(21)
    X = synth.two_group_gaussian(n1, n - n1, v, frac=0.05, effect=1.5, seed=21)
    Z = rng.standard_normal((n, q))
    perms = synth.perms_pcg32(n, P, seed=21)
    ctx = B.pt_prepare_glm(torch.as_tensor(X).cuda(), n1, Z)
    pd = torch.as_tensor(perms).cuda()
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=2, two_sided=two_sided)
    p = torch.empty(v, dtype=torch.float32, device="cuda")
    B.pt_fwer_pvalues(ctx, mx, p, two_sided=two_sided)
    B.pt_sync(ctx)
    ref = glm.glm_naive(X, Z, n1, perms, two_sided=two_sided)
    want = oracle.fwer_pvalues(ref.maxnull, ref.t_obs, two_sided=two_sided)
    got = p.cpu().numpy().astype(np.float64)
    # both sides compare float32 values: a p differs only where an FP64 maximum or
    # statistic rounds to a different float32 on the two sides, or at a near-tie row
    diff = np.abs(got - np.asarray(want, dtype=np.float32).astype(np.float64))
    assert np.mean(diff > 0) <= 0.01, np.flatnonzero(diff > 0)[:10]
    assert np.all(diff <= 3.0 / (P + 1)), diff.max()
    ctx.close()
