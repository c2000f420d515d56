"""GPU NaivePT (through the C ABI) against the FP64 oracle, element by element.

Tolerances (t-class paths, FP32 accumulation): max-null within 1e-5 relative
(absolute floor 1e-5), argmax equal except at recorded near-ties, per-voxel
counts equal except for entries the oracle records as near-ties with the
observed statistic.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu

PRECS = [0, 1, 2, 3]  # PT_PREC_FP32, PT_PREC_BF16X2, PT_PREC_BF16X3, PT_PREC_FP16X2


def tie_rel(precision, n):
    """Bound on |error of u - u_obs| per unit l1 norm of the unit-norm voxel:
    FP32 data and accumulation (FP32, BF16x3), 16-bit data pieces (BF16x2) or
    22-bit FP16 pieces (FP16x2: |2^15 y - hi - lo| <= 2^-22 |2^15 y|), for both
    the relabelled and the observed group sum."""
    eps24 = 2.0 ** -24
    if precision == 1:
        return 2.0 * (2.0 ** -17 + (n + 4) * eps24)
    if precision == 3:
        return 2.0 * (2.0 ** -22 + (n + 4) * eps24)
    return 2.0 * (n + 4) * eps24


def run_gpu(B, X, n1, perms, precision, two_sided=False, mask=None):
    dev = torch.device("cuda:0")
    Xd = torch.as_tensor(X).to(dev).contiguous()
    md = None if mask is None else torch.as_tensor(mask.astype(np.uint8)).to(dev)
    ctx = B.pt_prepare(Xd, n1, md)
    pd = torch.as_tensor(perms).to(dev).contiguous()
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=precision, two_sided=two_sided)
    out = (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
           ct.cpu().numpy().astype(np.int64))
    ctx.close()
    return out


def check(ref, got, precision, name=""):
    """maxnull within 1e-5 relative (and within FP32 output rounding when the
    argmax agrees: the winner's t is recomputed in FP64); argmax equal unless the
    oracle's best and runner-up are within the u-band; counts equal up to the
    oracle's near-tie entries."""
    mx, am, ct = got
    same = am == ref.argmax
    err = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7), (name, float(err[same].max()))
    band = 2.0 * float(np.max(ref.tau)) if ref.tau.size else 0.0
    gap_u = ref.u_of(ref.maxnull) - ref.u_of(ref.second)
    near_tie = gap_u <= band
    bad = ~same & ~near_tie
    assert not bad.any(), (name, np.flatnonzero(bad)[:10], am[bad][:5], ref.argmax[bad][:5])
    du = np.abs(ref.u_of(mx) - ref.u_of(ref.maxnull))
    assert np.all(du[~same] <= band), (name, du[~same])
    if ct.size:
        dc = np.abs(ct - ref.counts.astype(np.int64))
        badc = dc > ref.near.astype(np.int64)
        assert not badc.any(), (name, np.flatnonzero(badc)[:10], dc[badc][:10])


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("two_sided", [False, True])
def test_parity_gauss_n20_v2000(cuda_lib, precision, two_sided):
    n, n1, v, P = 20, 10, 2000, 1000
    X = synth.gaussian_mean_shift(n, v, seed=1)
    perms = synth.perms_pcg32(n, P, seed=1)
    ref = oracle.naive(X, n1, perms, two_sided=two_sided, tie_rel=tie_rel(precision, n))
    got = run_gpu(cuda_lib, X, n1, perms, precision, two_sided)
    check(ref, got, precision, "cfg0")


@pytest.mark.parametrize("precision", PRECS)
@pytest.mark.parametrize("n,n1,v,P", [(37, 15, 1007, 300), (100, 50, 3000, 1000),
                                      (3, 1, 129, 5), (64, 63, 513, 129), (200, 100, 700, 260),
                                      (360, 180, 700, 130)])
def test_parity_ragged_shapes(cuda_lib, precision, n, n1, v, P):
    X = synth.two_group_gaussian(n1, n - n1, v, frac=0.02, effect=1.0, seed=n + v)
    perms = synth.perms_pcg32(n, P, seed=7)
    ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(precision, n))
    got = run_gpu(cuda_lib, X, n1, perms, precision)
    check(ref, got, precision, (n, n1, v, P))


@pytest.mark.parametrize("precision", PRECS)
def test_parity_large_n(cuda_lib, precision):
    n, n1, v, P = 400, 200, 600, 200
    X = synth.gaussian_mean_shift(n, v, seed=4)
    perms = synth.perms_pcg32(n, P, seed=3)
    ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(precision, n))
    got = run_gpu(cuda_lib, X, n1, perms, precision)
    check(ref, got, precision, "n400")


@pytest.mark.parametrize("precision", PRECS)
def test_masked_brain_with_degenerate_voxels(cuda_lib, precision):
    n, n1, P = 24, 12, 400
    X, mask = synth.brain_field(n, n1, grid=(20, 24, 20), center=(10, 12, 10),
                                semi_axes=(8, 10, 8), fwhm=4.0, effect=0.5, effect_radius=3.0,
                                seed=2, device="cpu")
    X = X.numpy().copy()
    mask = mask.numpy().astype(bool)
    idx = np.flatnonzero(mask)
    X[:, idx[5]] = 0.5   # constant inside the mask -> excluded
    X[:, idx[77]] = 0.0
    perms = synth.perms_pcg32(n, P, seed=5)
    ref = oracle.naive(X[:, mask], n1, perms, tie_rel=tie_rel(precision, n))
    mx, am, ct = run_gpu(cuda_lib, X, n1, perms, precision, mask=mask)
    check(ref, (mx, am, ct), precision, "brain")
    assert ct[5] == 0 and ct[77] == 0


def test_identity_relabelling_counts_itself(cuda_lib):
    """An exact tie with the observed statistic (same group-1 set, any order) counts."""
    n, n1, v = 30, 15, 500
    X = synth.gaussian_mean_shift(n, v, seed=8)
    base = np.arange(n, dtype=np.int32)
    rows = np.stack([base, np.concatenate([base[:n1][::-1], base[n1:][::-1]])]).astype(np.int32)
    for prec in PRECS:
        _, _, ct = run_gpu(cuda_lib, X, n1, rows, prec)
        assert np.all(ct == 2), prec


def test_t_obs_matches_oracle(cuda_lib):
    B = cuda_lib
    n, n1, v = 33, 11, 777
    X = synth.gaussian_mean_shift(n, v, seed=9)
    ref = oracle.naive(X, n1, synth.identity_perm(n))
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    t = torch.empty(v, dtype=torch.float32, device="cuda")
    B.pt_t_obs(ctx, t)
    B.pt_sync(ctx)
    np.testing.assert_allclose(t.cpu().numpy(), ref.t_obs, rtol=2e-7, atol=1e-7)
    assert B.pt_num_voxels(ctx) == v and B.pt_num_valid_voxels(ctx) == v
    ctx.close()


@pytest.mark.parametrize("offset,unit", [(1.0e4, 1.0e-2), (-3.0e5, 1.0), (0.0, 1.0e-30),
                                         (0.0, 1.0e30), (2.0e37, 1.0e36)])
def test_moments_offsets_and_extreme_scales(cuda_lib, offset, unit):
    """Data far from unit scale: a mean 10^6 standard deviations from zero (the
    centring must not lose the spread; the FP32 values are quantised, so many
    relabellings tie), values whose squares underflow or overflow FP32, and
    values whose FP32 sum overflows (2e37 x 40 subjects). t_obs to FP32 output
    rounding, and the max-null and counts of the FP32 and FP16x2 paths, against
    the FP64 oracle on the same FP32 inputs."""
    B = cuda_lib
    n, n1, v, P = 40, 17, 3001, 300
    X = (synth.gaussian_mean_shift(n, v, seed=31).astype(np.float64) * unit
         + offset).astype(np.float32)
    assert np.all(np.isfinite(X))
    perms = synth.perms_pcg32(n, P, seed=32)
    t_ref = oracle.naive(X, n1, synth.identity_perm(n)).t_obs
    ok = ~np.isnan(t_ref)
    assert ok.mean() > 0.99
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    t = torch.empty(v, dtype=torch.float32, device="cuda")
    B.pt_t_obs(ctx, t)
    B.pt_sync(ctx)
    t = t.cpu().numpy().astype(np.float64)
    assert np.array_equal(np.isnan(t), ~ok)
    np.testing.assert_allclose(t[ok], t_ref[ok], rtol=2e-7, atol=1e-7)
    ctx.close()
    for precision in (0, 3):
        ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(precision, n))
        check(ref, run_gpu(B, X, n1, perms, precision), precision, (offset, unit, precision))


def test_invalid_relabelling_reported_and_context_survives(cuda_lib):
    B = cuda_lib
    n, n1, v, P = 16, 8, 300, 50
    X = synth.gaussian_mean_shift(n, v, seed=10)
    perms = synth.perms_pcg32(n, P, seed=1)
    bad = perms.copy()
    bad[17, 3] = bad[17, 4]
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    for prec in PRECS:
        with pytest.raises(B.PtError) as e:
            B.maxnull_naive(ctx, torch.as_tensor(bad).cuda(), precision=prec)
        assert e.value.status == B.PT_ERR_INVALID
        mx, _, _ = B.maxnull_naive(ctx, torch.as_tensor(perms).cuda(), precision=prec)
        ref = oracle.naive(X, n1, perms)
        assert np.allclose(mx.cpu().numpy(), ref.maxnull, rtol=1e-5)
    ctx.close()


def test_nan_input_rejected(cuda_lib):
    B = cuda_lib
    X = synth.gaussian_mean_shift(10, 50, seed=1)
    X[3, 7] = np.nan
    with pytest.raises(B.PtError) as e:
        B.pt_prepare(torch.as_tensor(X).cuda(), 5)
    assert e.value.status == B.PT_ERR_INVALID


def test_deterministic_repeat(cuda_lib):
    n, n1, v, P = 50, 25, 5000, 700
    X = synth.gaussian_mean_shift(n, v, seed=12)
    perms = synth.perms_pcg32(n, P, seed=12)
    for prec in PRECS:
        a = run_gpu(cuda_lib, X, n1, perms, prec)
        b = run_gpu(cuda_lib, X, n1, perms, prec)
        for x, y in zip(a, b):
            np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("precision", [2, 3])
@pytest.mark.parametrize("name", ["brain_n100_v232k", "brain_n200_v500k", "brain_n400_v600k"])
def test_full_size_sampled(cuda_lib, name, precision):
    """The full-size workloads (n=100 / 232k voxels / 10k relabellings, n=200 /
    500k / 100k, n=400 / 600k / 100k; split BF16x3 and FP16x2) in the launch configuration
    bench.py times (autotuned): sampled rows against the oracle's full-row
    maxima, sampled voxels against the oracle's counts over all rows."""
    B = cuda_lib
    w = synth.workload(name, device="cuda")
    X, mask, n1, perms = w["X"], w["mask"], w["n1"], w["perms"]
    ctx = B.pt_prepare(X, n1, mask)
    v = B.pt_num_voxels(ctx)
    pd = torch.as_tensor(perms).cuda()
    B.pt_tune_clear()
    B.pt_autotune_naive(ctx, pd, B.naive_opts(precision))
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=precision)
    B.pt_tune_clear()
    mx = mx.cpu().numpy().astype(np.float64)
    am = am.cpu().numpy()
    ct = ct.cpu().numpy().astype(np.int64)
    Xm = X[:, mask.bool()].cpu().numpy()
    del X
    assert Xm.shape[1] == v
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(perms.shape[0], 8, replace=False))
    n = Xm.shape[0]
    ref = oracle.naive(Xm, n1, perms[rows], tie_rel=tie_rel(precision, n))
    check(ref, (mx[rows], am[rows], np.zeros(0, np.int64)), precision, name + " rows")
    vox = np.sort(rng.choice(v, 32, replace=False))
    refc = oracle.naive(Xm[:, vox], n1, perms, tie_rel=tie_rel(precision, n))
    dc = np.abs(ct[vox] - refc.counts.astype(np.int64))
    assert np.all(dc <= refc.near.astype(np.int64)), dc
    ctx.close()


@pytest.mark.parametrize("masked", [True, False])
def test_prepare_from_pinned_host_memory(cuda_lib, masked):
    """X and mask in page-locked host memory (the mask voxels' values gathered
    over the host link, or all of X copied without a mask) give results
    identical to device copies, and t_obs too."""
    B = cuda_lib
    n, n1, P = 24, 12, 300
    X, mask = synth.brain_field(n, n1, grid=(20, 24, 20), center=(10, 12, 10),
                                semi_axes=(8, 10, 8), fwhm=4.0, effect=0.5, effect_radius=3.0,
                                seed=6, device="cpu")
    perms = torch.as_tensor(synth.perms_pcg32(n, P, seed=9)).cuda()
    outs = []
    for host in (False, True):
        Xa = X.contiguous().pin_memory() if host else X.cuda()
        ma = None
        if masked:
            ma = mask.to(torch.uint8).contiguous()
            ma = ma.pin_memory() if host else ma.cuda()
        ctx = B.pt_prepare(Xa, n1, ma)
        t = torch.empty(B.pt_num_voxels(ctx), dtype=torch.float32, device="cuda")
        B.pt_t_obs(ctx, t)
        outs.append([x.cpu() for x in B.maxnull_naive(ctx, perms, precision=2)] + [t.cpu()])
        ctx.close()
    for a, b in zip(*outs):
        assert torch.equal(a, b)


@pytest.mark.parametrize("two_sided", [False, True])
def test_fwer_pvalues_match_oracle(cuda_lib, two_sided):
    """Corrected p-values (Sec. 2) from the GPU max-null and observed statistics
    against the oracle's definition applied to the oracle's own max-null and
    observed statistics. Both sides compare float32 values; a voxel's p can
    differ only where an FP64 maximum or statistic rounds to a different float32
    on the two sides, or at a near-tie row whose winner differs."""
    B = cuda_lib
    n, n1, v, P = 30, 15, 3000, 5000
    X = synth.two_group_gaussian(n1, n - n1, v, frac=0.02, effect=1.5, seed=4)
    perms = synth.perms_pcg32(n, P, seed=2)
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    pd = torch.as_tensor(perms).cuda()
    mx, _, _ = B.maxnull_naive(ctx, pd, precision=2, two_sided=two_sided)
    p = torch.empty(v, dtype=torch.float32, device="cuda")
    B.pt_fwer_pvalues(ctx, mx, p, two_sided)
    B.pt_sync(ctx)
    ref = oracle.naive(X, n1, perms, two_sided=two_sided, tie_rel=tie_rel(2, n))
    want = oracle.fwer_pvalues(ref.maxnull, ref.t_obs, two_sided).astype(np.float32)
    got = p.cpu().numpy()
    diff = np.abs(got.astype(np.float64) - want.astype(np.float64))
    assert np.mean(diff > 0) <= 0.005, np.flatnonzero(diff > 0)[:10]
    assert np.all(diff <= 3.0 / (P + 1)), diff.max()
    assert np.nanmin(got) >= 1.0 / (P + 1) - 1e-9
    ctx.close()


@pytest.mark.parametrize("precision", PRECS)
def test_largest_tensor_core_n(cuda_lib, precision):
    """n = 544: the largest subject count whose BF16x3 data tile (64 voxels)
    still fits in shared memory, on every path."""
    n, n1, v, P = 544, 272, 300, 140
    X = synth.gaussian_mean_shift(n, v, seed=9)
    perms = synth.perms_pcg32(n, P, seed=8)
    ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(precision, n))
    got = run_gpu(cuda_lib, X, n1, perms, precision)
    check(ref, got, precision, "n544")


def test_maximum_n_fp32_and_tensor_core_limit(cuda_lib):
    """n = 1024 (the API maximum): the FP32 path matches the oracle; the BF16x3
    path reports PT_ERR_UNSUPPORTED (its resident data tile cannot fit) and
    leaves the context usable."""
    B = cuda_lib
    n, n1, v, P = 1024, 512, 257, 40
    X = synth.gaussian_mean_shift(n, v, seed=10)
    perms = synth.perms_pcg32(n, P, seed=11)
    ref = oracle.naive(X, n1, perms, tie_rel=tie_rel(0, n))
    ctx = B.pt_prepare(torch.as_tensor(X).cuda(), n1)
    pd = torch.as_tensor(perms).cuda()
    with pytest.raises(B.PtError) as e:
        B.maxnull_naive(ctx, pd, precision=2)
    assert e.value.status == B.PT_ERR_UNSUPPORTED
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=0)
    check(ref, (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
                ct.cpu().numpy().astype(np.int64)), 0, "n1024")
    ctx.close()
