"""Pins for the RapidPT oracle (Alg. 2, Sec. 4.1-4.2).

* Philox4x32-10 against its published known-answer vectors.
* Normal and index draws against N(0,1) / uniformity and the Box-Muller bound.
* The l1 weight solve (ADMM) against scipy's LP solution of the same
  least-absolute-deviations problem.
* QR with positive diagonal; the geodesic update keeps U orthonormal and, with
  every voxel sampled and step 1, puts the fitted column exactly in span(U)
  (GROUSE's greedy step).
* Exact low-rank special case: with the linear statistic mean1 - mean2, T has
  rank <= n-1; with r = n-1 the recovered max-null equals the exhaustive one.
Beyond these, RapidPT's t-statistic result is an approximation with no exact
value ("parity unpinned"); it is compared statistically with NaivePT.
"""
import math
import os

import numpy as np
import pytest
import scipy.optimize as so
import scipy.stats as st

import oracle
from oracle import rapid as R
from paper_1703_01506_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        f = [int(x, 16) for x in line.split()]
        out = R.philox4x32_10(*f[:6])
        assert [int(x) for x in out] == f[6:]


def test_normal_draws():
    d = R.draws(12345)
    j, c = np.meshgrid(np.arange(2000), np.arange(100), indexing="ij")
    z = d.normal(R.TAG_NOISE, j, c).ravel()
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    assert st.kstest(z, "norm").pvalue > 1e-3
    assert np.max(np.abs(z)) <= math.sqrt(-2.0 * math.log(2.0 ** -32))
    z2 = R.draws(12346).normal(R.TAG_NOISE, j, c).ravel()
    assert abs(np.corrcoef(z, z2)[0, 1]) < 0.01  # another key, another stream


def test_voxel_normal_draws():
    """Box-Muller pairs, four voxels per counter (words x0, x1 for voxels 4p,
    4p + 1; x2, x3 for 4p + 2, 4p + 3; cos for the even, sin for the odd voxel
    of a pair): each component N(0,1) with the |z| bound, neighbours
    uncorrelated, and z_even^2 + z_odd^2 = -2 ln u1 of the pair's first word
    exactly (so voxel 4p reproduces the single-normal draw of counter p)."""
    d = R.draws(12345)
    j, c = np.meshgrid(np.arange(4000), np.arange(50), indexing="ij")
    z = d.voxel_normal(R.TAG_NOISE, j, c)
    for k in range(4):
        part = z[k::4].ravel()
        assert abs(part.mean()) < 0.015 and abs(part.var() - 1.0) < 0.015
        assert st.kstest(part, "norm").pvalue > 1e-3
    assert np.max(np.abs(z)) <= math.sqrt(-2.0 * math.log(2.0 ** -32))
    for k in range(3):
        assert abs(np.corrcoef(z[k::4].ravel(), z[k + 1::4].ravel())[0, 1]) < 0.015
    p_ = np.arange(1000)
    np.testing.assert_allclose(z[0::4, 7], d.normal(R.TAG_NOISE, p_, 7), rtol=0, atol=0)
    x0, _, x2, _ = d.words(np.asarray(p_, dtype=np.uint64), 7, 0, R.TAG_NOISE)
    for first, w in ((0, x0), (2, x2)):
        rad2 = -2.0 * np.log((w.astype(np.float64) + 1.0) * 2.0 ** -32)
        np.testing.assert_allclose(z[first::4, 7] ** 2 + z[first + 1::4, 7] ** 2, rad2,
                                   rtol=1e-12)


def test_index_draws_uniform_in_range():
    d = R.draws(7)
    v = 37
    k = d.index(R.TAG_REC, np.arange(200000), 5, 0, v)
    assert k.min() >= 0 and k.max() < v
    assert st.chisquare(np.bincount(k, minlength=v)).pvalue > 1e-3
    big = d.index(R.TAG_TRAIN, np.arange(1000), 1, 2, 600000)
    assert big.max() < 600000 and big.min() >= 0


def test_admm_l1_matches_linear_program():
    rng = np.random.default_rng(3)
    m, r = 60, 5
    A = rng.standard_normal((m, r))
    b = A @ rng.standard_normal(r) + rng.laplace(size=m) * 0.3
    b[:4] += 8.0  # outliers
    w, s, y = R.admm_l1(A, b, rho=1.0, iters=4000)
    # LP: min sum(t) s.t. -t <= A w - b <= t
    c = np.concatenate([np.zeros(r), np.ones(m)])
    A_ub = np.block([[A, -np.eye(m)], [-A, -np.eye(m)]])
    b_ub = np.concatenate([b, -b])
    lp = so.linprog(c, A_ub=A_ub, b_ub=b_ub, bounds=[(None, None)] * r + [(0, None)] * m)
    obj = np.abs(A @ w - b).sum()
    assert abs(obj - lp.fun) <= 1e-6 * lp.fun
    assert np.max(np.abs(y)) <= 1.0 + 1e-6  # dual of an l1 fit lies in the unit box


def test_qr_posdiag():
    rng = np.random.default_rng(4)
    A = rng.standard_normal((300, 12))
    Q = R.qr_posdiag(A)
    np.testing.assert_allclose(Q.T @ Q, np.eye(12), atol=1e-12)
    Rm = Q.T @ A
    assert np.all(np.diag(Rm) > 0) and np.allclose(np.tril(Rm, -1), 0, atol=1e-12)


def test_geodesic_step_greedy_and_orthonormal():
    rng = np.random.default_rng(5)
    v, r = 200, 6
    U = R.qr_posdiag(rng.standard_normal((v, r)))
    b = rng.standard_normal(v)
    idx = np.arange(v)
    w = U.T @ b  # least-squares weights with every voxel sampled
    U1 = R.geodesic_step(U, idx, b, w, 1.0)
    np.testing.assert_allclose(U1.T @ U1, np.eye(r), atol=1e-12)
    resid = b - U1 @ (U1.T @ b)
    assert np.linalg.norm(resid) <= 1e-10 * np.linalg.norm(b)
    # half a step: still orthonormal, but b is not yet in the span
    U2 = R.geodesic_step(U, idx, b, w, 0.5)
    np.testing.assert_allclose(U2.T @ U2, np.eye(r), atol=1e-12)
    assert np.linalg.norm(b - U2 @ (U2.T @ b)) > 1e-3 * np.linalg.norm(b)
    # sampled step: orthonormal too (the direction is projected off span(U))
    idx_s = np.random.default_rng(6).integers(0, v, 40)
    ws, _, _ = R.admm_l1(U[idx_s], b[idx_s], 2.0, 30)
    U3 = R.geodesic_step(U, idx_s, b[idx_s], ws, 1.0)
    np.testing.assert_allclose(U3.T @ U3, np.eye(r), atol=1e-10)


def test_exact_low_rank_recovery():
    n, n1, v, P = 8, 4, 300, 120
    X = synth.gaussian_mean_shift(n, v, seed=4)
    perms = synth.perms_pcg32(n, P, seed=2)
    o = R.RapidOpts(train_passes=60, stat="meandiff", admm_iters=300, qr_every=50)
    res = R.rapid(X, n1, perms, n - 1, 0.3, 40, o)
    Lm = np.full(perms.shape, -1.0 / (n - n1))
    Lm[:, :n1] = 1.0 / n1
    Lw = np.zeros((P, n))
    np.put_along_axis(Lw, perms, Lm, axis=1)
    exact = (Lw @ X.astype(np.float64)).max(axis=1)
    assert res.sigma < 1e-9 and abs(res.mu) < 1e-9
    np.testing.assert_allclose(res.maxnull, exact, atol=1e-9)


def test_training_rows_exact_and_counts():
    n, n1, P = 24, 12, 300
    X, mask = synth.brain_field(n, n1, grid=(16, 18, 16), center=(8, 9, 8), semi_axes=(6, 7, 6),
                                fwhm=4.0, seed=2)
    X = X.numpy()[:, mask.numpy().astype(bool)]
    perms = synth.perms_pcg32(n, P, seed=3)
    res = R.rapid(X, n1, perms, 6, 0.05, 40, R.RapidOpts(train_passes=2))
    ref = oracle.naive(X, n1, perms[:40])
    np.testing.assert_allclose(res.maxnull[:40], ref.maxnull, rtol=1e-12)
    np.testing.assert_array_equal(res.counts, ref.counts)


def test_rapid_tracks_naive_max_null_on_smooth_field():
    """Statistical check on a smoothed field (no exact value exists): the
    recovered max-null is close to the exhaustive one in KL and thresholds."""
    n, n1, P = 40, 20, 1500
    X, mask = synth.brain_field(n, n1, grid=(30, 36, 30), center=(15, 18, 15),
                                semi_axes=(12, 15, 12), fwhm=6.0, seed=3)
    X = X.numpy()[:, mask.numpy().astype(bool)]
    perms = synth.perms_pcg32(n, P, seed=1)
    ref = oracle.naive(X, n1, perms)
    res = R.rapid(X, n1, perms, 20, 0.02, 80, R.RapidOpts(train_passes=20))
    kl = R.kl_divergence(ref.maxnull, res.maxnull)
    assert kl < 0.6, kl
    for a in (0.05, 0.01):
        t_ref, t_rap = R.fwer_threshold(ref.maxnull, a), R.fwer_threshold(res.maxnull, a)
        assert abs(t_rap - t_ref) / t_ref < 0.15, (a, t_ref, t_rap)


def _planted(ell=12, V=400, r=5, m=30, c=0.3, with_region=True, zero_model=False, seed=8):
    """Training columns T_ex = U* W* + R with everything known in closed form.
    U* = the unit vectors of voxels 0..r-1 (orthonormal); R is zero on those
    voxels, so U*^T R = 0 and the least-squares weights are W* exactly. R holds
    the constant c on voxels 100..199 (optional) and one spike h_i per column
    at a voxel of 300..399 that the column's sampled set Omega_i never draws.
    Omega_i (repeats allowed) draws two thirds of its entries from 100..199, so
    the sampled share of the c-region differs from its share of all voxels."""
    rng = np.random.default_rng(seed)
    U = np.zeros((V, r))
    U[np.arange(r), np.arange(r)] = 1.0
    W = np.zeros((r, ell)) if zero_model else rng.uniform(-1.0, 1.0, (r, ell))
    if not zero_model:
        W[:, 3] = -np.abs(W[:, 3]) - 0.1    # a column whose model maximum is a zero voxel
    Rm = np.zeros((ell, V))
    if with_region:
        Rm[:, 100:200] = c
    last_idx, spikes, h = [], [], 5.0 + 0.25 * np.arange(ell)
    for i in range(ell):
        k = 2 * m // 3
        idx = np.concatenate([rng.integers(100, 200, k), rng.integers(0, 100, m - k)])
        idx[1] = idx[0]                     # a repeated draw counts twice
        spike = 300 + int(rng.integers(0, 100))
        Rm[i, spike] = h[i]
        last_idx.append(idx)
        spikes.append(spike)
    T_ex = (U @ W).T + Rm
    return T_ex, U, W, Rm, last_idx, h


def test_training_summary_planted_residual_mode0():
    """W_ex = W*, sigma = the population std of R over the last pass's sampled
    entries (a two-valued sample: c * sqrt(p (1 - p)), p = share of sampled
    entries in the c-region, repeats counted), mu = the largest residual over
    all training entries (the spikes, never sampled)."""
    T_ex, U, W, Rres, last_idx, h = _planted()
    W_ex, sigma, mu = R_training_summary(T_ex, U, last_idx, 0)
    np.testing.assert_allclose(W_ex, W, rtol=0, atol=1e-15)
    hits = sum(int(np.sum((ix >= 100) & (ix < 200))) for ix in last_idx)
    N = sum(ix.size for ix in last_idx)
    p = hits / N
    assert abs(p - 0.25) > 0.2                      # sampled share != share of all voxels
    assert sigma == pytest.approx(0.3 * math.sqrt(p * (1.0 - p)), rel=1e-12)
    assert mu == pytest.approx(float(h.max()), rel=1e-15)


def test_training_summary_planted_residual_mode1_no_noise():
    """With R zero on every sampled entry, sigma = 0 and the shift is the mean
    over training columns of (column maximum of T_ex) - (column maximum of the
    model U W_ex): h_i - max(max_k W*[k, i], 0), the model being zero off
    voxels 0..r-1."""
    T_ex, U, W, Rres, last_idx, h = _planted(with_region=False)
    W_ex, sigma, mu = R_training_summary(T_ex, U, last_idx, 1)
    assert sigma == 0.0
    expect = np.mean(h - np.maximum(W.max(axis=0), 0.0))
    assert mu == pytest.approx(float(expect), rel=1e-14)
    assert W[:, 3].max() < 0.0                      # that column's model maximum is 0


def test_training_summary_planted_residual_mode1_zero_model():
    """With W* = 0 the model vanishes, so the shift is the mean over columns of
    h_i - sigma * max_j z_ij, z_ij the shift-estimate normals of column i."""
    T_ex, U, W, Rres, last_idx, h = _planted(zero_model=True)
    W_ex, sigma, mu = R_training_summary(T_ex, U, last_idx, 1)
    np.testing.assert_allclose(W_ex, 0.0, atol=0)
    hits = sum(int(np.sum((ix >= 100) & (ix < 200))) for ix in last_idx)
    p = hits / sum(ix.size for ix in last_idx)
    s = 0.3 * math.sqrt(p * (1.0 - p))
    assert sigma == pytest.approx(s, rel=1e-12)
    d = R.draws(1)
    zmax = np.array([d.voxel_normal(R.TAG_SHIFT, np.arange(T_ex.shape[1]), i).max()
                     for i in range(T_ex.shape[0])])
    assert mu == pytest.approx(float(np.mean(h - s * zmax)), rel=1e-12)


def test_training_weights_are_least_squares():
    """W_ex is the least-squares fit of every training column on U (Sec. 4.1):
    equal to LAPACK's lstsq for an orthonormal U and arbitrary columns."""
    rng = np.random.default_rng(9)
    U = R.qr_posdiag(rng.standard_normal((300, 7)))
    T_ex = rng.standard_normal((10, 300))
    W_ex, _, _ = R_training_summary(T_ex, U, [np.arange(5)] * 10, 0)
    ls = np.linalg.lstsq(U, T_ex.T, rcond=None)[0]
    np.testing.assert_allclose(W_ex, ls, atol=1e-12)


def R_training_summary(T_ex, U, last_idx, shift_mode):
    return R.training_summary(T_ex, U, last_idx, shift_mode, R.draws(1))


def test_u_statistic_exact_recovery_at_full_rank():
    """Modelling u (the group-1 share of the unit-norm centred voxel, linear in
    the relabelling, so its matrix has rank <= n - 1) instead of t: with
    r = n - 1 and a converged basis the residual vanishes (sigma, mu -> 0) and
    the recovered t maxima, t(max u), equal the exhaustive ones, because t(u)
    is strictly increasing and the same at every voxel."""
    n, n1, v, P = 10, 5, 400, 150
    X = synth.gaussian_mean_shift(n, v, seed=4)
    perms = synth.perms_pcg32(n, P, seed=2)
    ref = oracle.naive(X, n1, perms)
    o = R.RapidOpts(train_passes=60, stat="u", admm_iters=300, qr_every=50)
    res = R.rapid(X, n1, perms, n - 1, 0.3, 40, o)
    assert res.sigma < 1e-8 and abs(res.mu) < 1e-8
    np.testing.assert_allclose(res.maxnull, ref.maxnull, rtol=1e-7)
    np.testing.assert_array_equal(res.counts, oracle.naive(X, n1, perms[:40]).counts)


def _small_trained(stat="t", n=12, v=500, P=160, ell=40, r=6, eta=0.2, passes=4):
    X = synth.gaussian_mean_shift(n, v, seed=12)
    perms = synth.perms_pcg32(n, P, seed=13)
    o = R.RapidOpts(train_passes=passes, stat=stat)
    tr = R.rapid_train(X, n // 2, perms, r, eta, ell, o)
    return X, perms, tr, o


def test_recovery_updates_reconstruct_before_updating():
    """With U updates in recovery (rec_step > 0) each relabelling is recovered
    with the U it was fitted to, and U changes only afterwards: the first
    recovered row equals the frozen recovery's, later rows differ, and a
    vanishing step size tends to the frozen result."""
    X, perms, tr, o = _small_trained()
    rows = np.arange(40, 160)
    frozen = R.rapid_recover(X, 6, perms, rows, tr.U, tr.sigma, tr.mu, tr.m, o)
    upd = R.rapid_recover(X, 6, perms, rows, tr.U, tr.sigma, tr.mu, tr.m,
                          R.RapidOpts(train_passes=4, rec_step=1.0))
    assert upd[0] == frozen[0]
    assert np.max(np.abs(upd[1:] - frozen[1:])) > 1e-6
    tiny = R.rapid_recover(X, 6, perms, rows, tr.U, tr.sigma, tr.mu, tr.m,
                           R.RapidOpts(train_passes=4, rec_step=1e-9))
    np.testing.assert_allclose(tiny, frozen, rtol=0, atol=1e-6)


def test_recovery_updates_keep_exact_low_rank():
    """Linear statistic, r = n - 1, converged basis: every recovery fit is exact,
    so the geodesic steps change nothing and the recovered max-null still equals
    the exhaustive one."""
    n, n1, v, P = 8, 4, 300, 120
    X = synth.gaussian_mean_shift(n, v, seed=4)
    perms = synth.perms_pcg32(n, P, seed=2)
    o = R.RapidOpts(train_passes=60, stat="meandiff", admm_iters=300, qr_every=50, rec_step=1.0)
    res = R.rapid(X, n1, perms, n - 1, 0.3, 40, o)
    Lm = np.full(perms.shape, -1.0 / (n - n1))
    Lm[:, :n1] = 1.0 / n1
    Lw = np.zeros((P, n))
    np.put_along_axis(Lw, perms, Lm, axis=1)
    exact = (Lw @ X.astype(np.float64)).max(axis=1)
    np.testing.assert_allclose(res.maxnull, exact, atol=1e-9)
