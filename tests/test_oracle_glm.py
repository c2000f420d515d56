"""Pins of the covariate-adjusted two-group statistic of the oracle
(oracle/glm.py) against independent computations: the C oracle's pooled t
when there is no covariate, the Frisch-Waugh-Lovell residualised regression
computed by QR, and invariances of the least-squares fit."""
import numpy as np
import pytest
from scipy import stats

import oracle
from oracle import glm
from paper_1703_01506_gb300 import synth


def test_no_covariate_is_the_pooled_two_sample_t():
    n, n1, v, P = 23, 9, 300, 40
    X = synth.two_group_gaussian(n1, n - n1, v, frac=0.05, effect=1.0, seed=2)
    perms = synth.perms_pcg32(n, P, seed=2)
    T = glm.glm_t_rows(X, None, n1, perms)
    ref = oracle.t_rows(X, n1, perms)  # the C oracle, Eq. (5) directly
    np.testing.assert_allclose(T, ref, rtol=1e-10, atol=1e-12)
    t0 = glm.glm_t_obs(X, np.zeros((n, 0)), n1)
    want = stats.ttest_ind(X[:n1].astype(np.float64), X[n1:].astype(np.float64),
                           equal_var=True).statistic
    np.testing.assert_allclose(t0, want, rtol=1e-10)


def _fwl_t(X, Z, n1, row):
    """t of the group coefficient by residualising the group column and the
    data on [1, Z] (QR projection), then a one-regressor fit without intercept
    with n - q - 2 residual degrees of freedom."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    C = np.column_stack([np.ones(n), Z])
    Q, _ = np.linalg.qr(C)
    lab = np.zeros(n)
    lab[row[:n1]] = 1.0
    lr = lab - Q @ (Q.T @ lab)
    Xr = X - Q @ (Q.T @ X)
    b = (lr @ Xr) / (lr @ lr)
    e = Xr - np.outer(lr, b)
    df = n - C.shape[1] - 1
    return b / np.sqrt((e * e).sum(0) / df / (lr @ lr))


@pytest.mark.parametrize("q", [1, 2, 4])
def test_matches_residualised_regression(q):
    rng = np.random.default_rng(q)
    n, n1, v, P = 31, 14, 200, 25
    X = rng.standard_normal((n, v)) + rng.uniform(0, 1, v)
    Z = rng.standard_normal((n, q))
    X[:, :50] += Z @ rng.standard_normal((q, 50))  # voxels that depend on the covariates
    perms = synth.perms_pcg32(n, P, seed=q)
    T = glm.glm_t_rows(X, Z, n1, perms)
    for i in range(P):
        np.testing.assert_allclose(T[i], _fwl_t(X, Z, n1, perms[i]), rtol=1e-9, atol=1e-12)


def test_invariances():
    rng = np.random.default_rng(7)
    n, n1, v, P = 26, 13, 120, 20
    X = rng.standard_normal((n, v))
    Z = rng.standard_normal((n, 2))
    perms = synth.perms_pcg32(n, P, seed=7)
    T = glm.glm_t_rows(X, Z, n1, perms)
    # a reparametrised covariate space (invertible mix plus a shift) spans the same columns
    A = np.array([[2.0, 0.5], [-1.0, 3.0]])
    np.testing.assert_allclose(glm.glm_t_rows(X, Z @ A + 4.0, n1, perms), T, rtol=1e-9)
    # an affine change of the data leaves t unchanged; a sign flip negates it
    np.testing.assert_allclose(glm.glm_t_rows(3.0 * X + 7.0, Z, n1, perms), T, rtol=1e-9)
    np.testing.assert_allclose(glm.glm_t_rows(-X, Z, n1, perms), -T, rtol=1e-9)
    # reordering the subjects (data, covariates and relabellings together)
    pi = rng.permutation(n)
    inv = np.argsort(pi)
    perms2 = inv[perms]
    np.testing.assert_allclose(glm.glm_t_rows(X[pi], Z[pi], n1, perms2), T, rtol=1e-9)


def test_scale_and_monotone_map():
    """t = sqrt(df) w / sqrt(1 - w^2) with w = (l . r / ||r||) / sqrt(a), a = ||R l||^2:
    the map the library's epilogue relies on (t increasing in the contraction u = l . r/||r||
    for a fixed relabelling)."""
    rng = np.random.default_rng(11)
    n, n1, v, P = 30, 12, 80, 15
    X = rng.standard_normal((n, v))
    Z = rng.standard_normal((n, 3))
    perms = synth.perms_pcg32(n, P, seed=11)
    res = glm.glm_naive(X, Z, n1, perms)
    C = np.column_stack([np.ones(n), Z])
    Q, _ = np.linalg.qr(C)
    R = X - Q @ (Q.T @ X)
    Rn = R / np.linalg.norm(R, axis=0)
    for i in range(P):
        lab = np.zeros(n)
        lab[perms[i, :n1]] = 1.0
        u = lab @ Rn
        w = u / np.sqrt(res.a[i])
        t = np.sqrt(res.df) * w / np.sqrt(1.0 - w * w)
        np.testing.assert_allclose(t, res.T[i], rtol=1e-9)
        np.testing.assert_allclose(res.u_of(res.T[i], i), u, rtol=1e-9, atol=1e-12)


def test_naive_outputs_from_the_full_matrix():
    rng = np.random.default_rng(5)
    n, n1, v, P = 20, 10, 60, 30
    X = rng.standard_normal((n, v))
    X[:, 7] = 2.5  # constant voxel: no statistic
    Z = rng.standard_normal((n, 1))
    perms = synth.perms_pcg32(n, P, seed=5)
    perms[3] = np.arange(n)
    res = glm.glm_naive(X, Z, n1, perms)
    T = np.where(np.isnan(res.T), -np.inf, res.T)
    assert np.all(res.maxnull == T.max(axis=1))
    assert np.all(res.argmax == np.argmax(T, axis=1))
    assert res.counts[7] == 0 and np.isnan(res.t_obs[7])
    assert np.all(res.counts[np.arange(v) != 7] >= 1)  # the identity row counts itself
    two = glm.glm_naive(X, Z, n1, perms, two_sided=True)
    assert np.all(two.maxnull >= res.maxnull)
