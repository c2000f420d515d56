"""Pins for the one-way ANCOVA oracle (oracle/ancova.py): the F of a g-group
factor with nuisance covariates under relabellings.

* Without covariates it is scipy.stats.f_oneway at every voxel (identity
  labelling) and the one-way oracle under relabellings.
* With two groups it is the square of the covariate-adjusted t (oracle/glm.py).
* With one covariate it equals the textbook adjusted-sums-of-squares formula
  (total and within-group sums of squares and cross-products of y and z),
  written here without any least-squares solve.
* Invariances: adding a combination of the nuisance columns to a voxel or
  scaling it; reordering subjects within a group. Degenerate cases: a voxel in
  the span of [1, Z] has no statistic, a group column in that span is an
  error. B maps to F and back.
"""
import numpy as np
import pytest
import scipy.stats as st

from oracle import anova as A
from oracle import ancova as AC
from oracle import glm as G
from paper_1703_01506_gb300 import synth


def test_no_covariates_is_one_way_f():
    rng = np.random.default_rng(11)
    sizes = [5, 4, 6]
    n = 15
    X = rng.standard_normal((n, 30)) + np.repeat([0.0, 0.6, -0.4], sizes)[:, None]
    F = AC.f_rows(X, sizes, None, np.arange(n)[None, :])[0]
    b = np.cumsum([0] + sizes)
    for j in range(30):
        want = st.f_oneway(*[X[b[h]:b[h + 1], j] for h in range(3)]).statistic
        assert abs(F[j] - want) <= 1e-10 * max(1.0, abs(want))
    perms = synth.perms_pcg32(n, 12, seed=3)
    np.testing.assert_allclose(AC.f_rows(X, sizes, None, perms), A.f_rows(X, sizes, perms),
                               rtol=1e-10)


def test_two_groups_is_adjusted_t_squared():
    rng = np.random.default_rng(12)
    n, n1 = 16, 7
    X = rng.standard_normal((n, 25))
    Z = rng.standard_normal((n, 2))
    perms = synth.perms_pcg32(n, 10, seed=5)
    F = AC.f_rows(X, [n1, n - n1], Z, perms)
    T = G.glm_t_rows(X, Z, n1, perms)
    np.testing.assert_allclose(F, T * T, rtol=1e-9)


def _textbook_one_covariate(y, z, groups):
    """Classic one-way ANCOVA F with one covariate from total (T) and within-
    group (W) sums of squares and cross-products."""
    yc, zc = y - y.mean(), z - z.mean()
    Tyy, Tzz, Tzy = yc @ yc, zc @ zc, zc @ yc
    Wyy = Wzz = Wzy = 0.0
    for ix in groups:
        yw, zw = y[ix] - y[ix].mean(), z[ix] - z[ix].mean()
        Wyy += yw @ yw
        Wzz += zw @ zw
        Wzy += zw @ yw
    sse_full = Wyy - Wzy * Wzy / Wzz
    sse_red = Tyy - Tzy * Tzy / Tzz
    g, n = len(groups), y.size
    return ((sse_red - sse_full) / (g - 1)) / (sse_full / (n - g - 1))


def test_one_covariate_matches_textbook_formula():
    rng = np.random.default_rng(13)
    sizes = [4, 5, 3, 6]
    n = sum(sizes)
    z = rng.standard_normal(n)
    X = rng.standard_normal((n, 12)) + 0.8 * z[:, None]
    X += np.repeat([0.0, 0.5, -0.7, 0.2], sizes)[:, None]
    perms = np.vstack([np.arange(n), synth.perms_pcg32(n, 6, seed=7)]).astype(np.int32)
    F = AC.f_rows(X, sizes, z[:, None], perms)
    b = np.cumsum([0] + sizes)
    for i, row in enumerate(perms):
        groups = [row[b[h]:b[h + 1]] for h in range(len(sizes))]
        for j in range(X.shape[1]):
            want = _textbook_one_covariate(X[:, j], z, groups)
            assert abs(F[i, j] - want) <= 1e-9 * max(1.0, abs(want)), (i, j)


def test_invariances_degenerate_cases_and_map():
    rng = np.random.default_rng(14)
    sizes = [5, 6, 4]
    n = 15
    Z = rng.standard_normal((n, 2))
    X = rng.standard_normal((n, 20))
    perms = synth.perms_pcg32(n, 8, seed=9)
    F = AC.f_rows(X, sizes, Z, perms)
    shift = 3.0 + Z @ np.array([1.5, -2.0])
    np.testing.assert_allclose(AC.f_rows(2.5 * X + shift[:, None], sizes, Z, perms), F,
                               rtol=1e-8)
    p2 = perms.copy()
    p2[:, 5:11] = p2[:, 5:11][:, ::-1]  # reorder within group 2
    np.testing.assert_allclose(AC.f_rows(X, sizes, Z, p2), F, rtol=1e-10)
    Xd = X.copy()
    Xd[:, 3] = 1.0 + Z[:, 0] - 0.5 * Z[:, 1]  # in the span of [1, Z]
    assert np.all(np.isnan(AC.f_rows(Xd, sizes, Z, perms)[:, 3]))
    Zs = np.column_stack([Z, np.r_[np.ones(5), np.zeros(10)]])  # group 1 of the identity
    with pytest.raises(ValueError):
        AC.f_rows(X, sizes, Zs, np.arange(n)[None, :])
    Bv = AC.b_of_f(F, n, sizes, Z)
    back = Bv * AC.df_of(n, sizes, Z) / ((1.0 - Bv) * (len(sizes) - 1))
    np.testing.assert_allclose(back, F, rtol=1e-10)


def test_ancova_summary():
    rng = np.random.default_rng(15)
    sizes = [6, 6, 6]
    n = 18
    Z = rng.standard_normal((n, 1))
    X = rng.standard_normal((n, 40))
    X[:, 7] = 2.0  # no statistic
    perms = synth.perms_pcg32(n, 50, seed=10)
    perms[4] = np.arange(n)
    r = AC.ancova(X, sizes, Z, perms)
    F = AC.f_rows(X, sizes, Z, perms)
    Fm = np.where(np.isnan(F), -np.inf, F)
    np.testing.assert_array_equal(r.argmax, np.argmax(Fm, axis=1))
    np.testing.assert_allclose(r.maxnull, Fm.max(axis=1))
    assert r.counts[7] == 0 and np.isnan(r.F_obs[7])
    ok = ~np.isnan(r.F_obs)
    assert np.all(r.counts[ok] >= 1)  # the identity row counts itself
    np.testing.assert_array_equal(r.counts, (F >= r.F_obs[None, :]).sum(axis=0))
