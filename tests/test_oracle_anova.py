"""Pins for the one-way F oracle (oracle/anova.py).

* The identity labelling reproduces scipy.stats.f_oneway at every voxel.
* With two groups F = t^2 of the two-sample oracle (Eq. 5).
* Exact enumeration: over every distinct relabelling of a tiny design the
  counts give scipy.stats.permutation_test's exact p-values (f_oneway
  statistic, independent samples).
* Invariances: reordering subjects within groups, affine changes of a voxel;
  B = SS_between / SS_total maps to F and back.
"""
import itertools

import numpy as np
import scipy.stats as st

import oracle
from oracle import anova as A
from paper_1703_01506_gb300 import synth


def test_identity_matches_scipy_f_oneway():
    rng = np.random.default_rng(1)
    sizes = [4, 6, 5]
    X = rng.standard_normal((15, 40)) + np.repeat([0.0, 0.7, -0.3], sizes)[:, None]
    F = A.f_rows(X, sizes, np.arange(15)[None, :])[0]
    b = np.cumsum([0] + sizes)
    for j in range(40):
        want = st.f_oneway(*[X[b[h]:b[h + 1], j] for h in range(3)]).statistic
        assert abs(F[j] - want) <= 1e-12 * max(1.0, abs(want))


def test_two_groups_is_t_squared():
    X = synth.gaussian_mean_shift(14, 60, seed=3)
    perms = synth.perms_pcg32(14, 25, seed=4)
    F = A.f_rows(X, [6, 8], perms)
    t = oracle.t_rows(X, 6, perms)
    np.testing.assert_allclose(F, t * t, rtol=1e-11)


def test_exact_enumeration_pvalues():
    rng = np.random.default_rng(5)
    sizes = [2, 2, 3]
    n = 7
    X = rng.standard_normal((n, 6)) + np.repeat([0.0, 1.0, -0.5], sizes)[:, None]
    perms = np.array(list(itertools.permutations(range(n))), dtype=np.int32)
    res = A.anova(X, sizes, perms)
    b = np.cumsum([0] + sizes)
    for j in range(6):
        samples = [X[b[h]:b[h + 1], j] for h in range(3)]
        pt = st.permutation_test(samples, lambda *s: st.f_oneway(*s).statistic,
                                 permutation_type="independent", alternative="greater",
                                 n_resamples=np.inf)
        # every distinct partition appears prod(n_h!) times among the n! rows
        assert abs(res.counts[j] / perms.shape[0] - pt.pvalue) <= 1e-12


def test_invariances_and_map():
    rng = np.random.default_rng(6)
    sizes = [5, 4, 6]
    X = rng.standard_normal((15, 30))
    perms = synth.perms_pcg32(15, 20, seed=2)
    F = A.f_rows(X, sizes, perms)
    p2 = perms.copy()
    p2[:, :5] = np.sort(p2[:, :5], axis=1)[:, ::-1]     # reorder within group 1
    np.testing.assert_allclose(A.f_rows(X, sizes, p2), F, rtol=1e-12)
    np.testing.assert_allclose(A.f_rows(3.0 * X - 2.0, sizes, perms), F, rtol=1e-9)
    Bv = A.b_of_f(F, 15, 3)
    back = Bv * (15 - 3) / ((1.0 - Bv) * (3 - 1))
    np.testing.assert_allclose(back, F, rtol=1e-10)
    Xc = X - X.mean(axis=0)
    ssb = sum(len(ix) * (X[ix].mean(axis=0) - X.mean(axis=0)) ** 2
              for ix in A._groups(perms[0], sizes))
    np.testing.assert_allclose(Bv[0], ssb / (Xc * Xc).sum(axis=0), rtol=1e-10)
