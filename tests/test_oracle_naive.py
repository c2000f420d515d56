"""Pins for the NaivePT oracle (Alg. 1, Eq. (5)) against things other than itself.

Each test fixes a fact the paper or the mathematics determines: a textbook
closed form, scipy's independent t-test and exact permutation test, exact
enumeration, symmetry under label swap, and uniformity of uncorrected
p-values under a null with no signal.
"""
import itertools
import os

import numpy as np
import pytest
import scipy.stats as st

import oracle
from paper_1703_01506_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _combo_perms(n, n1):
    """Every group-1 set of size n1 once, as relabelling rows."""
    rows = []
    for c in itertools.combinations(range(n), n1):
        rest = [s for s in range(n) if s not in c]
        rows.append(list(c) + rest)
    return np.array(rows, dtype=np.int32)


def test_closed_form_golden():
    path = os.path.join(GOLDEN, "two_sample_t_closed_form.txt")
    for line in open(path):
        if line.startswith("#") or not line.strip():
            continue
        f = line.split()
        n1, n2 = int(f[0]), int(f[1])
        vals = np.array([float(x) for x in f[2:2 + n1 + n2]])
        want = float(f[-1])
        X = vals[:, None]  # one voxel
        ident = synth.identity_perm(n1 + n2)
        r = oracle.naive(X, n1, ident)
        assert abs(r.t_obs[0] - want) <= 1e-14 * abs(want)
        assert abs(r.maxnull[0] - want) <= 1e-14 * abs(want)


@pytest.mark.parametrize("n1,n2", [(10, 10), (7, 13), (3, 17)])
def test_identity_matches_scipy_pooled_t(n1, n2):
    X = synth.gaussian_mean_shift(n1 + n2, 300, seed=3).astype(np.float64)
    r = oracle.naive(X, n1, synth.identity_perm(n1 + n2))
    ref = st.ttest_ind(X[:n1], X[n1:], axis=0, equal_var=True).statistic
    np.testing.assert_allclose(r.t_obs, ref, rtol=1e-12, atol=1e-13)
    if n1 != n2:
        welch = st.ttest_ind(X[:n1], X[n1:], axis=0, equal_var=False).statistic
        assert np.max(np.abs(welch - r.t_obs)) > 1e-6  # pooled, not Welch


@pytest.mark.parametrize("two_sided", [False, True])
def test_rows_max_argmax_match_scipy(two_sided):
    n, n1, v, P = 16, 6, 400, 40
    X = synth.gaussian_mean_shift(n, v, seed=5)
    perms = synth.perms_pcg32(n, P, seed=9)
    r = oracle.naive(X, n1, perms, two_sided=two_sided)
    T = oracle.t_rows(X, n1, perms)
    Xd = X.astype(np.float64)
    for i in range(P):
        a, b = Xd[perms[i, :n1]], Xd[perms[i, n1:]]
        ref = st.ttest_ind(a, b, axis=0, equal_var=True).statistic
        np.testing.assert_allclose(T[i], ref, rtol=1e-12, atol=1e-13)
        s = np.abs(ref) if two_sided else ref
        assert r.argmax[i] == int(np.argmax(s))
        assert abs(r.maxnull[i] - s.max()) <= 1e-12 * abs(s.max())
    so = np.abs(r.t_obs) if two_sided else r.t_obs
    S = np.abs(T) if two_sided else T
    np.testing.assert_array_equal(r.counts, (S >= so[None, :]).sum(0))


def test_exact_enumeration_matches_scipy_permutation_test():
    """All C(10,5) relabellings: counts / 252 are scipy's exact p-values."""
    n, n1, v = 10, 5, 6
    X = synth.gaussian_mean_shift(n, v, seed=11).astype(np.float64)
    X[:n1, 0] += 1.5  # one voxel with signal
    perms = _combo_perms(n, n1)
    r = oracle.naive(X, n1, perms)
    assert perms.shape[0] == 252
    assert np.all(r.counts >= 1)  # the observed labelling is one of them
    for j in range(v):
        res = st.permutation_test(
            (X[:n1, j], X[n1:, j]),
            lambda a, b: st.ttest_ind(a, b, equal_var=True).statistic,
            permutation_type="independent", alternative="greater", n_resamples=np.inf)
        assert r.counts[j] == int(round(res.pvalue * 252)), j


def test_enumeration_symmetry_two_sided_counts():
    """Over all balanced relabellings the t distribution is symmetric, so the
    two-sided count equals #(t >= |t_obs|) + #(t <= -|t_obs|) = 2 #(t >= |t_obs|)."""
    n, n1, v = 10, 5, 8
    X = synth.gaussian_mean_shift(n, v, seed=12)
    perms = _combo_perms(n, n1)
    one = oracle.naive(X, n1, perms)
    two = oracle.naive(X, n1, perms, two_sided=True)
    T = oracle.t_rows(X, n1, perms)
    up = (T >= np.abs(one.t_obs)[None, :] - 1e-12).sum(0)
    np.testing.assert_array_equal(two.counts, 2 * up)


def test_label_swap_negates_t_exactly():
    n, n1, v = 12, 6, 200
    X = synth.gaussian_mean_shift(n, v, seed=13)
    perms = synth.perms_pcg32(n, 10, seed=2)
    swapped = np.concatenate([perms[:, n1:], perms[:, :n1]], axis=1)
    T = oracle.t_rows(X, n1, perms)
    Ts = oracle.t_rows(X, n1, swapped)
    np.testing.assert_array_equal(Ts, -T)


def test_same_group_set_gives_identical_t():
    """Group sums run in subject order, so reordering within the groups of a
    relabelling changes nothing (ties with the observed labelling are exact)."""
    n, n1, v = 14, 7, 100
    X = synth.gaussian_mean_shift(n, v, seed=14)
    base = synth.identity_perm(n)[0]
    shuf = np.concatenate([base[:n1][::-1], base[n1:][::-1]])[None, :].astype(np.int32)
    r = oracle.naive(X, n1, shuf)
    np.testing.assert_array_equal(r.counts, np.ones(v, np.uint32))


def test_null_uncorrected_pvalues_uniform():
    n, n1, v, P = 20, 10, 2000, 1000
    X = synth.gaussian_mean_shift(n, v, seed=1)
    perms = synth.perms_pcg32(n, P, seed=1)
    r = oracle.naive(X, n1, perms)
    p = (r.counts.astype(np.float64) + 1.0) / (P + 1.0)
    assert st.kstest(p, "uniform").pvalue > 1e-3


def test_degenerate_voxel_excluded():
    n, n1, v = 10, 5, 20
    X = synth.gaussian_mean_shift(n, v, seed=15)
    X[:, 3] = 0.25  # constant voxel
    X[:, 7] = 9.0
    perms = synth.perms_pcg32(n, 30, seed=4)
    r = oracle.naive(X, n1, perms)
    assert np.isnan(r.t_obs[3]) and np.isnan(r.t_obs[7])
    assert r.counts[3] == 0 and r.counts[7] == 0
    assert not np.any(np.isin(r.argmax, [3, 7]))
    keep = np.setdiff1d(np.arange(v), [3, 7])
    r2 = oracle.naive(X[:, keep], n1, perms)
    np.testing.assert_array_equal(r2.maxnull, r.maxnull)


def test_invalid_relabelling_rejected():
    n, n1 = 8, 4
    X = synth.gaussian_mean_shift(n, 10, seed=16)
    perms = synth.perms_pcg32(n, 5, seed=4)
    bad = perms.copy()
    bad[3, 2] = bad[3, 5]  # duplicate index
    with pytest.raises(ValueError):
        oracle.naive(X, n1, bad)
    bad = perms.copy()
    bad[1, 0] = n  # out of range
    with pytest.raises(ValueError):
        oracle.naive(X, n1, bad)


def test_pcg32_published_stream():
    """PCG32 XSH-RR seeded (42, 54): the first outputs published with the
    reference C implementation (pcg32-demo)."""
    got = synth.pcg32_raw(42, 54, 6)
    want = [0xa15c02b7, 0x7b47f409, 0xba1d3330, 0x83d2f293, 0xbfa4784b, 0xcbed606e]
    np.testing.assert_array_equal(got, np.array(want, dtype=np.uint32))


def test_fisher_yates_rows_are_permutations():
    p = synth.perms_pcg32(37, 500, seed=1)
    assert np.all(np.sort(p, axis=1) == np.arange(37)[None, :])
    # uniformity of the first position over 500 rows (chi-square, loose)
    cnt = np.bincount(p[:, 0], minlength=37)
    assert st.chisquare(cnt).pvalue > 1e-4


def test_fwer_pvalues_definition():
    """Corrected p-values: brute-force counting on a tiny case, the smallest
    attainable value 1/(P+1), monotone in t_obs, and the exact permutation
    distribution of the maximum over all C(8,4) relabellings."""
    rng = np.random.default_rng(5)
    m = rng.standard_normal(50).astype(np.float32)
    t = np.array([-1.0, 0.0, 0.3, 5.0, np.nan, float(m[7])])
    p = oracle.fwer_pvalues(m, t)
    for j, tj in enumerate(t):
        if np.isnan(tj):
            assert np.isnan(p[j])
        else:
            cnt = sum(1 for x in m if x >= np.float32(tj))
            assert p[j] == (1 + cnt) / 51.0
    assert p[3] == 1.0 / 51.0  # above every maximum
    assert p[0] >= p[1] >= p[2]
    p2 = oracle.fwer_pvalues(m, t, two_sided=True)
    assert p2[0] == (1 + np.sum(m >= 1.0)) / 51.0
    # exact: all C(8,4) relabellings (each group-1 set once, observed one included)
    import itertools
    n, n1, v = 8, 4, 30
    X = rng.standard_normal((n, v))
    X[:4, 3] += 3.0
    sets = [c for c in itertools.combinations(range(n), n1) if c != (0, 1, 2, 3)]
    perms = np.array([list(c) + [s for s in range(n) if s not in c] for c in sets],
                     dtype=np.int32)
    ref = oracle.naive(X, n1, perms)
    p = oracle.fwer_pvalues(ref.maxnull, ref.t_obs)
    allmax = np.concatenate([ref.maxnull, [np.max(ref.t_obs)]])
    for j in range(v):
        exact = np.mean(allmax.astype(np.float32) >= np.float32(ref.t_obs[j]))
        assert abs(p[j] - exact) < 1e-12


def test_resampling_risk_paper_examples():
    """Eq. (6) against the two worked values of Sec. 6: RapidPT rejecting 59 and
    SnPM 71 voxels (the 59 among the 71) gives 8.45%; 2158 among 2241 gives 1.85%."""
    for a, b, want in [(59, 71, 0.0845), (2158, 2241, 0.0185)]:
        v = 600000
        r_small = np.zeros(v, bool)
        r_small[:a] = True
        r_large = np.zeros(v, bool)
        r_large[:b] = True
        risk, v1, v2, vc = oracle.resampling_risk(r_small, r_large)
        assert (v1, v2, vc) == (a, b, a)
        assert round(100 * risk, 2) == round(100 * want, 2)
        assert oracle.resampling_risk(r_large, r_small)[0] == risk  # symmetric


def test_resampling_risk_special_cases():
    rng = np.random.default_rng(3)
    r = rng.random(1000) < 0.1
    assert oracle.resampling_risk(r, r)[0] == 0.0            # same decisions
    assert oracle.resampling_risk(r, ~r)[0] == 1.0           # disjoint rejections
    none = np.zeros(1000, bool)
    assert oracle.resampling_risk(none, none)[0] == 0.0
    assert oracle.resampling_risk(none, r)[0] == 0.5
    # brute force over a small case: the fraction of each method's rejections
    # that the other method does not reject, averaged
    a = rng.random(50) < 0.3
    b = rng.random(50) < 0.3
    miss_a = sum(1 for i in range(50) if a[i] and not b[i]) / max(1, a.sum())
    miss_b = sum(1 for i in range(50) if b[i] and not a[i]) / max(1, b.sum())
    assert abs(oracle.resampling_risk(a, b)[0] - (miss_a + miss_b) / 2) < 1e-15


def test_package_resampling_risk_matches_oracle():
    from paper_1703_01506_gb300 import metrics
    rng = np.random.default_rng(4)
    for _ in range(20):
        p1 = rng.random(5000)
        p2 = np.clip(p1 + rng.normal(0, 0.02, 5000), 0, 1)
        p1[rng.random(5000) < 0.01] = np.nan
        for alpha in (0.01, 0.05, 0.2):
            got = metrics.resampling_risk(p1, p2, alpha)
            want = oracle.resampling_risk(p1 <= alpha, p2 <= alpha)  # NaN <= alpha is False
            assert got["risk"] == want[0] and (got["v1"], got["v2"], got["vc"]) == want[1:]
