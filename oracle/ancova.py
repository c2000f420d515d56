"""F of a g-group factor with nuisance covariates (one-way ANCOVA) under
relabellings (test infrastructure only; see ``oracle/__init__.py``).

Alg. 1 and 2 take the voxel statistic as an input ("stat"; Sec. 3.2 uses the
two-sample t as its instance). For g groups of fixed sizes and covariates Z
(n x q, an intercept always added) the statistic of a relabelling is the F of
the factor in the least-squares fit

    full:    y = E beta + [1, Z] gamma + e,   E = indicators of groups 1..g-1,
    reduced: y = [1, Z] gamma + e,

    F = ((RSS_reduced - RSS_full) / (g - 1)) / (RSS_full / (n - g - q)),

with the relabelled rows of E and every subject keeping its covariate values.
A relabelling row is a permutation of the n subjects: its first n_1 entries
form group 1, the next n_2 group 2, and so on (the identity is the observed
labelling). Without covariates this is the one-way F of oracle/anova.py; with
g = 2 it is the square of the covariate-adjusted t of oracle/glm.py.

Plain FP64 numpy: two least-squares solves per relabelling (numpy.linalg.lstsq
as a library step), all voxels at once. The comparison scale for near-ties is
B = (RSS_reduced - RSS_full) / RSS_reduced in [0, 1]: F = B (n - g - q) /
((1 - B)(g - 1)), strictly increasing.
"""
import numpy as np

from oracle import glm as G


class AncovaResult:
    pass


def _indicators(row, sizes):
    row = np.asarray(row)
    n = row.size
    assert sorted(row.tolist()) == list(range(n)), "not a permutation"
    bounds = np.concatenate([[0], np.cumsum(sizes)])
    E = np.zeros((n, len(sizes) - 1))
    for h in range(len(sizes) - 1):
        E[row[bounds[h]:bounds[h + 1]], h] = 1.0
    return E


def df_of(n, sizes, Z):
    q = G.design_base(Z, n).shape[1] - 1
    return n - len(sizes) - q


def f_rows(X, sizes, Z, perms):
    """F (P x v, FP64) of the factor for every relabelling row and voxel; NaN
    where the voxel has no statistic (glm.degenerate_voxels)."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    g = len(sizes)
    assert sum(sizes) == n and g >= 2 and min(sizes) >= 1
    C = G.design_base(Z, n)
    df = n - g - (C.shape[1] - 1)
    assert df >= 1
    dead = G.degenerate_voxels(X, C)
    Rr = X - C @ np.linalg.lstsq(C, X, rcond=None)[0]
    rss_red = np.einsum("sj,sj->j", Rr, Rr)
    out = np.empty((len(perms), v))
    for i, row in enumerate(perms):
        D = np.column_stack([_indicators(row, sizes), C])
        beta, _, rank, _ = np.linalg.lstsq(D, X, rcond=None)
        if rank < D.shape[1]:
            raise ValueError("relabelling %d: group columns in the span of the covariates" % i)
        Rf = X - D @ beta
        rss_full = np.einsum("sj,sj->j", Rf, Rf)
        with np.errstate(divide="ignore", invalid="ignore"):
            F = ((rss_red - rss_full) / (g - 1)) / (rss_full / df)
        F[dead] = np.nan
        out[i] = F
    return out


def b_of_f(F, n, sizes, Z):
    """B = (RSS_reduced - RSS_full) / RSS_reduced for a given F (exact inverse)."""
    F = np.asarray(F, dtype=np.float64)
    a = F * (len(sizes) - 1) / df_of(n, sizes, Z)
    return np.where(np.isinf(F), 1.0, a / (1.0 + a))


def ancova(X, sizes, Z, perms):
    """Max-null of F over voxels, argmax (smallest voxel on ties), runner-up,
    counts F >= F_obs, F_obs and the full F."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    F = f_rows(X, sizes, Z, perms)
    F_obs = f_rows(X, sizes, Z, np.arange(n)[None, :])[0]
    Fm = np.where(np.isnan(F), -np.inf, F)
    res = AncovaResult()
    rows = np.arange(F.shape[0])
    res.argmax = np.argmax(Fm, axis=1)
    res.maxnull = Fm[rows, res.argmax]
    Fs = Fm.copy()
    Fs[rows, res.argmax] = -np.inf
    res.second = Fs.max(axis=1)
    with np.errstate(invalid="ignore"):
        res.counts = np.where(np.isnan(F_obs)[None, :], False, F >= F_obs[None, :]).sum(axis=0)
    res.F_obs = F_obs
    res.F = F
    return res
