"""F statistic of a one-way layout with g groups, under relabellings (test
infrastructure only).

Alg. 1 and 2 take the voxel statistic as an input ("stat"); Sec. 3.2 uses the
two-sample t as one instance. With g groups of fixed sizes n_1..n_g the
per-voxel statistic is the one-way ANOVA F:

    F = (SS_between / (g - 1)) / (SS_within / (n - g)),
    SS_between = sum_h n_h (mean_h - mean)^2,
    SS_within  = sum_h sum_{s in group h} (x_s - mean_h)^2,

computed here in FP64 with two passes over each group, per relabelling and
voxel. A relabelling row is a permutation of the n subjects: its first n_1
entries form group 1, the next n_2 group 2, and so on; the observed labelling
is the identity. Outputs mirror the two-sample oracle: the max-null of F
with its argmax (smallest voxel on ties) and runner-up, the per-voxel counts
#{i : F_ij >= F_obs_j}, F_obs, and for near-tie checks the statistic on the
scale B = SS_between / SS_total (F = B (n - g) / ((1 - B)(g - 1)), strictly
increasing). Voxels whose values are all equal have no F (NaN, no count).
"""
import numpy as np


class AnovaResult:
    pass


def _groups(row, sizes):
    row = np.asarray(row)
    assert sorted(row.tolist()) == list(range(row.size)), "not a permutation"
    bounds = np.concatenate([[0], np.cumsum(sizes)])
    return [row[bounds[h]:bounds[h + 1]] for h in range(len(sizes))]


def f_rows(X, sizes, perms):
    """F of every voxel (columns of X, n x v) under every relabelling: (P, v)."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    g = len(sizes)
    assert sum(sizes) == n and g >= 2 and min(sizes) >= 1 and n > g
    const = np.all(X == X[:1], axis=0)
    out = np.empty((len(perms), v))
    for i, row in enumerate(perms):
        grp = _groups(row, sizes)
        mean = X.mean(axis=0)
        ssb = np.zeros(v)
        ssw = np.zeros(v)
        for idx in grp:
            Xg = X[idx]
            mg = Xg.mean(axis=0)
            ssb += len(idx) * (mg - mean) ** 2
            ssw += ((Xg - mg) ** 2).sum(axis=0)
        with np.errstate(divide="ignore", invalid="ignore"):
            F = (ssb / (g - 1)) / (ssw / (n - g))
        F[const] = np.nan
        out[i] = F
    return out


def b_of_f(F, n, g):
    """B = SS_between / SS_total for a given F (the exact inverse map)."""
    F = np.asarray(F, dtype=np.float64)
    a = F * (g - 1) / (n - g)
    return np.where(np.isinf(F), 1.0, a / (1.0 + a))


def anova(X, sizes, perms):
    """Max-null of F over voxels, argmax, runner-up, counts F >= F_obs, F_obs."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    F = f_rows(X, sizes, perms)
    F_obs = f_rows(X, sizes, np.arange(n)[None, :])[0]
    Fm = np.where(np.isnan(F), -np.inf, F)
    res = AnovaResult()
    res.argmax = np.argmax(Fm, axis=1)
    res.maxnull = Fm[np.arange(F.shape[0]), res.argmax]
    Fs = Fm.copy()
    Fs[np.arange(F.shape[0]), res.argmax] = -np.inf
    res.second = Fs.max(axis=1)
    with np.errstate(invalid="ignore"):
        res.counts = np.where(np.isnan(F_obs)[None, :], False, F >= F_obs[None, :]).sum(axis=0)
    res.F_obs = F_obs
    res.F = F
    return res
