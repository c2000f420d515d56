"""Oracle for the general-contrast form of the statistic: the two-group t with
nuisance covariates (test infrastructure only; see ``oracle/__init__.py``).

The paper computes a "stat" per relabelling and voxel (Sec. 3.2 takes the
two-sample t as its instance; Alg. 1/2 take the statistic as an input). With
covariates Z (n x q, an intercept always added) the statistic of a relabelling
with group-1 indicator l is the t of beta in the least-squares fit

    y = beta l + [1, Z] gamma + e,      t = beta_hat / se(beta_hat),
    se^2 = RSS / (n - q - 2) * [(D^T D)^{-1}]_{00},   D = [l, 1, Z],

i.e. the group column is relabelled and the covariates stay with their
subjects. With q = 0 this is the pooled two-sample t of Eq. (5).

Plain FP64 numpy: one least-squares solve per relabelling (numpy.linalg.lstsq
as a library step), all voxels at once.
"""
import numpy as np


def design_base(Z, n):
    """[1, Z] (n x (q+1)); Z may be None or have zero columns."""
    if Z is None:
        return np.ones((n, 1))
    Z = np.asarray(Z, dtype=np.float64).reshape(n, -1)
    return np.column_stack([np.ones(n), Z])


def glm_t_rows(X, Z, n1, perms):
    """T (P x v, FP64): the t of the group coefficient for every relabelling
    row of ``perms`` (group 1 = its first n1 entries) and every voxel."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    C = design_base(Z, n)
    perms = np.asarray(perms)
    T = np.empty((perms.shape[0], v))
    dead = degenerate_voxels(X, C)
    for i, row in enumerate(perms):
        lab = np.zeros(n)
        lab[row[:n1]] = 1.0
        D = np.column_stack([lab, C])
        beta, _, rank, _ = np.linalg.lstsq(D, X, rcond=None)
        if rank < D.shape[1]:
            raise ValueError("relabelling %d: group column in the span of the covariates" % i)
        E = X - D @ beta
        rss = np.einsum("sj,sj->j", E, E)
        df = n - D.shape[1]
        g00 = np.linalg.inv(D.T @ D)[0, 0]
        with np.errstate(divide="ignore", invalid="ignore"):
            T[i] = beta[0] / np.sqrt(rss / df * g00)
        T[i, dead] = np.nan
    return T


def degenerate_voxels(X, C):
    """Voxels without a statistic: all n values equal, or values in the span of
    [1, Z] (residual sum of squares at most 1e-24 of the centred one, decided
    in FP64)."""
    X = np.asarray(X, dtype=np.float64)
    const = np.all(X == X[0], axis=0)
    Q, _ = np.linalg.qr(C)
    R = X - Q @ (Q.T @ X)
    Xc = X - X.mean(axis=0)
    ss_r = np.einsum("sj,sj->j", R, R)
    ss_c = np.einsum("sj,sj->j", Xc, Xc)
    return const | (ss_r <= 1e-24 * ss_c)


def glm_t_obs(X, Z, n1):
    """The observed statistic (identity labelling: subjects 0..n1-1 in group 1)."""
    n = np.asarray(X).shape[0]
    return glm_t_rows(X, Z, n1, np.arange(n)[None, :])[0]


class GlmResult:
    """maxnull / argmax (smallest voxel on ties) / second (runner-up value) per
    row, counts #{i : stat_ij >= stat_obs_j} per voxel, t_obs, the full T, and
    the per-row scale a_i = ||R l_i||^2 (R = I - H_[1,Z]) with df."""

    def __init__(self, **kw):
        self.__dict__.update(kw)

    def z_of(self, t, rows):
        """The library's comparison scale for row i: w_i sqrt(a_obs) with
        w = t / sqrt(df + t^2) = (group-1 share of the unit residual) / sqrt(a_i)."""
        t = np.asarray(t, dtype=np.float64)
        w = t / np.sqrt(self.df + t * t)
        return w * np.sqrt(self.a_obs) * np.ones_like(self.a[rows])

    def u_of(self, t, rows):
        """Group-1 share u = w sqrt(a_i) of the unit-norm residual voxel (the
        contraction's value; the row maximum of t sits at the row maximum of u)."""
        t = np.asarray(t, dtype=np.float64)
        w = t / np.sqrt(self.df + t * t)
        return w * np.sqrt(self.a[rows])


def residual_scale(Z, n, n1, perms):
    """a_i = ||(I - H) l_i||^2 for every relabelling (H the projector on [1, Z])."""
    C = design_base(Z, n)
    Q, _ = np.linalg.qr(C)
    out = np.empty(len(perms))
    for i, row in enumerate(perms):
        lab = np.zeros(n)
        lab[np.asarray(row)[:n1]] = 1.0
        out[i] = lab @ lab - np.sum((Q.T @ lab) ** 2)
    return out


def glm_naive(X, Z, n1, perms, two_sided=False):
    """NaivePT (Alg. 1) with the covariate-adjusted statistic."""
    X = np.asarray(X, dtype=np.float64)
    n, v = X.shape
    perms = np.asarray(perms)
    T = glm_t_rows(X, Z, n1, perms)
    t_obs = glm_t_obs(X, Z, n1)
    S = np.abs(T) if two_sided else T
    s_obs = np.abs(t_obs) if two_sided else t_obs
    S = np.where(np.isnan(S), -np.inf, S)
    order = np.argsort(-S, axis=1, kind="stable")
    argmax = order[:, 0]
    rows = np.arange(S.shape[0])
    maxnull = S[rows, argmax]
    second = S[rows, order[:, 1]] if v > 1 else np.full(S.shape[0], -np.inf)
    counts = (S >= s_obs[None, :]).sum(axis=0)
    q = design_base(Z, n).shape[1] - 1
    a = residual_scale(Z, n, n1, perms)
    a_obs = residual_scale(Z, n, n1, np.arange(n)[None, :])[0]
    return GlmResult(maxnull=maxnull, argmax=argmax, second=second, counts=counts,
                     t_obs=t_obs, T=T, a=a, a_obs=a_obs, df=n - q - 2, n=n, n1=n1)
