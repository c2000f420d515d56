"""RapidPT oracle (test infrastructure only): plain numpy FP64 statement of
Alg. 2 (Sec. 4.1 training, Sec. 4.2 recovery).

The paper cites GROUSE/GRASTA for its subspace tracking and gives no formulas
(its supplement is not available), so the tracking step below is one explicit
reading, written out the same way on both sides:

* weights (``Complete``): the l1 fit min_w ||U_O w - b||_1 solved by ADMM on
  min ||s||_1 s.t. U_O w + s = b (scaled dual y, penalty rho, fixed iterations):
      w <- (U_O^T U_O)^{-1} U_O^T (b - s - y/rho)
      s <- soft(b - U_O w - y/rho, 1/rho)
      y <- y + rho (U_O w + s - b)
* update of U (training only): a rank-one geodesic step on the Grassmannian
  towards the residual of that fit, r = b - U_O w, lifted to all voxels
  (entries summed where a voxel was drawn twice) and projected off span(U):
      Gamma = lift(r) - U (U_O^T r),  theta = step * arctan(||r|| / ||w||),
      U <- U + [(cos theta - 1) U w / ||w|| + sin theta Gamma / ||Gamma||] w^T / ||w||
  (||w|| = ||U w||, the full prediction, as in GROUSE; with every voxel
  sampled and step 1 the new span contains the fitted column exactly), a QR
  re-orthonormalisation (positive diagonal of R) every qr_every steps and
  after the last one, and several passes over the training columns (Sec. 4.1:
  "multiple passes over the training set ... until convergence"; Alg. 2
  lists one).
* sampling: the ceil(eta v) voxels of a column are drawn i.i.d. UNIF over the
  voxels (Alg. 2 writes k ~ UNIF[1, v]); random numbers come from the
  counter-based generator Philox4x32-10 (Salmon et al., SC 2011), keyed by the
  seed, with a per-use counter, as documented in ``draws``.
* after training: W_ex = U^T T_ex (least squares, U orthonormal), residual
  R = T_ex - U W_ex, sigma = std of R at the entries sampled in the last pass
  (Alg. 2, "{T_ex - U W_ex}_Omega"), and the shift mu either literally as in
  Alg. 2 (shift_mode 0: the largest residual over all training entries) or as
  the amount the maximum moves (shift_mode 1, Sec. 4.1 "Bias-variance
  trade-off": the mean over training columns of max_j T_ex minus the maximum
  of the model U W_ex + sigma z).
* recovery (Sec. 4.2, Alg. 2): per later relabelling, exact t at its sampled
  voxels, w = Complete(U, t, Omega) with U frozen, T_hat = U w + s with s
  i.i.d. N(0, sigma^2), m_i = max_j T_hat + mu; training columns enter the
  max-null exactly (m_i = max_j T_ex[i, j], no mu).

Voxels are the ones with a defined t (not all values equal), in mask order.
"""
import math

import numpy as np

from . import t_rows, t_entries, voxel_major

MASK32 = np.uint64(0xFFFFFFFF)
PHILOX_M0, PHILOX_M1 = np.uint64(0xD2511F53), np.uint64(0xCD9E8D57)
PHILOX_W0, PHILOX_W1 = np.uint64(0x9E3779B9), np.uint64(0xBB67AE85)

TAG_U0, TAG_TRAIN, TAG_REC, TAG_NOISE, TAG_SHIFT = 1, 2, 3, 4, 5


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds (Random123). All arguments are arrays (or
    scalars) of uint32 values held in uint64; returns the four output words."""
    c0, c1, c2, c3 = (np.asarray(x, dtype=np.uint64) & MASK32 for x in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & MASK32
    k1 = np.asarray(k1, dtype=np.uint64) & MASK32
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3


def _key(seed):
    seed = int(seed)
    return np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF)


class draws:
    """The random numbers of the method, by counter (a, b, c, tag):

    normal(tag, a, b)      z = sqrt(-2 ln u1) cos(2 pi u2) from words (x0, x1),
                           u1 = (x0 + 1) 2^-32, u2 = x1 2^-32   (counter (a, b, 0, tag))
    voxel_normal(tag, j, b) one counter (floor(j / 4), b, 0, tag) serves four
                           voxels: words (x0, x1) give the Box-Muller pair of
                           voxels 4p, 4p + 1 and words (x2, x3) that of 4p + 2,
                           4p + 3; in each pair sqrt(-2 ln u1) cos(2 pi u2) for the
                           even voxel and sqrt(-2 ln u1) sin(2 pi u2) for the odd
                           one, u1 = (first word + 1) 2^-32, u2 = second word 2^-32
    index(tag, q, i, p, v) floor((x1 2^32 + x0) v / 2^64)         (counter (q, i, p, tag))

    U0[j, c]            = normal(TAG_U0, j, c)
    training sample q   = index(TAG_TRAIN, q, i, pass, v)   of column i in a pass
    recovery sample q   = index(TAG_REC, q, i, 0, v)        of relabelling i
    recovery noise      = voxel_normal(TAG_NOISE, j, i)     at voxel j, relabelling i
    shift-estimate noise= voxel_normal(TAG_SHIFT, j, i)     at voxel j, training column i
    """

    def __init__(self, seed):
        self.k0, self.k1 = _key(seed)

    def words(self, a, b, c, tag):
        return philox4x32_10(a, b, c, np.uint64(tag), self.k0, self.k1)

    def normal(self, tag, a, b):
        x0, x1, _, _ = self.words(a, b, 0, tag)
        u1 = (x0.astype(np.float64) + 1.0) * 2.0 ** -32
        u2 = x1.astype(np.float64) * 2.0 ** -32
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)

    def voxel_normal(self, tag, j, b):
        j = np.asarray(j, dtype=np.uint64)
        x0, x1, x2, x3 = self.words(j >> np.uint64(2), b, 0, tag)
        second = ((j >> np.uint64(1)) & np.uint64(1)) == 1  # voxels 4p + 2, 4p + 3
        a = np.where(second, x2, x0)
        c = np.where(second, x3, x1)
        u1 = (a.astype(np.float64) + 1.0) * 2.0 ** -32
        u2 = c.astype(np.float64) * 2.0 ** -32
        r = np.sqrt(-2.0 * np.log(u1))
        return np.where((j & np.uint64(1)) == 0, r * np.cos(2.0 * np.pi * u2),
                        r * np.sin(2.0 * np.pi * u2))

    def index(self, tag, q, i, p, v):
        x0, x1, _, _ = self.words(q, i, p, tag)
        v = np.uint64(v)
        # floor((x1 * 2^32 + x0) * v / 2^64) with exact 64-bit pieces
        return ((x1 * v + ((x0 * v) >> np.uint64(32))) >> np.uint64(32)).astype(np.int64)


def qr_posdiag(A):
    """Orthonormal factor of A with the diagonal of R made positive (unique)."""
    Q, R = np.linalg.qr(A)
    d = np.sign(np.diag(R))
    d[d == 0] = 1.0
    return Q * d[None, :]


def soft(x, tau):
    return np.sign(x) * np.maximum(np.abs(x) - tau, 0.0)


def admm_l1(A, b, rho, iters):
    """GRASTA-style ADMM for min ||s||_1 s.t. A w + s = b (scaled dual y)."""
    G = A.T @ A
    C = np.linalg.cholesky(G)
    s = np.zeros_like(b)
    y = np.zeros_like(b)
    w = np.zeros(A.shape[1])
    for _ in range(iters):
        rhs = A.T @ (b - s - y / rho)
        w = np.linalg.solve(C.T, np.linalg.solve(C, rhs))
        Aw = A @ w
        s = soft(b - Aw - y / rho, 1.0 / rho)
        y = y + rho * (Aw + s - b)
    return w, s, y


def geodesic_step(U, idx, b, w, step):
    """Rank-one Grassmannian update of U towards the residual of the fit."""
    UO = U[idx]
    Uw_O = UO @ w
    r = b - Uw_O
    lift = np.zeros(U.shape[0])
    np.add.at(lift, idx, r)
    Gam = lift - U @ (UO.T @ r)
    nG, nw, nr = (np.linalg.norm(x) for x in (Gam, w, r))
    if nG == 0.0 or nw == 0.0:
        return U
    theta = step * math.atan(nr / nw)
    p = U @ w
    dirv = (math.cos(theta) - 1.0) * p / nw + math.sin(theta) * Gam / nG
    return U + np.outer(dirv, w / nw)


class RapidOpts:
    def __init__(self, train_passes=1, qr_every=100, admm_iters=30, admm_rho=2.0, step=1.0,
                 shift_mode=1, seed=1, stat="t", rec_step=0.0):
        """stat: the statistic whose permutation matrix is modelled, "t" or "u"
        (see _stat_fns); maxima are reported as t either way. rec_step: 0 keeps
        U frozen during recovery (Alg. 2 as printed); > 0 takes a geodesic
        step of that size after every recovery fit (sequential updates, the
        training step applied to the recovery samples)."""
        self.train_passes, self.qr_every = train_passes, qr_every
        self.admm_iters, self.admm_rho, self.step = admm_iters, admm_rho, step
        self.shift_mode, self.seed, self.stat = shift_mode, seed, stat
        self.rec_step = rec_step


class RapidResult:
    pass


def valid_voxels(X):
    Xd = np.asarray(X, dtype=np.float64)
    return ~np.all(Xd == Xd[:1], axis=0)


def _stat_fns(X, n1, perms, o):
    """The modelled statistic: rows(sel) gives its rows for relabellings sel,
    entries(i, idx) its values at voxels idx under relabelling i, and to_t maps
    a (maximum) value of it to the t statistic.
      "t"        -- Eq. 5's pooled t itself (to_t = identity);
      "u"        -- the group-1 share of the unit-norm centred voxel,
                    u = t / sqrt(k (n-2) + k t^2), k = 1/n1 + 1/n2: linear in
                    the relabelling, so its matrix has rank <= n - 1 exactly
                    (the low-rank structure of Sec. 3.2 without the t
                    non-linearity); t = sqrt(k (n-2)) u / sqrt(1 - k u^2) is
                    strictly increasing and the same at every voxel, so the
                    maximum of t over voxels is t(maximum of u);
      "meandiff" -- mean(group 1) - mean(group 2), linear (test statistic).
    """
    n = X.shape[0]
    valid = valid_voxels(X)
    Xt = voxel_major(X[:, valid])
    k = 1.0 / n1 + 1.0 / (n - n1)

    def to_t(u):
        u = np.asarray(u, dtype=np.float64)
        ku2 = k * u * u
        with np.errstate(divide="ignore", invalid="ignore"):
            t = math.sqrt(k * (n - 2)) * u / np.sqrt(1.0 - ku2)
        return np.where(ku2 >= 1.0, np.sign(u) * np.inf, t)

    def u_of(t):
        return t / np.sqrt(k * (n - 2) + k * t * t)

    if o.stat in ("t", "u"):
        f = u_of if o.stat == "u" else (lambda t: t)

        def rows(sel):
            return f(t_rows(None, n1, sel, Xt=Xt))

        def entries(i, idx):
            return f(t_entries(Xt, n1, perms, np.full(idx.size, i), idx))
    else:  # "meandiff": mean(group 1) - mean(group 2), a linear statistic (T has rank <= n-1)
        def rows(sel):
            Lm = np.full(sel.shape, -1.0 / (n - n1))
            Lm[:, :n1] = 1.0 / n1
            Lw = np.zeros((sel.shape[0], n))
            np.put_along_axis(Lw, sel, Lm, axis=1)
            return Lw @ Xt.T

        def entries(i, idx):
            return rows(perms[i:i + 1])[0, idx]
    if o.stat != "u":
        to_t = lambda x: np.asarray(x, dtype=np.float64)  # noqa: E731
    return valid, Xt, rows, entries, to_t


def training_summary(T_ex, U, last_idx, shift_mode, dr):
    """What Alg. 2 computes once the basis is trained (Sec. 4.1): the training
    weights by least squares, W_ex = U^T T_ex (U orthonormal); the residual
    R = T_ex - U W_ex; sigma = population standard deviation of R over the
    entries Omega sampled in the last pass (last_idx[i] = the voxels drawn for
    column i, repeats counted as drawn); and the shift mu:
      shift_mode 0 -- as Alg. 2 prints it, the largest residual over every
                      training entry: sup_i max_j R[i, j];
      shift_mode 1 -- the amount the maximum moves (Sec. 4.1, "Bias-variance
                      trade-off"): mean over training columns i of
                      max_j T_ex[i, j] - max_j (U W_ex[:, i] + sigma z_ij)_j,
                      z_ij = voxel_normal(TAG_SHIFT, j, i).
    T_ex is (ell x V), U (V x r). Returns (W_ex (r x ell), sigma, mu)."""
    ell, V = T_ex.shape
    W_ex = U.T @ T_ex.T                       # r x ell
    model = (U @ W_ex).T                      # ell x V
    R = T_ex - model
    sampled = np.concatenate([R[i, last_idx[i]] for i in range(ell)])
    sigma = float(np.std(sampled))
    if shift_mode == 0:
        mu = float(np.max(R))
    else:
        gaps = np.empty(ell)
        for i in range(ell):
            z = dr.voxel_normal(TAG_SHIFT, np.arange(V), i)
            gaps[i] = np.max(T_ex[i]) - np.max(model[i] + sigma * z)
        mu = float(np.mean(gaps))
    return W_ex, sigma, mu


def rapid_train(X, n1, perms, rank, sample_rate, n_train, opts=None):
    """Training phase (Sec. 4.1, Alg. 2 TRAINING): U, W_ex, sigma, mu from the
    first n_train relabellings. Returns a RapidResult (U, W_ex, T_ex, sigma, mu,
    m, steps, w_hist = per-step weights, counts over the training rows)."""
    o = opts or RapidOpts()
    X = np.asarray(X)
    n = X.shape[0]
    valid, Xt, rows, _, to_t = _stat_fns(X, n1, perms, o)
    V = Xt.shape[0]
    m = int(math.ceil(sample_rate * V))
    dr = draws(o.seed)
    ell = n_train
    # Training set: ell columns of T computed in full (Sec. 4.1)
    T_ex = rows(perms[:ell])
    jj, cc = np.meshgrid(np.arange(V), np.arange(rank), indexing="ij")
    U = qr_posdiag(dr.normal(TAG_U0, jj, cc))
    steps = 0
    w_hist = []
    last_idx = [None] * ell
    for p in range(o.train_passes):
        for i in range(ell):
            idx = dr.index(TAG_TRAIN, np.arange(m), i, p, V)
            b = T_ex[i, idx]
            w, _, _ = admm_l1(U[idx], b, o.admm_rho, o.admm_iters)
            w_hist.append(w.copy())
            U = geodesic_step(U, idx, b, w, o.step)
            steps += 1
            if steps % o.qr_every == 0:
                U = qr_posdiag(U)
            last_idx[i] = idx
    U = qr_posdiag(U)
    W_ex, sigma, mu = training_summary(T_ex, U, last_idx, o.shift_mode, dr)
    T_obs = rows(np.arange(n, dtype=np.int32)[None, :])[0]
    counts = np.zeros(X.shape[1], dtype=np.int64)
    counts[np.flatnonzero(valid)] = (T_ex >= T_obs[None, :]).sum(axis=0)
    res = RapidResult()
    res.U, res.W_ex, res.T_ex, res.sigma, res.mu, res.m = U, W_ex, T_ex, sigma, mu, m
    res.steps, res.w_hist, res.counts = steps, w_hist, counts
    res.train_max = to_t(T_ex.max(axis=1))
    return res


def rapid_recover(X, n1, perms, rows_sel, U, sigma, mu, m, opts=None, return_w=False):
    """Recovery phase (Sec. 4.2, Alg. 2 RECOVERY) for relabellings rows_sel with
    U frozen: exact statistic at the m sampled voxels, w = Complete(U, t, Omega),
    m_i = max_j (U w + sigma z)_j + mu (mapped to t when the modelled
    statistic is u).

    With opts.rec_step > 0 the relabellings are taken in order and, after
    each one's maximum is formed with the current U, U takes the training
    step (geodesic_step with step rec_step) towards that relabelling's fit
    residual on its samples; QR every qr_every recovery steps. The rows then
    depend on the ones before them."""
    o = opts or RapidOpts()
    X = np.asarray(X)
    _, Xt, _, entries, to_t = _stat_fns(X, n1, perms, o)
    V = Xt.shape[0]
    dr = draws(o.seed)
    out = np.empty(len(rows_sel))
    ws = []
    steps = 0
    for k, i in enumerate(rows_sel):
        idx = dr.index(TAG_REC, np.arange(m), int(i), 0, V)
        tt = entries(int(i), idx)
        w, _, _ = admm_l1(U[idx], tt, o.admm_rho, o.admm_iters)
        ws.append(w)
        z = dr.voxel_normal(TAG_NOISE, np.arange(V), int(i))
        out[k] = to_t(np.max(U @ w + sigma * z) + mu)
        if o.rec_step > 0.0:
            U = geodesic_step(U, idx, tt, w, o.rec_step)
            steps += 1
            if steps % o.qr_every == 0:
                U = qr_posdiag(U)
    return (out, np.array(ws)) if return_w else out


def rapid(X, n1, perms, rank, sample_rate, n_train, opts=None, keep=False):
    """RapidPT (Alg. 2) over relabellings ``perms`` (P x n); first n_train rows train.

    Returns a RapidResult with maxnull (P; training rows exact, no shift),
    counts (exceedances over the n_train exactly computed rows, per mask
    voxel), sigma, mu, m (samples per column), and with keep=True the
    training state (U, W_ex, T_ex, w_hist).
    """
    o = opts or RapidOpts()
    P = perms.shape[0]
    assert 1 <= n_train < P and rank >= 1
    tr = rapid_train(X, n1, perms, rank, sample_rate, n_train, o)
    maxnull = np.empty(P)
    maxnull[:n_train] = tr.train_max
    maxnull[n_train:] = rapid_recover(X, n1, perms, range(n_train, P), tr.U, tr.sigma, tr.mu,
                                      tr.m, o)
    res = RapidResult()
    res.maxnull, res.counts, res.sigma, res.mu, res.m = maxnull, tr.counts, tr.sigma, tr.mu, tr.m
    res.steps = tr.steps
    if keep:
        res.U, res.W_ex, res.T_ex, res.w_hist = tr.U, tr.W_ex, tr.T_ex, tr.w_hist
    return res


def kl_divergence(p_samples, q_samples, bins=100, eps=1e-10):
    """KL(P || Q) between two samples' histograms on a common equal-width grid
    over [min, max] of the union; eps added to every bin before normalising."""
    lo = min(np.min(p_samples), np.min(q_samples))
    hi = max(np.max(p_samples), np.max(q_samples))
    hp, _ = np.histogram(p_samples, bins=bins, range=(lo, hi))
    hq, _ = np.histogram(q_samples, bins=bins, range=(lo, hi))
    pp = (hp + eps) / (hp + eps).sum()
    qq = (hq + eps) / (hq + eps).sum()
    return float(np.sum(pp * np.log(pp / qq)))


def fwer_threshold(maxnull, alpha):
    """The c-th largest max-null value, c = floor(alpha P) + 1."""
    s = np.sort(np.asarray(maxnull))[::-1]
    c = int(math.floor(alpha * s.size)) + 1
    return float(s[min(c, s.size) - 1])
