"""Oracle: plain, slow, FP64 CPU statement of the permutation-testing path.

Test infrastructure only. Tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import it; the product package never does,
and nothing here imports the product package except its seeded input
generators (``paper_1703_01506_gb300.synth``), which hold none of the
method's arithmetic.

* ``naive``  -- NaivePT (Alg. 1) with the pooled-variance t of Eq. (5), in C
  (``naive_fp64.c``) behind ctypes.
* ``rapid``  -- RapidPT (Alg. 2, Sec. 4.1-4.2) in numpy FP64, with the
  counter-based generator (Philox4x32-10) both sides implement.
* ``cluster`` -- clusters of thresholded maps (Sec. 6 cluster tables) and the
  largest cluster per relabelling, with scipy's connected-component labelling.
* ``glm``, ``anova``, ``ancova`` -- other instances of the per-voxel "stat"
  (Alg. 1/2 input): the two-group t with nuisance covariates, the one-way F of
  g groups, and the F of a g-group factor with nuisance covariates, each from
  its least-squares or sums-of-squares definition in FP64.
"""

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle_naive.so")
_SRC = os.path.join(_HERE, "naive_fp64.c")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, f64 = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_naive.restype = i64
            lib.oracle_naive.argtypes = [P, i32, i64, i32, P, i64, i32, i32, f64,
                                         P, P, P, P, P, P, P]
            lib.oracle_t_rows.restype = i64
            lib.oracle_t_rows.argtypes = [P, i32, i64, i32, P, i64, i32, P]
            lib.oracle_t_entries.restype = i64
            lib.oracle_t_entries.argtypes = [P, i32, i64, i32, P, P, P, i64, P]
            _lib = lib
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def voxel_major(X):
    """FP64 voxel-major copy (v x n) of subject-major data X (n x v)."""
    return np.ascontiguousarray(np.asarray(X, dtype=np.float64).T)


class NaiveResult:
    """Outputs of :func:`naive` (all numpy arrays)."""

    def __init__(self, maxnull, argmax, second, counts, t_obs, near, tau, n, n1):
        self.maxnull, self.argmax, self.second = maxnull, argmax, second
        self.counts, self.t_obs, self.near, self.tau = counts, t_obs, near, tau
        self.n, self.n1 = n, n1

    def u_of(self, t):
        """Monotone rescaling u = t / sqrt(k(n-2) + k t^2) (group-1 share of the
        unit-norm centred voxel); near-ties are judged on this scale."""
        k = 1.0 / self.n1 + 1.0 / (self.n - self.n1)
        t = np.asarray(t, dtype=np.float64)
        with np.errstate(invalid="ignore"):
            u = t / np.sqrt(k * (self.n - 2) + k * t * t)
        return np.where(np.isinf(t), np.sign(t) / np.sqrt(k), u)


def naive(X, n1, perms, two_sided=False, nthreads=0, tie_rel=0.0):
    """NaivePT (Alg. 1) over the rows of ``perms``.

    X: (n, v) data, subject-major (any float dtype; promoted to FP64).
    perms: (P, n) int32; group 1 = first n1 entries of each row.
    Returns a :class:`NaiveResult` with maxnull (FP64, t or |t|), argmax
    (smallest voxel on ties), second (runner-up value for near-tie checks),
    counts (#{i: stat_ij >= stat_obs_j}), t_obs, tau (per-voxel tie band
    tie_rel * l1 norm of the unit-norm centred voxel) and near (entries whose
    u lies within tau of the observed u).
    """
    lib = _load()
    Xt = voxel_major(X)
    v, n = Xt.shape
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    P = perms.shape[0]
    assert perms.shape[1] == n
    out = NaiveResult(np.empty(P), np.empty(P, np.int64), np.empty(P),
                      np.empty(v, np.uint32), np.empty(v), np.empty(v, np.uint32), np.empty(v),
                      n, int(n1))
    rc = lib.oracle_naive(_ptr(Xt), n, v, int(n1), _ptr(perms), P, int(bool(two_sided)),
                          int(nthreads), float(tie_rel), _ptr(out.maxnull), _ptr(out.argmax),
                          _ptr(out.second), _ptr(out.counts), _ptr(out.t_obs), _ptr(out.near),
                          _ptr(out.tau))
    if rc != 0:
        raise ValueError("oracle_naive failed (rc=%d)" % rc)
    return out


def t_rows(X, n1, perms, nthreads=0, Xt=None):
    """Rows of T (P x v, FP64): t of every voxel under every relabelling."""
    lib = _load()
    if Xt is None:
        Xt = voxel_major(X)
    v, n = Xt.shape
    perms = np.ascontiguousarray(perms, dtype=np.int32).reshape(-1, n)
    T = np.empty((perms.shape[0], v))
    rc = lib.oracle_t_rows(_ptr(Xt), n, v, int(n1), _ptr(perms), perms.shape[0],
                           int(nthreads), _ptr(T))
    if rc != 0:
        raise ValueError("oracle_t_rows failed (rc=%d)" % rc)
    return T


def t_entries(Xt, n1, perms, rows, idx):
    """t at (rows[q], idx[q]) pairs; Xt is the voxel-major FP64 data."""
    lib = _load()
    v, n = Xt.shape
    perms = np.ascontiguousarray(perms, dtype=np.int32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(rows.shape[0])
    rc = lib.oracle_t_entries(_ptr(Xt), n, v, int(n1), _ptr(perms), _ptr(rows), _ptr(idx),
                              rows.shape[0], _ptr(out))
    if rc != 0:
        raise ValueError("oracle_t_entries failed (rc=%d)" % rc)
    return out


def fwer_pvalues(maxnull, t_obs, two_sided=False):
    """FWER-corrected p-value of every voxel from a max-null (Sec. 2: the
    fraction of the permutation distribution of the maximum at or above the
    voxel's observed statistic), counting the observed labelling as one of
    the P + 1 labellings: p_j = (1 + #{i : m_i >= T_j}) / (P + 1), with
    T_j = t_obs_j (|t_obs_j| two-sided). The comparison is made on float32
    values, as the library stores both. Voxels without a statistic get NaN.
    Brute force over all (voxel, relabelling) pairs."""
    m = np.asarray(maxnull, dtype=np.float32)
    t = np.asarray(t_obs, dtype=np.float64).astype(np.float32)
    T = np.abs(t) if two_sided else t
    P = m.shape[0]
    out = np.full(T.shape[0], np.nan)
    ok = ~np.isnan(T)
    ms = np.sort(m)
    # #{i : m_i >= T_j} = P - #{i : m_i < T_j}
    below = np.searchsorted(ms, T[ok], side="left")
    out[ok] = (1.0 + (P - below)) / (P + 1.0)
    return out


def resampling_risk(reject1, reject2):
    """Resampling risk of two methods' voxel-wise decisions (Sec. 5.5, Eq. (6)):
    with v1 and v2 the numbers of voxels whose null hypothesis method 1 and
    method 2 reject, and vc the number both reject,
        risk = ((v1 - vc) / v1 + (v2 - vc) / v2) / 2.
    The paper leaves v1 = 0 or v2 = 0 open; reading taken here: a method that
    rejects nothing contributes 0 for its own term (none of its rejections is
    missed by the other), so two empty sets give 0 and one empty set against
    a non-empty one gives 1/2. Returns (risk, v1, v2, vc)."""
    a = np.asarray(reject1, dtype=bool)
    b = np.asarray(reject2, dtype=bool)
    v1 = int(a.sum())
    v2 = int(b.sum())
    vc = int(np.logical_and(a, b).sum())
    t1 = (v1 - vc) / v1 if v1 else 0.0
    t2 = (v2 - vc) / v2 if v2 else 0.0
    return (t1 + t2) / 2.0, v1, v2, vc
