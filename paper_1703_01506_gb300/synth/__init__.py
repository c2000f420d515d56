"""Seeded synthetic inputs shared by the CUDA path, the oracle, tests and bench.

Input generation only: nothing here computes any step of the permutation
test. Everything is a deterministic function of its seed.

* Relabelling lists: PCG32 + Fisher-Yates (``pcg32_perms.c``), one stream.
* Voxel data, stand-ins for the paper's workloads (the ADNI gray-matter maps
  of Sec. 5.3 are not available; synthetic fields take their shapes):
    - ``gaussian_mean_shift``: X[i,j] = mu_j + N(0,1), mu_j ~ U(0,1).
    - ``two_group_gaussian``: Simulation Data I/II of Sec. 5.1-5.2 (N(0,1)
      everywhere, N(effect,1) for a fraction of voxels in one group).
    - ``brain_field``: per-subject white noise on a 3D grid, separable
      Gaussian smoothing (FWHM in voxels), exact per-voxel unit-variance
      rescaling, optional z-shift inside a sphere for group 1, then the
      normal CDF maps it to gray-matter-like values in [0, 1]; an ellipsoid
      mask gives the brain.
"""

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "pcg32_perms.c")
_LIB = os.path.join(_BUILD, "libpcg32_perms.so")
_lock = threading.Lock()
_lib = None


def build(force=False):
    """Compile the PCG32 helper (plain C, host only)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.pcg32_raw.restype = None
            lib.pcg32_raw.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int64,
                                      ctypes.c_void_p]
            lib.pcg32_fisher_yates.restype = None
            lib.pcg32_fisher_yates.argtypes = [ctypes.c_uint64, ctypes.c_uint64,
                                               ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p]
            _lib = lib
    return _lib


def pcg32_raw(seed, seq, count):
    out = np.empty(count, np.uint32)
    _load().pcg32_raw(seed, seq, count, ctypes.c_void_p(out.ctypes.data))
    return out


def perms_pcg32(n, P, seed=1, seq=1):
    """(P, n) int32: P Fisher-Yates relabellings from PCG32(seed, seq)."""
    out = np.empty((P, n), np.int32)
    _load().pcg32_fisher_yates(seed, seq, n, P, ctypes.c_void_p(out.ctypes.data))
    return out


def identity_perm(n):
    return np.arange(n, dtype=np.int32)[None, :]


# ----------------------------------------------------------------------------
# Simple Gaussian workloads
# ----------------------------------------------------------------------------

def gaussian_mean_shift(n, v, seed=1):
    """X[i,j] = mu_j + N(0,1), mu_j ~ U(0,1); (n, v) float32, no signal."""
    g = np.random.Generator(np.random.Philox(seed))
    mu = g.uniform(0.0, 1.0, size=v)
    X = mu[None, :] + g.standard_normal((n, v))
    return X.astype(np.float32)


def two_group_gaussian(n1, n2, v, frac=0.01, effect=1.0, seed=1):
    """Simulation data of Sec. 5.1-5.2: N(0,1) noise, ``frac`` of the voxels
    drawn from N(effect,1) in group 1 (the first n1 subjects)."""
    g = np.random.Generator(np.random.Philox(seed))
    X = g.standard_normal((n1 + n2, v))
    k = int(round(frac * v))
    if k > 0:
        cols = g.choice(v, size=k, replace=False)
        X[:n1, cols] += effect
    return X.astype(np.float32)


# ----------------------------------------------------------------------------
# Smoothed brain-shaped fields
# ----------------------------------------------------------------------------

def ellipsoid_mask(grid, center, semi_axes, v_limit=None):
    """Boolean (prod(grid),) C-order mask of the ellipsoid; optionally keep only
    the first ``v_limit`` voxels in raster order."""
    axes = [np.arange(s, dtype=np.float64) for s in grid]
    xx, yy, zz = np.meshgrid(*axes, indexing="ij")
    r2 = (((xx - center[0]) / semi_axes[0]) ** 2 + ((yy - center[1]) / semi_axes[1]) ** 2
          + ((zz - center[2]) / semi_axes[2]) ** 2)
    m = (r2 <= 1.0).reshape(-1)
    if v_limit is not None:
        idx = np.flatnonzero(m)
        if idx.size < v_limit:
            raise ValueError("mask has %d voxels < %d" % (idx.size, v_limit))
        m = np.zeros_like(m)
        m[idx[:v_limit]] = True
    return m


def sphere_mask(grid, center, radius):
    axes = [np.arange(s, dtype=np.float64) for s in grid]
    xx, yy, zz = np.meshgrid(*axes, indexing="ij")
    r2 = (xx - center[0]) ** 2 + (yy - center[1]) ** 2 + (zz - center[2]) ** 2
    return (r2 <= radius * radius).reshape(-1)


def gaussian_taps(fwhm):
    """Normalised 1D Gaussian taps for a FWHM in voxels, truncated at 4 sigma."""
    sigma = fwhm / (2.0 * math.sqrt(2.0 * math.log(2.0)))
    rad = int(math.ceil(4.0 * sigma))
    k = np.arange(-rad, rad + 1, dtype=np.float64)
    w = np.exp(-0.5 * (k / sigma) ** 2)
    return w / w.sum()


def _axis_variance(length, w):
    """Variance of the zero-padded smoothed unit white noise at each position."""
    rad = len(w) // 2
    var = np.zeros(length)
    w2 = w * w
    for p in range(length):
        lo, hi = max(0, p - rad), min(length - 1, p + rad)
        var[p] = w2[lo - p + rad: hi - p + rad + 1].sum()
    return var


def brain_field(n, n1, grid=(91, 109, 91), center=(45, 54, 45), semi_axes=(34, 44, 37),
                fwhm=8.0, effect=0.0, effect_center=None, effect_radius=10.0, seed=1,
                device="cpu", v_limit=None, chunk=16):
    """Smoothed brain-shaped gray-matter-like field (torch tensors).

    Returns ``(X, mask)``: X is (n, prod(grid)) float32 on ``device``, mask is
    (prod(grid),) uint8 on ``device``. Group 1 (the first n1 subjects) gets
    ``effect`` added in the z domain inside a sphere before the normal CDF.
    """
    import torch
    import torch.nn.functional as F

    dev = torch.device(device)
    G = tuple(int(s) for s in grid)
    V = G[0] * G[1] * G[2]
    w = gaussian_taps(fwhm)
    wt = torch.tensor(w, dtype=torch.float32, device=dev).view(1, 1, -1)
    inv_sd = 1.0 / np.sqrt(np.einsum("i,j,k->ijk", _axis_variance(G[0], w),
                                     _axis_variance(G[1], w), _axis_variance(G[2], w)))
    inv_sd = torch.tensor(inv_sd.astype(np.float32), device=dev)
    sph = None
    if effect != 0.0:
        c = effect_center if effect_center is not None else center
        sph = torch.tensor(sphere_mask(G, c, effect_radius).reshape(G), device=dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(int(seed))
    X = torch.empty((n, V), dtype=torch.float32, device=dev)
    pad = wt.shape[-1] // 2
    for s0 in range(0, n, chunk):
        s1 = min(n, s0 + chunk)
        z = torch.randn((s1 - s0,) + G, generator=gen, device=dev, dtype=torch.float32)
        for ax in (1, 2, 3):
            zt = z.movedim(ax, -1)
            shp = zt.shape
            y = F.conv1d(zt.reshape(-1, 1, shp[-1]), wt, padding=pad)
            z = y.reshape(shp).movedim(-1, ax)
        z = z * inv_sd
        if sph is not None and s0 < n1:
            g1 = min(s1, n1) - s0
            z[:g1] = torch.where(sph, z[:g1] + effect, z[:g1])
        X[s0:s1] = torch.special.ndtr(z).reshape(s1 - s0, V)
    mask = ellipsoid_mask(G, center, semi_axes, v_limit=v_limit)
    return X, torch.tensor(mask.astype(np.uint8), device=dev)


# ----------------------------------------------------------------------------
# Named workloads (the shapes of the paper's experiments, Sec. 5)
# ----------------------------------------------------------------------------

BIG_GRID = (121, 145, 121)
BIG_CENTER = (60, 72, 60)


def workload(name, device="cpu", seed=1):
    """Return a dict describing a named synthetic workload.

    Keys: X (n, V_grid) float32 array/tensor, mask (or None), n, n1, P,
    perms (P, n) int32 numpy, plus RapidPT settings where relevant.
    """
    if name == "gauss_n20_v2000":
        n, n1, v, P = 20, 10, 2000, 1000
        X = gaussian_mean_shift(n, v, seed=seed)
        return dict(name=name, X=X, mask=None, n=n, n1=n1, P=P,
                    perms=perms_pcg32(n, P, seed=1))
    if name == "brain_n100_v232k":
        n, n1, P = 100, 50, 10000
        X, mask = brain_field(n, n1, effect=0.3, seed=seed, device=device)
        return dict(name=name, X=X, mask=mask, n=n, n1=n1, P=P,
                    perms=perms_pcg32(n, P, seed=1))
    if name == "brain_n200_v500k":
        n, n1, P = 200, 100, 100000
        sa = tuple(a * 4.0 / 3.0 for a in (34, 44, 37))
        X, mask = brain_field(n, n1, grid=BIG_GRID, center=BIG_CENTER, semi_axes=sa,
                              seed=seed, device=device, v_limit=500000)
        return dict(name=name, X=X, mask=mask, n=n, n1=n1, P=P, rank=50, n_train=400,
                    sample_rate=0.0035, perms=perms_pcg32(n, P, seed=1))
    if name == "brain_n400_v600k":
        n, n1, P = 400, 200, 100000
        sa = tuple(a * 1.4 for a in (34, 44, 37))
        X, mask = brain_field(n, n1, grid=BIG_GRID, center=BIG_CENTER, semi_axes=sa,
                              effect=0.2, effect_radius=8.0, seed=seed, device=device,
                              v_limit=600000)
        return dict(name=name, X=X, mask=mask, n=n, n1=n1, P=P, rank=100, n_train=800,
                    sample_rate=0.0035, perms=perms_pcg32(n, P, seed=1))
    raise KeyError(name)


def uneven_study_shapes(count=64, vmin=50000, vmax=600000, nmin=24, nmax=400):
    """(n, n1, v) for ``count`` studies: n ~ U{nmin..nmax}, v ~ U{vmin..vmax}
    from PCG32 seeded 1000+k, n1 = floor(n/2)."""
    out = []
    for k in range(count):
        r = pcg32_raw(1000 + k, 1, 2)
        n = nmin + int(r[0]) % (nmax - nmin + 1)
        v = vmin + int(r[1]) % (vmax - vmin + 1)
        out.append((n, n // 2, v))
    return out
