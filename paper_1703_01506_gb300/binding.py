"""Thin ctypes binding of ``libpt.so`` (declared in ``include/pt.h``).

Argument marshalling only: every step of the computation runs in the
library's CUDA kernels. Functions carry the C names; array arguments are
CUDA torch tensors (their device pointers are passed through), and a status
other than PT_OK raises :class:`PtError` with the library's message.

The library must have been built (``__graft_entry__.build()``); importing
this module does not build it, and :func:`load` raises if it is missing.
"""
import ctypes
import os

import torch

from .build import LIB

PT_OK, PT_ERR_INVALID, PT_ERR_NOMEM, PT_ERR_CUDA, PT_ERR_TIMEOUT, PT_ERR_UNSUPPORTED = range(6)
PT_PREC_FP32, PT_PREC_BF16X2, PT_PREC_BF16X3, PT_PREC_FP16X2 = 0, 1, 2, 3
_STATUS = {0: "PT_OK", 1: "PT_ERR_INVALID", 2: "PT_ERR_NOMEM", 3: "PT_ERR_CUDA",
           4: "PT_ERR_TIMEOUT", 5: "PT_ERR_UNSUPPORTED"}


class PtError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (_STATUS.get(status, status), msg))
        self.status = status


class pt_naive_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("two_sided", ctypes.c_int32),
                ("accumulate_counts", ctypes.c_int32)]


class pt_tc_config(ctypes.Structure):
    _fields_ = [("voxel_tile", ctypes.c_int32), ("stages", ctypes.c_int32),
                ("ksteps_per_stage", ctypes.c_int32), ("items_per_sm", ctypes.c_int32)]

    def as_tuple(self):
        return (self.voxel_tile, self.stages, self.ksteps_per_stage, self.items_per_sm)


class pt_rapid_opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("train_passes", ctypes.c_int32),
                ("qr_every", ctypes.c_int32), ("admm_iters", ctypes.c_int32),
                ("admm_rho", ctypes.c_float), ("step", ctypes.c_float),
                ("shift_mode", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("rec_step", ctypes.c_float)]


class pt_rapid_info(ctypes.Structure):
    _fields_ = [("sigma", ctypes.c_double), ("mu", ctypes.c_double),
                ("m_per_perm", ctypes.c_int64), ("train_steps", ctypes.c_int64)]


_lib = None
_VP = ctypes.c_void_p


def load(path=None):
    """Load the built library (raises OSError/RuntimeError when it is absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB
    if not os.path.exists(path):
        raise RuntimeError("libpt.so not built (%s); run __graft_entry__.build()" % path)
    lib = ctypes.CDLL(path)
    i32, i64 = ctypes.c_int32, ctypes.c_int64
    sig = {
        "pt_naive_opts_default": (None, [ctypes.POINTER(pt_naive_opts)]),
        "pt_prepare": (ctypes.c_int, [_VP, i32, i64, _VP, i32, _VP, ctypes.POINTER(_VP)]),
        "pt_prepare_glm": (ctypes.c_int, [_VP, i32, i64, _VP, i32, _VP, i32, _VP,
                                          ctypes.POINTER(_VP)]),
        "pt_maxnull_naive": (ctypes.c_int, [_VP, _VP, i64, _VP, _VP, _VP]),
        "pt_maxnull_naive_ex": (ctypes.c_int, [_VP, _VP, i64, ctypes.POINTER(pt_naive_opts),
                                               _VP, _VP, _VP]),
        "pt_maxnull_naive_batched": (ctypes.c_int, [_VP, i32, _VP, _VP,
                                                    ctypes.POINTER(pt_naive_opts), _VP, _VP,
                                                    _VP]),
        "pt_fwer_pvalues": (ctypes.c_int, [_VP, _VP, i64, i32, _VP]),
        "pt_sync": (ctypes.c_int, [_VP]),
        "pt_t_obs": (ctypes.c_int, [_VP, _VP]),
        "pt_t_rows": (ctypes.c_int, [_VP, _VP, i64, i32, _VP]),
        "pt_cluster_maxnull": (ctypes.c_int, [_VP, _VP, i64, ctypes.c_double, _VP, i32, i32,
                                              _VP]),
        "pt_cluster_observed": (ctypes.c_int, [_VP, ctypes.c_double, _VP, i32, _VP, _VP]),
        "pt_maxnull_anova": (ctypes.c_int, [_VP, _VP, i64, _VP, i32, i32, _VP, _VP, _VP]),
        "pt_voxel_grid_index": (ctypes.c_int, [_VP, _VP]),
        "pt_num_voxels": (i64, [_VP]),
        "pt_num_valid_voxels": (i64, [_VP]),
        "pt_last_error": (ctypes.c_char_p, [_VP]),
        "pt_destroy": (None, [_VP]),
        "pt_release_cached_memory": (None, []),
        "pt_profile_enable": (ctypes.c_int, [_VP, i32]),
        "pt_profile_read": (ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(i64)]),
        "pt_kernel_launch_count": (i64, []),
        "pt_maxnull_naive_noalloc": (ctypes.c_int, [_VP, i32, i64, i32, _VP, i64, i32, _VP, _VP,
                                                    _VP, _VP]),
        "pt_rapid_opts_default": (None, [ctypes.POINTER(pt_rapid_opts)]),
        "pt_maxnull_rapid": (ctypes.c_int, [_VP, _VP, i64, i32, ctypes.c_double, i32,
                                            ctypes.POINTER(pt_rapid_opts), _VP, _VP,
                                            ctypes.POINTER(pt_rapid_info)]),
        "pt_rapid_train": (ctypes.c_int, [_VP, _VP, i32, i32, ctypes.c_double,
                                          ctypes.POINTER(pt_rapid_opts), _VP, _VP, _VP, _VP,
                                          ctypes.POINTER(pt_rapid_info)]),
        "pt_rapid_recover": (ctypes.c_int, [_VP, _VP, i64, i64, _VP, i32, ctypes.c_double,
                                            ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(pt_rapid_opts), _VP, _VP]),
        "pt_autotune_naive": (ctypes.c_int, [_VP, _VP, i64, ctypes.POINTER(pt_naive_opts),
                                             ctypes.POINTER(pt_tc_config),
                                             ctypes.POINTER(ctypes.c_double)]),
        "pt_autotune_naive_batched": (ctypes.c_int, [_VP, i32, _VP, _VP,
                                                     ctypes.POINTER(pt_naive_opts)]),
        "pt_tune_lookup": (i32, [i32, i32, i32, i64, i64, ctypes.POINTER(pt_tc_config)]),
        "pt_tune_set": (ctypes.c_int, [i32, i32, i32, i64, i64, ctypes.POINTER(pt_tc_config)]),
        "pt_tune_save": (ctypes.c_int, [ctypes.c_char_p]),
        "pt_tune_load": (ctypes.c_int, [ctypes.c_char_p]),
        "pt_tune_clear": (None, []),
        "pt_debug_fail_allocations": (None, [i64]),
        "pt_debug_device_reset": (ctypes.c_int, []),
        "pt_selftest_bounded_wait": (ctypes.c_int, [_VP, i32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t, host_ok=False):
    """Device pointer of a CUDA tensor; with host_ok, also of a page-locked
    (pinned) CPU tensor, which the device addresses directly."""
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a tensor")
    if not (t.is_cuda or (host_ok and t.is_pinned())):
        raise TypeError("expected a CUDA tensor" + (" or a pinned CPU tensor" if host_ok else ""))
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _check(status, ctx_handle=None):
    if status != PT_OK:
        msg = load().pt_last_error(ctx_handle)
        raise PtError(status, msg.decode() if msg else "")


class Ctx:
    """Owns a ``pt_ctx*``; destroyed with :meth:`close` or on garbage collection."""

    def __init__(self, handle):
        self.handle = handle

    def close(self):
        if self.handle:
            load().pt_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _stream_ptr(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def pt_prepare(X, n1, mask=None, stream=None):
    """X: (n, n_grid) float32 CUDA tensor, or pinned CPU tensor read by the
    kernels over the host link; mask: (n_grid,) uint8 (same choice) or None."""
    lib = load()
    assert X.dtype == torch.float32 and X.dim() == 2
    if mask is not None:
        assert mask.dtype == torch.uint8 and mask.numel() == X.shape[1]
    out = ctypes.c_void_p()
    st = lib.pt_prepare(_ptr(X, True), X.shape[0], X.shape[1], _ptr(mask, True), int(n1),
                        _stream_ptr(stream), ctypes.byref(out))
    _check(st, None)
    return Ctx(out)


def pt_prepare_glm(X, n1, Z=None, mask=None, stream=None):
    """pt_prepare with nuisance covariates: Z is an (n, q) array (host, float64)
    or None; the statistic is the least-squares t of the group column."""
    import numpy as np
    lib = load()
    assert X.dtype == torch.float32 and X.dim() == 2
    n = X.shape[0]
    if mask is not None:
        assert mask.dtype == torch.uint8 and mask.numel() == X.shape[1]
    if Z is None:
        Zc, q, zp = None, 0, None
    else:
        Zc = np.ascontiguousarray(np.asarray(Z, dtype=np.float64).reshape(n, -1))
        q = Zc.shape[1]
        zp = ctypes.c_void_p(Zc.ctypes.data) if q > 0 else None
    out = ctypes.c_void_p()
    st = lib.pt_prepare_glm(_ptr(X, True), n, X.shape[1], _ptr(mask, True), int(n1), zp, int(q),
                            _stream_ptr(stream), ctypes.byref(out))
    _check(st, None)
    return Ctx(out)


def pt_maxnull_naive(ctx, perms, maxnull, argmax, counts=None):
    lib = load()
    assert perms.dtype == torch.int32
    st = lib.pt_maxnull_naive(ctx.handle, _ptr(perms), perms.shape[0], _ptr(maxnull),
                              _ptr(argmax), _ptr(counts))
    _check(st, ctx.handle)


def pt_maxnull_naive_ex(ctx, perms, opts, maxnull, argmax, counts=None):
    lib = load()
    assert perms.dtype == torch.int32
    st = lib.pt_maxnull_naive_ex(ctx.handle, _ptr(perms), perms.shape[0], ctypes.byref(opts),
                                 _ptr(maxnull), _ptr(argmax), _ptr(counts))
    _check(st, ctx.handle)


def pt_maxnull_naive_batched(ctxs, perms, opts, maxnull, argmax, counts=None):
    """Lists of equal length: contexts, int32 perms (P_i x n_i), float32[P_i]
    maxnull, int32[P_i] argmax and uint32[v_i] counts (or None)."""
    lib = load()
    m = len(ctxs)
    if not (len(perms) == len(maxnull) == len(argmax) == m) or (counts is not None and
                                                                 len(counts) != m):
        raise ValueError("per-study lists must have one entry per context")
    for p in perms:
        assert p.dtype == torch.int32
    h = (_VP * m)(*[c.handle for c in ctxs])
    pp = (_VP * m)(*[_ptr(p) for p in perms])
    P = (ctypes.c_int64 * m)(*[p.shape[0] for p in perms])
    mx = (_VP * m)(*[_ptr(t) for t in maxnull])
    am = (_VP * m)(*[_ptr(t) for t in argmax])
    cn = None if counts is None else (_VP * m)(*[_ptr(t) for t in counts])
    st = lib.pt_maxnull_naive_batched(h, m, pp, P, ctypes.byref(opts), mx, am, cn)
    _check(st, None)


def pt_autotune_naive(ctx, perms, opts):
    """Times the fused kernel's launch configurations on this problem and
    records the fastest; returns (pt_tc_config, ms)."""
    lib = load()
    assert perms.dtype == torch.int32
    cfg = pt_tc_config()
    ms = ctypes.c_double()
    st = lib.pt_autotune_naive(ctx.handle, _ptr(perms), perms.shape[0], ctypes.byref(opts),
                               ctypes.byref(cfg), ctypes.byref(ms))
    _check(st, ctx.handle)
    return cfg, ms.value


def pt_autotune_naive_batched(ctxs, perms, opts):
    lib = load()
    m = len(ctxs)
    if len(perms) != m:
        raise ValueError("one relabelling tensor per context")
    h = (_VP * m)(*[c.handle for c in ctxs])
    pp = (_VP * m)(*[_ptr(p) for p in perms])
    P = (ctypes.c_int64 * m)(*[p.shape[0] for p in perms])
    _check(lib.pt_autotune_naive_batched(h, m, pp, P, ctypes.byref(opts)), None)


def pt_tune_lookup(n, precision, two_sided, v, P):
    """Returns (found, pt_tc_config); found is 1 (tuned entry), 0 (default) or -1 (bad)."""
    cfg = pt_tc_config()
    r = load().pt_tune_lookup(int(n), int(precision), int(two_sided), int(v), int(P),
                              ctypes.byref(cfg))
    return int(r), cfg


def pt_tune_set(n, precision, two_sided, v, P, voxel_tile, stages, ksteps_per_stage=1,
                items_per_sm=2):
    cfg = pt_tc_config(int(voxel_tile), int(stages), int(ksteps_per_stage), int(items_per_sm))
    _check(load().pt_tune_set(int(n), int(precision), int(two_sided), int(v), int(P),
                              ctypes.byref(cfg)), None)


def pt_tune_save(path):
    _check(load().pt_tune_save(os.fsencode(path)), None)


def pt_tune_load(path):
    _check(load().pt_tune_load(os.fsencode(path)), None)


def pt_tune_clear():
    load().pt_tune_clear()


def pt_debug_fail_allocations(after):
    """After ``after`` more device allocations every later one fails (< 0: off)."""
    load().pt_debug_fail_allocations(int(after))


def pt_selftest_bounded_wait(ctx, limit_ms):
    _check(load().pt_selftest_bounded_wait(ctx.handle, int(limit_ms)), ctx.handle)


def pt_sync(ctx):
    _check(load().pt_sync(ctx.handle), ctx.handle)


def pt_fwer_pvalues(ctx, maxnull, p_out, two_sided=False):
    _check(load().pt_fwer_pvalues(ctx.handle, _ptr(maxnull), maxnull.shape[0], int(bool(two_sided)),
                                  _ptr(p_out)), ctx.handle)


def pt_t_obs(ctx, t_obs):
    _check(load().pt_t_obs(ctx.handle, _ptr(t_obs)), ctx.handle)


def pt_voxel_grid_index(ctx, grid_index):
    _check(load().pt_voxel_grid_index(ctx.handle, _ptr(grid_index)), ctx.handle)


def pt_num_voxels(ctx):
    return int(load().pt_num_voxels(ctx.handle))


def pt_num_valid_voxels(ctx):
    return int(load().pt_num_valid_voxels(ctx.handle))


def pt_last_error(ctx=None):
    msg = load().pt_last_error(ctx.handle if ctx is not None else None)
    return msg.decode() if msg else ""


def pt_destroy(ctx):
    ctx.close()


def pt_release_cached_memory():
    load().pt_release_cached_memory()


def naive_opts(precision=PT_PREC_BF16X3, two_sided=False, accumulate_counts=False):
    o = pt_naive_opts()
    load().pt_naive_opts_default(ctypes.byref(o))
    o.precision = int(precision)
    o.two_sided = int(bool(two_sided))
    o.accumulate_counts = int(bool(accumulate_counts))
    return o


def maxnull_naive(ctx, perms, precision=PT_PREC_BF16X3, two_sided=False, counts=True, sync=True):
    """Allocates outputs, runs pt_maxnull_naive_ex, optionally pt_sync; returns
    (maxnull float32[P], argmax int32[P], counts int32[v] or None) as tensors."""
    dev = perms.device
    P = perms.shape[0]
    mx = torch.empty(P, dtype=torch.float32, device=dev)
    am = torch.empty(P, dtype=torch.int32, device=dev)
    # uint32 counts held in an int32 tensor (counts < 2^31)
    ct = torch.empty(pt_num_voxels(ctx), dtype=torch.int32, device=dev) if counts else None
    pt_maxnull_naive_ex(ctx, perms, naive_opts(precision, two_sided), mx, am, ct)
    if sync:
        pt_sync(ctx)
    return mx, am, ct


def pt_t_rows(ctx, perms, precision=PT_PREC_BF16X3, out=None):
    """Rows of T: (P, v) float32 CUDA tensor, NaN where a voxel has no t."""
    P = perms.shape[0]
    v = int(load().pt_num_voxels(ctx.handle))
    if perms.dim() != 2 or perms.dtype != torch.int32:
        raise ValueError("perms must be a 2-D int32 tensor")
    if out is None:
        out = torch.empty((P, v), dtype=torch.float32, device=perms.device)
    elif out.dtype != torch.float32 or out.numel() < P * v:
        raise ValueError("out must be float32 with at least P * v elements")
    _check(load().pt_t_rows(ctx.handle, _ptr(perms), P, int(precision), _ptr(out)), ctx.handle)
    return out


def pt_maxnull_anova(ctx, perms, group_sizes, precision=PT_PREC_FP16X2, counts=True):
    """One-way F max-null over g groups: (maxnull float32[P], argmax int32[P],
    counts int32[v] or None) CUDA tensors."""
    if perms.dim() != 2 or perms.dtype != torch.int32:
        raise ValueError("perms must be a 2-D int32 tensor")
    P = perms.shape[0]
    g = len(group_sizes)
    sz = (ctypes.c_int32 * g)(*[int(x) for x in group_sizes])
    mx = torch.empty(P, dtype=torch.float32, device=perms.device)
    am = torch.empty(P, dtype=torch.int32, device=perms.device)
    ct = None
    if counts:
        ct = torch.empty(int(load().pt_num_voxels(ctx.handle)), dtype=torch.int32,
                         device=perms.device)
    _check(load().pt_maxnull_anova(ctx.handle, _ptr(perms), P, sz, g, int(precision), _ptr(mx),
                                   _ptr(am), _ptr(ct)), ctx.handle)
    return mx, am, ct


def _dims(dims):
    if len(dims) != 3:
        raise ValueError("dims must be (d0, d1, d2)")
    return (ctypes.c_int32 * 3)(*[int(d) for d in dims])


def pt_cluster_maxnull(ctx, perms, tau, dims, connectivity=6, precision=PT_PREC_FP16X2,
                       out=None):
    """Largest cluster of {t >= tau} per relabelling: (P,) int32 CUDA tensor."""
    if perms.dim() != 2 or perms.dtype != torch.int32:
        raise ValueError("perms must be a 2-D int32 tensor")
    P = perms.shape[0]
    if out is None:
        out = torch.empty(P, dtype=torch.int32, device=perms.device)
    elif out.dtype != torch.int32 or out.numel() < P:
        raise ValueError("out must be int32 with at least P elements")
    _check(load().pt_cluster_maxnull(ctx.handle, _ptr(perms), P, float(tau), _dims(dims),
                                     int(connectivity), int(precision), _ptr(out)), ctx.handle)
    return out


def pt_cluster_observed(ctx, tau, dims, connectivity=6, device="cuda"):
    """Observed map's clusters of {t >= tau}: (label, size), (v,) int32 tensors."""
    v = int(load().pt_num_voxels(ctx.handle))
    label = torch.empty(v, dtype=torch.int32, device=device)
    size = torch.empty(v, dtype=torch.int32, device=device)
    _check(load().pt_cluster_observed(ctx.handle, float(tau), _dims(dims), int(connectivity),
                                      _ptr(label), _ptr(size)), ctx.handle)
    return label, size


def pt_profile_enable(ctx, on=True):
    _check(load().pt_profile_enable(ctx.handle, int(bool(on))), ctx.handle)


def pt_profile_read(ctx):
    """Returns (total_ms, launches) of the dominant kernel since the last read."""
    ms = ctypes.c_double()
    n = ctypes.c_int64()
    _check(load().pt_profile_read(ctx.handle, ctypes.byref(ms), ctypes.byref(n)), ctx.handle)
    return ms.value, n.value


def pt_kernel_launch_count():
    return int(load().pt_kernel_launch_count())


def pt_maxnull_naive_noalloc(X, n1, perms, maxnull, argmax, counts=None, two_sided=False,
                             stream=None):
    """NaivePT without any device allocation (see include/pt.h). X: (n, v)
    float32 CUDA tensor, every column a voxel; perms (P, n) int32; maxnull
    (>= P) float32, argmax (>= P) int32, counts (>= v) int32/uint32 or None.
    Shapes are checked here, before the library is called: the kernels read
    perms row by row and write P maxima and v counts. Synchronous."""
    if X.dtype != torch.float32 or X.dim() != 2:
        raise ValueError("X must be a 2-D float32 tensor (n x v)")
    n, v = X.shape
    if perms.dtype != torch.int32 or perms.dim() != 2 or perms.shape[1] != n:
        raise ValueError("perms must be a 2-D int32 tensor with X.shape[0] = %d columns" % n)
    P = perms.shape[0]
    if maxnull.dtype != torch.float32 or maxnull.numel() < P:
        raise ValueError("maxnull must be float32 with at least P = %d elements" % P)
    if argmax.dtype != torch.int32 or argmax.numel() < P:
        raise ValueError("argmax must be int32 with at least P = %d elements" % P)
    if counts is not None and (counts.dtype not in (torch.int32, torch.uint32)
                               or counts.numel() < v):
        raise ValueError("counts must be int32/uint32 with at least v = %d elements" % v)
    lib = load()
    st = lib.pt_maxnull_naive_noalloc(_ptr(X), n, v, int(n1), _ptr(perms), P,
                                      int(bool(two_sided)), _ptr(maxnull), _ptr(argmax),
                                      _ptr(counts), _stream_ptr(stream))
    _check(st, None)


def pt_debug_device_reset():
    """cudaDeviceReset on the current device through the library's runtime (tests only)."""
    _check(load().pt_debug_device_reset(), None)


def rapid_opts(**kw):
    """pt_rapid_opts with the library defaults, overridden by keyword."""
    o = pt_rapid_opts()
    load().pt_rapid_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def pt_maxnull_rapid(ctx, perms, rank, sample_rate, n_train, opts, maxnull, counts=None):
    """Returns a pt_rapid_info (sigma, mu, m_per_perm, train_steps)."""
    info = pt_rapid_info()
    st = load().pt_maxnull_rapid(ctx.handle, _ptr(perms), perms.shape[0], int(rank),
                                 float(sample_rate), int(n_train), ctypes.byref(opts),
                                 _ptr(maxnull), _ptr(counts), ctypes.byref(info))
    _check(st, ctx.handle)
    return info


def pt_rapid_train(ctx, perms, n_train, rank, sample_rate, opts, U_out=None, train_max=None,
                   counts=None, w_hist=None):
    info = pt_rapid_info()
    st = load().pt_rapid_train(ctx.handle, _ptr(perms), int(n_train), int(rank),
                               float(sample_rate), ctypes.byref(opts), _ptr(U_out),
                               _ptr(train_max), _ptr(counts), _ptr(w_hist), ctypes.byref(info))
    _check(st, ctx.handle)
    return info


def pt_rapid_recover(ctx, perms, first_row, U, rank, sample_rate, sigma, mu, opts, maxnull,
                     W_out=None):
    st = load().pt_rapid_recover(ctx.handle, _ptr(perms), perms.shape[0], int(first_row), _ptr(U),
                                 int(rank), float(sample_rate), float(sigma), float(mu),
                                 ctypes.byref(opts), _ptr(maxnull), _ptr(W_out))
    _check(st, ctx.handle)
