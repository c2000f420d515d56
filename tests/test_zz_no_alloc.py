"""The allocation-free NaivePT entry point against the regular one and the oracle.

pt_maxnull_naive_noalloc serves callers that cannot call cudaMalloc (code
inside another runtime's memory pool, or under a fixed memory budget after
start-up); its buffers live in one static device array. It must give what
pt_prepare + pt_maxnull_naive (FP32 path) give, within the tolerances of the
other GPU tests, on consecutive calls that reuse the array; it must agree
with the FP64 oracle directly; and it must keep working in a fresh primary
context after cudaDeviceReset, where the array has a new device address.
This file is collected last on purpose.
"""
import json
import os
import subprocess
import sys
import tempfile

import numpy as np
import pytest
import torch

import oracle
from paper_1703_01506_gb300 import synth

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TIE = lambda n: 2.0 * (n + 4) * 2.0 ** -24  # FP32 path's u band per unit l1 norm


def _regular(B, Xd, n1, pd, two_sided):
    ctx = B.pt_prepare(Xd, n1)
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=B.PT_PREC_FP32, two_sided=two_sided)
    ctx.close()
    return mx, am, ct


def _noalloc(B, Xd, n1, pd, two_sided):
    P, v = pd.shape[0], Xd.shape[1]
    mx = torch.full((P,), float("nan"), dtype=torch.float32, device="cuda")
    am = torch.full((P,), -7, dtype=torch.int32, device="cuda")
    ct = torch.full((v,), -7, dtype=torch.int32, device="cuda")
    B.pt_maxnull_naive_noalloc(Xd, n1, pd, mx, am, ct, two_sided=two_sided)
    return mx, am, ct


def _near(ref):
    return (ref.u_of(ref.maxnull) - ref.u_of(ref.second)) <= 2 * np.max(ref.tau)


def _compare(ref_or, a, b):
    """a = regular entry point, b = allocation-free one."""
    mxa, ama, cta = (t.cpu().numpy().astype(np.float64) for t in a)
    mxb, amb, ctb = (t.cpu().numpy().astype(np.float64) for t in b)
    same = ama == amb
    assert np.all(same | _near(ref_or))
    err = np.abs(mxa - mxb) / np.maximum(np.abs(mxa), 1.0)
    assert np.all(err[same] <= 1e-5)
    assert np.all(np.abs(cta - ctb) <= ref_or.near.astype(np.float64))


def _against_oracle(ref, mx, am, ct, invalid=()):
    """Maxima within FP32 output rounding of the oracle where the argmax agrees
    (the winner's t is recomputed in FP64), argmax equal outside near-ties,
    counts equal outside the oracle's near-tie entries, 0 at voxels without t."""
    mx, am, ct = (np.asarray(x, dtype=np.float64) for x in (mx, am, ct))
    same = am == ref.argmax
    assert np.all(same | _near(ref))
    err = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    assert np.all(err[same] <= 2.5e-7), float(err[same].max())
    assert np.all(err <= 1e-5)
    assert np.all(np.abs(ct - ref.counts) <= ref.near.astype(np.float64))
    for j in invalid:
        assert ct[j] == 0


@pytest.mark.parametrize("two_sided", [False, True])
def test_noalloc_matches_regular_on_two_calls(cuda_lib, two_sided):
    B = cuda_lib
    cases = [(40, 17, 3001, 700, 21), (20, 10, 2000, 1000, 1)]  # second call reuses the array
    for n, n1, v, P, seed in cases:
        X = synth.gaussian_mean_shift(n, v, seed=seed)
        X[:, 5] = 0.25  # a voxel without a t statistic
        perms = synth.perms_pcg32(n, P, seed=seed)
        Xd = torch.as_tensor(X).cuda()
        pd = torch.as_tensor(perms).cuda()
        ref = oracle.naive(X, n1, perms, two_sided=two_sided, tie_rel=TIE(n))
        a = _regular(B, Xd, n1, pd, two_sided)
        b = _noalloc(B, Xd, n1, pd, two_sided)
        _compare(ref, a, b)
        assert int(b[2][5].item()) == 0
        _against_oracle(ref, *(t.cpu().numpy() for t in b), invalid=[5])


def test_noalloc_many_invalid_columns_against_oracle(cuda_lib):
    """Every third column constant: the compaction of valid voxels decides
    which column each argmax names and where each count lands."""
    B = cuda_lib
    n, n1, v, P = 36, 18, 2999, 640
    X = synth.gaussian_mean_shift(n, v, seed=7)
    invalid = np.arange(0, v, 3)
    X[:, invalid] = np.float32(0.5)
    perms = synth.perms_pcg32(n, P, seed=7)
    ref = oracle.naive(X, n1, perms, tie_rel=TIE(n))
    assert not np.isin(ref.argmax, invalid).any()
    Xd = torch.as_tensor(X).cuda()
    pd = torch.as_tensor(perms).cuda()
    for _ in range(2):
        mx, am, ct = _noalloc(B, Xd, n1, pd, False)
        _against_oracle(ref, mx.cpu().numpy(), am.cpu().numpy(), ct.cpu().numpy(), invalid)


def test_noalloc_rejects_oversize_and_bad_rows(cuda_lib):
    B = cuda_lib
    n, n1 = 100, 50
    X = torch.zeros((n, 400_000), dtype=torch.float32, device="cuda")  # needs > 64 MiB
    perms = torch.as_tensor(synth.perms_pcg32(n, 10, seed=1)).cuda()
    mx = torch.empty(10, dtype=torch.float32, device="cuda")
    am = torch.empty(10, dtype=torch.int32, device="cuda")
    with pytest.raises(B.PtError) as e:
        B.pt_maxnull_naive_noalloc(X, n1, perms, mx, am)
    assert e.value.status == B.PT_ERR_INVALID and "static limit" in str(e.value)
    Xs = torch.as_tensor(synth.gaussian_mean_shift(n, 500, seed=3)).cuda()
    bad = perms.clone()
    bad[2, 0] = bad[2, 1]
    with pytest.raises(B.PtError):
        B.pt_maxnull_naive_noalloc(Xs, n1, bad, mx, am)
    B.pt_maxnull_naive_noalloc(Xs, n1, perms, mx, am)  # still usable


# Runs in a fresh process that never initialises CUDA through torch: device
# memory comes from the driver API in the primary context, the entry point is
# called, the library's runtime resets the device (cudaDeviceReset), and the
# same problem runs again in the new primary context, where the static array
# has a new device address.
_CHILD = r'''
import ctypes, json, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1703_01506_gb300 import binding
d = np.load(sys.argv[2])
X, perms, n1 = d["X"], d["perms"], int(d["n1"])
n, v = X.shape
P = perms.shape[0]
cu = ctypes.CDLL("libcuda.so.1")
def ck(r, what):
    if r != 0:
        raise SystemExit("%s returned %d" % (what, r))
ck(cu.cuInit(0), "cuInit")
dev = ctypes.c_int()
ck(cu.cuDeviceGet(ctypes.byref(dev), 0), "cuDeviceGet")
lib = binding.load()
V = ctypes.c_void_p
def run():
    ctx = V()
    ck(cu.cuDevicePrimaryCtxRetain(ctypes.byref(ctx), dev), "cuDevicePrimaryCtxRetain")
    ck(cu.cuCtxSetCurrent(ctx), "cuCtxSetCurrent")
    bufs = {}
    for name, nbytes in (("X", X.nbytes), ("perms", perms.nbytes), ("mx", 4 * P),
                         ("am", 4 * P), ("ct", 4 * v)):
        p = ctypes.c_uint64()
        ck(cu.cuMemAlloc_v2(ctypes.byref(p), ctypes.c_size_t(nbytes)), "cuMemAlloc")
        bufs[name] = p.value
    for name, arr in (("X", X), ("perms", perms)):
        ck(cu.cuMemcpyHtoD_v2(ctypes.c_uint64(bufs[name]), arr.ctypes.data_as(V),
                              ctypes.c_size_t(arr.nbytes)), "cuMemcpyHtoD")
    st = lib.pt_maxnull_naive_noalloc(V(bufs["X"]), n, v, n1, V(bufs["perms"]), P, 0,
                                      V(bufs["mx"]), V(bufs["am"]), V(bufs["ct"]), None)
    if st != 0:
        raise SystemExit("pt_maxnull_naive_noalloc: %d %s" % (st, lib.pt_last_error(None)))
    out = (np.empty(P, np.float32), np.empty(P, np.int32), np.empty(v, np.uint32))
    for name, arr in zip(("mx", "am", "ct"), out):
        ck(cu.cuMemcpyDtoH_v2(arr.ctypes.data_as(V), ctypes.c_uint64(bufs[name]),
                              ctypes.c_size_t(arr.nbytes)), "cuMemcpyDtoH")
    for p in bufs.values():
        ck(cu.cuMemFree_v2(ctypes.c_uint64(p)), "cuMemFree")
    return out
a = run()
st = lib.pt_debug_device_reset()
if st != 0:
    raise SystemExit("pt_debug_device_reset: %d" % st)
b = run()
np.savez(sys.argv[3], mx_a=a[0], am_a=a[1], ct_a=a[2], mx_b=b[0], am_b=b[1], ct_b=b[2])
print(json.dumps({"ok": True}))
'''


def test_noalloc_after_device_reset(cuda_lib):
    n, n1, v, P = 30, 15, 1500, 400
    X = synth.gaussian_mean_shift(n, v, seed=11)
    X[:, 9] = np.float32(0.125)
    perms = synth.perms_pcg32(n, P, seed=11)
    ref = oracle.naive(X, n1, perms, tie_rel=TIE(n))
    with tempfile.TemporaryDirectory() as td:
        inp, out = os.path.join(td, "in.npz"), os.path.join(td, "out.npz")
        np.savez(inp, X=X, perms=perms, n1=n1)
        p = subprocess.run([sys.executable, "-c", _CHILD, ROOT, inp, out], capture_output=True,
                           text=True, timeout=300)
        assert p.returncode == 0, p.stdout + p.stderr
        r = np.load(out)
        for key in ("mx", "am", "ct"):
            assert np.array_equal(r[key + "_a"], r[key + "_b"]), key
        _against_oracle(ref, r["mx_b"], r["am_b"], r["ct_b"], invalid=[9])
