"""Error of each contraction path against the FP64 oracle (run as a script on a
GPU; not collected by pytest): python tests/precision_report.py

For the FP32 CUDA-core path and the BF16x2 / BF16x3 tensor-core paths, on
  * gauss_n20_v2000 (n=20, 2,000 voxels, 1,000 relabellings: every output), and
  * brain_n100_v232k (n=100, 231,719 voxels, 10,000 relabellings: 16 sampled rows
    against the oracle's full rows, 64 sampled voxels' counts over all rows),
it reports the largest relative error of the max-null values, the share of rows
whose argmax agrees, count disagreements (and how many lie outside the
oracle's near-tie entries), and the relative error of the FWER 0.05 / 0.01
thresholds (full max-null only). Prints one JSON line per (workload, path).
"""
import json
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import rapid as R  # noqa: E402
from paper_1703_01506_gb300 import binding as B  # noqa: E402
from paper_1703_01506_gb300 import synth  # noqa: E402

NAMES = {0: "fp32", 1: "bf16x2", 2: "bf16x3"}


def tie_rel(precision, n):
    eps24 = 2.0 ** -24
    if precision == 1:
        return 2.0 * (2.0 ** -17 + (n + 4) * eps24)
    return 2.0 * (n + 4) * eps24


def gpu_run(X, mask, n1, perms, precision):
    ctx = B.pt_prepare(X, n1, mask)
    pd = torch.as_tensor(perms).cuda()
    mx, am, ct = B.maxnull_naive(ctx, pd, precision=precision)
    ctx.close()
    return (mx.cpu().numpy().astype(np.float64), am.cpu().numpy().astype(np.int64),
            ct.cpu().numpy().astype(np.int64))


def summarise(name, precision, ref, mx, am, ct, ct_ref=None, near=None, full=True):
    rel = np.abs(mx - ref.maxnull) / np.maximum(np.abs(ref.maxnull), 1.0)
    out = {"workload": name, "path": NAMES[precision], "rows": int(mx.size),
           "maxnull_max_rel_err": float(rel.max()),
           "argmax_agree": float(np.mean(am == ref.argmax))}
    if ct_ref is not None:
        d = np.abs(ct - ct_ref)
        out["count_disagreements"] = int(d.sum())
        out["count_disagreements_outside_near_ties"] = int(np.maximum(d - near, 0).sum())
    if full:
        for a in (0.05, 0.01):
            ta, tb = R.fwer_threshold(ref.maxnull, a), R.fwer_threshold(mx, a)
            out["fwer%g_rel_err" % a] = float(abs(tb - ta) / abs(ta))
    return out


def main():
    torch.cuda.set_device(0)
    B.load()
    # gauss_n20_v2000: every output
    w = synth.workload("gauss_n20_v2000")
    X = torch.as_tensor(w["X"]).cuda()
    for p in (0, 1, 2):
        ref = oracle.naive(w["X"], w["n1"], w["perms"], tie_rel=tie_rel(p, w["n"]))
        mx, am, ct = gpu_run(X, None, w["n1"], w["perms"], p)
        print(json.dumps(summarise(w["name"], p, ref, mx, am, ct, ref.counts.astype(np.int64),
                                   ref.near.astype(np.int64))), flush=True)
    # brain_n100_v232k: sampled rows and voxels
    w = synth.workload("brain_n100_v232k", device="cuda")
    Xm = w["X"][:, w["mask"].bool()].cpu().numpy()
    rng = np.random.default_rng(0)
    rows = np.sort(rng.choice(w["P"], 16, replace=False))
    vox = np.sort(rng.choice(Xm.shape[1], 64, replace=False))
    for p in (0, 1, 2):
        ref = oracle.naive(Xm, w["n1"], w["perms"][rows], tie_rel=tie_rel(p, w["n"]))
        refc = oracle.naive(Xm[:, vox], w["n1"], w["perms"], tie_rel=tie_rel(p, w["n"]))
        mx, am, ct = gpu_run(w["X"], w["mask"], w["n1"], w["perms"], p)
        print(json.dumps(summarise(w["name"], p, ref, mx[rows], am[rows], ct[vox],
                                   refc.counts.astype(np.int64), refc.near.astype(np.int64),
                                   full=False)), flush=True)


if __name__ == "__main__":
    main()
