"""NaivePT over a long list of relabellings in chunks, with a checkpoint after
every chunk, so that an interrupted run continues where it stopped.

Rows of the permutation testing matrix are independent (each row's maximum is
its own), and the per-voxel exceedance counts are integer sums over rows, so a
run split at any row gives exactly the outputs of one call: the maxima of a
chunk are written to their rows, and the counts of every chunk are added in
place on the device (``pt_naive_opts.accumulate_counts``). The checkpoint
(``.npz``, replaced atomically) holds the rows done, the maxima and argmax so
far and the counts; it also holds a digest of the relabellings, the sizes and
the options, and a checkpoint of another problem is refused.

Every step of the computation runs in the library; this module only cuts the
rows, stores the state and restores it.
"""
import hashlib
import os

import numpy as np
import torch

from . import binding as B

_FMT = 1


def problem_digest(perms, v, opts):
    """Digest of what a checkpoint must match: the relabellings (bytes), the
    number of mask voxels and the options that change the outputs."""
    h = hashlib.sha256()
    p = np.ascontiguousarray(perms.cpu().numpy() if torch.is_tensor(perms) else perms,
                             dtype=np.int32)
    h.update(np.asarray(p.shape, dtype=np.int64).tobytes())
    h.update(p.tobytes())
    h.update(np.asarray([v, opts.precision, opts.two_sided], dtype=np.int64).tobytes())
    return h.hexdigest()


def save_state(path, digest, rows_done, maxnull, argmax, counts):
    """Writes the checkpoint atomically (a temporary file, then a rename)."""
    tmp = path + ".tmp.npz"
    np.savez(tmp, fmt=np.int64(_FMT), digest=np.array(digest), rows_done=np.int64(rows_done),
             maxnull=maxnull, argmax=argmax, counts=counts)
    os.replace(tmp, path)


def load_state(path, digest, P, v):
    """The saved state, or None when there is no checkpoint. Raises ValueError
    for a checkpoint of another problem or a damaged one."""
    if not os.path.exists(path):
        return None
    with np.load(path) as z:
        if int(z["fmt"]) != _FMT or str(z["digest"]) != digest:
            raise ValueError("checkpoint %s belongs to another problem" % path)
        rows_done = int(z["rows_done"])
        mx, am, ct = z["maxnull"], z["argmax"], z["counts"]
    if not (0 <= rows_done <= P and mx.shape == (P,) and am.shape == (P,) and ct.shape == (v,)):
        raise ValueError("checkpoint %s is damaged" % path)
    return rows_done, mx, am, ct


def maxnull_naive_resumable(ctx, perms, chunk_rows, checkpoint, precision=B.PT_PREC_BF16X3,
                            two_sided=False, max_chunks=None):
    """NaivePT (Alg. 1) over the rows of ``perms`` (P x n int32 CUDA tensor) in
    chunks of ``chunk_rows`` rows. After each chunk the state goes to
    ``checkpoint``; if the file exists when the call starts, the run continues
    after its last chunk. ``max_chunks`` stops after that many chunks of this
    call (returns None). Returns host arrays (maxnull float32[P], argmax
    int32[P], counts uint32[v]); the checkpoint is left in place."""
    if chunk_rows < 1:
        raise ValueError("chunk_rows must be >= 1")
    dev = perms.device
    P = perms.shape[0]
    v = B.pt_num_voxels(ctx)
    opts = B.naive_opts(precision, two_sided, accumulate_counts=True)
    digest = problem_digest(perms, v, opts)
    st = load_state(checkpoint, digest, P, v)
    if st is None:
        rows_done = 0
        mx_h = np.zeros(P, np.float32)
        am_h = np.full(P, -1, np.int32)
        ct_h = np.zeros(v, np.uint32)
    else:
        rows_done, mx_h, am_h, ct_h = st
        mx_h, am_h, ct_h = mx_h.copy(), am_h.copy(), ct_h.copy()
    counts = torch.as_tensor(ct_h.view(np.int32)).to(dev)  # device copy the chunks add to
    done_now = 0
    while rows_done < P:
        if max_chunks is not None and done_now >= max_chunks:
            return None
        r1 = min(P, rows_done + chunk_rows)
        part = perms[rows_done:r1].contiguous()
        mx = torch.empty(r1 - rows_done, dtype=torch.float32, device=dev)
        am = torch.empty(r1 - rows_done, dtype=torch.int32, device=dev)
        B.pt_maxnull_naive_ex(ctx, part, opts, mx, am, counts)
        B.pt_sync(ctx)
        mx_h[rows_done:r1] = mx.cpu().numpy()
        am_h[rows_done:r1] = am.cpu().numpy()
        ct_h = counts.cpu().numpy().view(np.uint32).copy()
        rows_done = r1
        done_now += 1
        save_state(checkpoint, digest, rows_done, mx_h, am_h, ct_h)
    return mx_h, am_h, ct_h
