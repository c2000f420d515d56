"""Pins for the cluster-level oracle (oracle/cluster.py).

* Hand-built volumes whose component sizes are known: cubes, a line, voxels
  that touch only along an edge or at a corner (separate under 6-connectivity,
  joined under 18 / 26).
* A breadth-first flood fill written here, on random small volumes, for each
  connectivity.
* Monotone in the threshold; below every value, the largest connected part of
  the mask; the per-voxel table agrees with the maximum.
"""
import itertools
from collections import deque

import numpy as np
import pytest

import oracle
from oracle import cluster as C
from paper_1703_01506_gb300 import synth


def _offsets(connectivity):
    out = []
    for d in itertools.product((-1, 0, 1), repeat=3):
        s = sum(abs(x) for x in d)
        if s == 0:
            continue
        if (connectivity == 6 and s == 1) or (connectivity == 18 and s <= 2) or connectivity == 26:
            out.append(d)
    return out


def _bfs_sizes(vol, connectivity):
    seen = np.zeros(vol.shape, dtype=bool)
    sizes = []
    offs = _offsets(connectivity)
    for p in zip(*np.nonzero(vol)):
        if seen[p]:
            continue
        seen[p] = True
        q, k = deque([p]), 0
        while q:
            x = q.popleft()
            k += 1
            for d in offs:
                y = tuple(a + b for a, b in zip(x, d))
                if all(0 <= y[i] < vol.shape[i] for i in range(3)) and vol[y] and not seen[y]:
                    seen[y] = True
                    q.append(y)
        sizes.append(k)
    return sorted(sizes)


def test_known_shapes():
    vol = np.zeros((8, 9, 10), dtype=bool)
    vol[0:2, 0:2, 0:2] = True          # cube of 8
    vol[5, 2, 3:8] = True              # line of 5
    vol[3, 6, 6] = True                # two voxels sharing only an edge
    vol[4, 7, 6] = True
    vol[7, 8, 9] = True                # two voxels sharing only a corner
    vol[6, 7, 8] = True
    for conn, want in ((6, [1, 1, 1, 1, 5, 8]), (18, [1, 1, 2, 5, 8]), (26, [2, 2, 5, 8])):
        _, sizes = C.label_volume(vol, conn)
        assert sorted(sizes.tolist()) == want, conn


@pytest.mark.parametrize("conn", [6, 18, 26])
def test_against_flood_fill(conn):
    rng = np.random.default_rng(conn)
    for _ in range(5):
        vol = rng.random((7, 6, 9)) < 0.3
        _, sizes = C.label_volume(vol, conn)
        assert sorted(sizes.tolist()) == _bfs_sizes(vol, conn)


def _fixture():
    dims = (12, 14, 11)
    X, mask = synth.brain_field(24, 12, grid=dims, center=(6, 7, 5), semi_axes=(5, 6, 4.5),
                                fwhm=3.0, effect=0.8, effect_radius=3.0, seed=5)
    mask = mask.numpy().astype(bool)
    return X.numpy()[:, mask], mask, dims


def test_monotone_and_whole_mask():
    Xm, mask, dims = _fixture()
    perms = synth.perms_pcg32(24, 30, seed=3)
    prev = None
    for tau in (-50.0, 0.0, 1.0, 2.0, 3.5):
        m = C.cluster_max_sizes(Xm, 12, perms, mask, dims, tau)
        if prev is not None:
            assert np.all(m <= prev)
        prev = m
    _, sizes = C.label_volume(mask.reshape(dims), 6)
    assert np.all(C.cluster_max_sizes(Xm, 12, perms, mask, dims, -1e9) == sizes.max())


def test_table_matches_maximum_and_labels():
    Xm, mask, dims = _fixture()
    ident = np.arange(24, dtype=np.int32)[None, :]
    t = oracle.t_rows(Xm, 12, ident)[0]
    for conn in (6, 26):
        label, size = C.cluster_table(t, mask, dims, 2.0, conn)
        mx = C.cluster_max_sizes(Xm, 12, ident, mask, dims, 2.0, conn)[0]
        assert size.max() == mx
        on = t >= 2.0
        assert np.all((label >= 0) == on) and np.all(size[~on] == 0)
        for lab in np.unique(label[on]):   # representative = smallest index of the cluster
            members = np.flatnonzero(label == lab)
            assert members.min() == lab and np.all(size[members] == members.size)
