"""Cluster-level summaries of thresholded statistic maps (test infrastructure only).

The paper reports SnPM's cluster tables (Sec. 6, Figs. 8-9): clusters of
voxels of a thresholded t map with their size k and peak statistic T. With
relabellings, the same clustering gives the permutation distribution of the
largest cluster, the cluster-level analogue of the max-null (Sec. 2):

    max_size_i = largest connected set of mask voxels with t_ij >= tau,

for each relabelling i, under 6-, 18- or 26-connectivity on the 3D grid
(voxels sharing a face; a face or an edge; a face, an edge or a corner).

Plain statement: the rows of T come from the FP64 oracle (``t_rows``), each
row is put back on the grid and labelled with scipy's connected-component
routine (``scipy.ndimage.label``) with the matching structuring element, and
the component sizes are counted. Grid index g = (i0 * d1 + i1) * d2 + i2
(C order); voxels without a statistic (NaN) never exceed tau.
"""
import numpy as np
from scipy import ndimage

from . import t_rows

_RANK = {6: 1, 18: 2, 26: 3}


def label_volume(active, connectivity=6):
    """Connected components of a boolean 3D volume: (labels, sizes), labels 0
    outside, 1..k inside; sizes[c - 1] = voxels of component c."""
    st = ndimage.generate_binary_structure(3, _RANK[connectivity])
    lab, k = ndimage.label(active, structure=st)
    sizes = np.bincount(lab.ravel(), minlength=k + 1)[1:]
    return lab, sizes


def _volume(values, mask, dims, tau):
    vol = np.zeros(int(np.prod(dims)), dtype=bool)
    with np.errstate(invalid="ignore"):
        vol[np.flatnonzero(mask)] = values >= tau
    return vol.reshape(dims)


def cluster_max_sizes(X, n1, perms, mask, dims, tau, connectivity=6):
    """Largest cluster of {t >= tau} per relabelling (0 when no voxel exceeds).
    X: (n, v) data of the mask voxels in mask (raster) order; mask: (prod(dims),)
    bool; perms: (P, n)."""
    mask = np.asarray(mask, dtype=bool)
    T = t_rows(X, n1, perms)
    out = np.zeros(T.shape[0], dtype=np.int64)
    for i in range(T.shape[0]):
        _, sizes = label_volume(_volume(T[i], mask, dims, tau), connectivity)
        out[i] = sizes.max() if sizes.size else 0
    return out


def cluster_table(t_map, mask, dims, tau, connectivity=6):
    """Clusters of the map {t >= tau}: per mask voxel its cluster's smallest
    mask index (-1 below tau) and its cluster's size (0 below tau)."""
    mask = np.asarray(mask, dtype=bool)
    lab, sizes = label_volume(_volume(np.asarray(t_map, dtype=np.float64), mask, dims, tau),
                              connectivity)
    lm = lab.ravel()[np.flatnonzero(mask)]
    rep = np.full(sizes.size + 1, -1, dtype=np.int64)
    for j in range(lm.size - 1, -1, -1):  # smallest mask index of each component
        if lm[j]:
            rep[lm[j]] = j
    label = np.where(lm > 0, rep[lm], -1)
    size = np.where(lm > 0, np.concatenate([[0], sizes])[lm], 0)
    return label, size
