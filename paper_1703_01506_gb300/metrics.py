"""Host-side evaluation measures of the paper (Sec. 5.5) over results the
library computed on the GPU (FWER p-value maps from ``pt_fwer_pvalues``)."""
import numpy as np


def resampling_risk(p1, p2, alpha):
    """Resampling risk (Sec. 5.5, Eq. (6)) between two methods' FWER-corrected
    p-value maps at level ``alpha``: a voxel is rejected when p <= alpha (NaN,
    a voxel without a statistic, is never rejected). v1, v2 are the two
    methods' rejection counts and vc the count of voxels both reject;
    risk = ((v1 - vc)/v1 + (v2 - vc)/v2) / 2, where a method with no rejection
    contributes 0 for its own term. Returns a dict with risk, v1, v2, vc."""
    p1 = np.asarray(p1, dtype=np.float64)
    p2 = np.asarray(p2, dtype=np.float64)
    if p1.shape != p2.shape:
        raise ValueError("p-value maps of different shapes")
    r1 = np.nan_to_num(p1, nan=2.0) <= alpha
    r2 = np.nan_to_num(p2, nan=2.0) <= alpha
    v1, v2 = int(r1.sum()), int(r2.sum())
    vc = int((r1 & r2).sum())
    risk = ((v1 - vc) / v1 if v1 else 0.0) + ((v2 - vc) / v2 if v2 else 0.0)
    return {"risk": risk / 2.0, "v1": v1, "v2": v2, "vc": vc}
