"""Writes rapid_seed_spread_smooth_n40.txt: the FP64 RapidPT oracle's own
spread over seeds on the smoothed-field fixture of the GPU end-to-end test.

RapidPT (Alg. 2) is randomised (the basis initialisation, the sampled voxels
and the residual draws depend on the seed), so its FWER thresholds (Sec. 5.4)
differ from the exhaustive ones by an amount that varies from seed to seed.
This script runs the oracle (and nothing else) for seeds 1..8 and records, per
seed, KL(NaivePT || RapidPT) and the relative FWER 0.05 / 0.01 threshold
errors against the oracle's exhaustive max-null. The GPU test bounds each of
its own seeds by these numbers.

Run from the repository root: python tests/golden/make_rapid_seed_spread.py
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from oracle import rapid as R  # noqa: E402
from paper_1703_01506_gb300 import synth  # noqa: E402

# the fixture of tests/test_gpu_rapid.py::test_maxnull_rapid_end_to_end
N, N1, P, RANK, ETA, ELL, PASSES = 40, 20, 3000, 20, 0.02, 80, 20
GRID, AXES, FWHM, DATA_SEED = (30, 36, 30), (12, 15, 12), 6.0, 3
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "rapid_seed_spread_smooth_n40.txt")


def fixture():
    X, mask = synth.brain_field(N, N1, grid=GRID, center=tuple(g // 2 for g in GRID),
                                semi_axes=AXES, fwhm=FWHM, seed=DATA_SEED)
    return X.numpy()[:, mask.numpy().astype(bool)], synth.perms_pcg32(N, P, seed=1)


def main():
    X, perms = fixture()
    ref = oracle.naive(X, N1, perms).maxnull
    lines = ["# FP64 RapidPT oracle vs its exhaustive max-null on the smoothed field",
             "# n=%d n1=%d v=%d P=%d rank=%d eta=%g n_train=%d train_passes=%d "
             "(brain_field grid %s axes %s fwhm %g seed %d; PCG32 relabellings seed 1)"
             % (N, N1, X.shape[1], P, RANK, ETA, ELL, PASSES, GRID, AXES, FWHM, DATA_SEED),
             "# thresholds: c-th largest value, c = floor(alpha P) + 1; KL over 100 common bins",
             "# columns: seed KL rel_err_thr_0.05 rel_err_thr_0.01"]
    for seed in range(1, 9):
        mx = R.rapid(X, N1, perms, RANK, ETA, ELL, R.RapidOpts(train_passes=PASSES, seed=seed)).maxnull
        e = [R.fwer_threshold(mx, a) / R.fwer_threshold(ref, a) - 1.0 for a in (0.05, 0.01)]
        lines.append("%d %.6f %+.6f %+.6f" % (seed, R.kl_divergence(ref, mx), e[0], e[1]))
        print(lines[-1], flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
