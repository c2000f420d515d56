"""The table of tuned launch configurations (host only, no GPU): defaults per n,
validation of recorded configurations, bucketed lookup, and the text file
round trip."""
import os

import pytest

PREC_BF16X2, PREC_BF16X3 = 1, 2


@pytest.fixture()
def B():
    from paper_1703_01506_gb300 import binding, build
    build.build()
    binding.load()
    binding.pt_tune_clear()
    yield binding
    binding.pt_tune_clear()


def test_default_tile_follows_n(B):
    # The largest voxel tile whose BF16x3 pieces fit in shared memory beside a
    # label ring of at least 8 stages and 2,048 columns x k-steps, else beside
    # 4 stages (544); the 96-voxel tile is for two pieces only.
    for n, tile in [(3, 256), (100, 256), (128, 256), (129, 128), (240, 128), (256, 128),
                    (300, 64), (352, 64), (544, 64)]:
        found, cfg = B.pt_tune_lookup(n, PREC_BF16X3, 0, 10000, 1000)
        assert found == 0 and cfg.voxel_tile == tile, (n, cfg.as_tuple())
        assert cfg.ksteps_per_stage in (1, 2, 4, 8) and cfg.stages >= 2
        assert cfg.items_per_sm == 8
    assert B.pt_tune_lookup(560, PREC_BF16X3, 0, 10000, 1000)[0] == -1  # no tile fits
    assert B.pt_tune_lookup(560, PREC_BF16X2, 0, 10000, 1000)[0] == 0
    for n, tile in [(100, 256), (200, 128), (380, 128), (392, 96), (400, 96), (512, 64)]:
        found, cfg = B.pt_tune_lookup(n, PREC_BF16X2, 0, 10000, 1000)  # two pieces
        assert found == 0 and cfg.voxel_tile == tile, (n, cfg.as_tuple())
    assert B.pt_tune_lookup(2, PREC_BF16X3, 0, 10, 10)[0] == -1
    assert B.pt_tune_lookup(100, 0, 0, 10, 10)[0] == -1  # FP32 has no tensor-core config


def test_set_lookup_and_buckets(B):
    B.pt_tune_set(360, PREC_BF16X3, 0, 200000, 10000, 64, 4, 4, 2)
    found, cfg = B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 10000)
    assert found == 1 and cfg.as_tuple() == (64, 4, 4, 2)
    # same half-octave buckets of v and P, same padded n (353..368 -> 368)
    assert B.pt_tune_lookup(357, PREC_BF16X3, 0, 210000, 11000)[0] == 1
    # other bucket, precision or sidedness: no entry
    assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 400000, 10000)[0] == 0
    assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 30000)[0] == 0
    assert B.pt_tune_lookup(360, PREC_BF16X2, 0, 200000, 10000)[0] == 0
    assert B.pt_tune_lookup(360, PREC_BF16X3, 1, 200000, 10000)[0] == 0


@pytest.mark.parametrize("cfg", [
    (128, 4, 4, 2),   # another tile than n fixes
    (64, 1, 8, 2),    # fewer than 2 stages
    (64, 40, 1, 2),   # more stages than fit
    (64, 4, 3, 2),    # k-steps per stage not a power of two
    (64, 4, 16, 2),   # k-steps per stage too large
    (64, 4, 4, 0),    # items per SM out of range
    (64, 4, 4, 65),
])
def test_set_rejects_invalid(B, cfg):
    with pytest.raises(B.PtError):
        B.pt_tune_set(360, PREC_BF16X3, 0, 200000, 10000, *cfg)
    assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 10000)[0] == 0


def test_save_load_round_trip(B, tmp_path):
    B.pt_tune_set(360, PREC_BF16X3, 0, 200000, 10000, 64, 4, 4, 2)
    B.pt_tune_set(100, PREC_BF16X3, 1, 231719, 10000, 256, 2, 4, 1)
    B.pt_tune_set(200, PREC_BF16X2, 0, 500000, 100000, 128, 2, 2, 4)
    path = str(tmp_path / "tune.txt")
    B.pt_tune_save(path)
    lines = open(path).read().splitlines()
    assert lines[0].startswith("# pt tuned launch configurations")
    assert len([ln for ln in lines if not ln.startswith("#")]) == 3
    B.pt_tune_clear()
    assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 10000)[0] == 0
    B.pt_tune_load(path)
    assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 10000)[1].as_tuple() == (64, 4, 4, 2)
    assert B.pt_tune_lookup(100, PREC_BF16X3, 1, 231719, 10000)[1].as_tuple() == (256, 2, 4, 1)
    assert B.pt_tune_lookup(200, PREC_BF16X2, 0, 500000, 100000)[1].as_tuple() == (128, 2, 2, 4)


def test_load_rejects_bad_files_and_keeps_table(B, tmp_path):
    B.pt_tune_set(360, PREC_BF16X3, 0, 200000, 10000, 64, 4, 4, 2)
    good = "# pt tuned launch configurations v2\n"
    cases = {
        "missing_header": "368 2 0 35 26 64 4 4 2 1.0\n",
        "short_line": good + "368 2 0 35 26 64 4 4\n",
        "wrong_tile": good + "368 2 0 35 26 128 4 4 2 1.0\n",
        "odd_n_pad": good + "300 2 0 35 26 64 4 4 2 1.0\n",
        "bad_precision": good + "368 0 0 35 26 64 4 4 2 1.0\n",
        "empty": "",
    }
    for name, text in cases.items():
        path = str(tmp_path / (name + ".txt"))
        with open(path, "w") as f:
            f.write(text)
        with pytest.raises(B.PtError):
            B.pt_tune_load(path)
        # the earlier entry is untouched and no partial entry was merged
        assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 10000)[1].as_tuple() == (64, 4, 4, 2)
    with pytest.raises(B.PtError):
        B.pt_tune_load(str(tmp_path / "does_not_exist.txt"))
    with open(str(tmp_path / "ok.txt"), "w") as f:
        f.write(good + "# comment\n\n368 2 0 35 26 64 2 8 1 2.5\n")
    B.pt_tune_load(str(tmp_path / "ok.txt"))
    assert B.pt_tune_lookup(360, PREC_BF16X3, 0, 200000, 10000)[1].as_tuple() == (64, 2, 8, 1)
