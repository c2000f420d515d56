"""Host-side check of the fused tensor-core kernel's index arithmetic (no GPU):
for the launch configurations the library reports (defaults for every n, and
every configuration the autotuner may try), the shared-memory carve-up fits the
opt-in limit, the TMEM accumulators fit their allocation, the MMA shapes are
legal for kind::f16 (M = 128: N a multiple of 16 in [16, 256]), shared-memory
descriptor addresses fit their 14-bit field, and every TMA box starts inside
its tensor map (a data tile runs past the padded voxel count only into columns
the epilogue masks; a label box may run past the last block only into zero
fill)."""
import pytest

SMEM_LIMIT = 232448 - 1024   # opt-in maximum the host code keeps below
STEP_BYTES = 4096            # one k-step of labels: 128 x 16 BF16
MAX_BLOCKS_PER_ITEM = 255


@pytest.fixture(scope="module")
def B():
    from paper_1703_01506_gb300 import binding, build
    build.build()
    binding.load()
    binding.pt_tune_clear()
    return binding


def smem_bytes(NT, n_pad, pieces, stages, kps):
    return (pieces * NT * n_pad * 2 + stages * kps * STEP_BYTES + NT * 4 +
            (MAX_BLOCKS_PER_ITEM + 1) + (7 + 2 * stages) * 8 + 16)


def nacc(NT, pieces):
    return 1 if NT == 256 else (2 if NT >= 96 else pieces)


def check_config(n, pieces, cfg, v, P):
    NT, S, kps = cfg.voxel_tile, cfg.stages, cfg.ksteps_per_stage
    n_pad = (n + 15) // 16 * 16
    assert NT in (256, 128, 96, 64) and S >= 2 and kps in (1, 2, 4, 8)
    # shared memory: data tile, label ring, voxel thresholds, block flags, barriers
    assert smem_bytes(NT, n_pad, pieces, S, kps) <= SMEM_LIMIT, (n, cfg.as_tuple())
    xs_end = pieces * NT * n_pad * 2
    ring_end = xs_end + S * kps * STEP_BYTES
    assert (ring_end >> 4) < (1 << 14)           # descriptor start-address field
    assert xs_end % 16 == 0 and STEP_BYTES % 16 == 0  # TMA destinations 16-byte aligned
    # TMEM: two accumulator sets of NACC x NT FP32 columns, allocation a power of two
    acc = nacc(NT, pieces) * NT
    cols = 2 * acc
    alloc = 128 if cols <= 128 else (256 if cols <= 256 else 512)
    assert cols <= alloc <= 512
    # MMA widths issued per k-step (M = 128)
    if nacc(NT, pieces) == 1:
        widths = [NT] * pieces
    elif nacc(NT, pieces) == pieces:
        widths = [pieces * NT]
    else:
        widths = [2 * NT, NT]
    for N in widths:
        assert N % 16 == 0 and 16 <= N <= 256, (n, pieces, NT, N)
    # TMA boxes (view rows of 512 bytes = 256 BF16)
    assert NT * n_pad // 256 <= 256 and 8 * kps <= 256
    v_pad = (v + 255) // 256 * 256
    x_rows = 3 * v_pad * n_pad // 256
    for q in range(pieces):
        for vt in range((v + NT - 1) // NT):
            row0 = (q * v_pad * n_pad + vt * NT * n_pad) // 256
            assert (q * v_pad * n_pad + vt * NT * n_pad) % 256 == 0
            assert row0 < x_rows                   # every box starts inside the map
            # a tile that runs past v_pad (NT = 96 does not divide 256) reads the
            # next piece's rows or the map's zero fill into voxel columns >= v
            # only, which the epilogue never counts or compares
            if vt * NT + NT > v_pad:
                assert vt * NT < v <= v_pad
    nblocks = (P + 127) // 128
    l_rows = nblocks * 128 * n_pad // 256
    ksteps = n_pad // 16
    for b in range(nblocks):
        for ks in range(0, ksteps, kps):
            row = b * (n_pad // 2) + ks * 8
            assert row < l_rows                    # every box starts inside the labels
            nk = min(kps, ksteps - ks)
            assert row + 8 * nk <= l_rows          # the k-steps it feeds are real labels


@pytest.mark.parametrize("pieces,prec", [(3, 2), (2, 1)])
def test_default_configurations(B, pieces, prec):
    n_max = 544 if pieces == 3 else 800
    for n in list(range(3, 130)) + list(range(130, n_max + 1, 7)) + [n_max]:
        found, cfg = B.pt_tune_lookup(n, prec, 0, 1000, 1000)
        assert found == 0, n
        check_config(n, pieces, cfg, v=1000 + n, P=1000 + 3 * n)


@pytest.mark.parametrize("pieces,prec", [(3, 2), (2, 1)])
@pytest.mark.parametrize("n", [20, 100, 112, 128, 200, 240, 300, 400, 544])
def test_autotuner_candidates(B, pieces, prec, n):
    """Every configuration the library accepts for n (what pt_autotune_naive may
    try and record): all ring shapes that pt_tune_set takes."""
    found, d = B.pt_tune_lookup(n, prec, 0, 5000, 5000)
    if found < 0:
        pytest.skip("no tile fits this n")
    tried = 0
    for kps in (1, 2, 4, 8):
        for S in range(2, 33):
            try:
                B.pt_tune_set(n, prec, 0, 5000, 5000, d.voxel_tile, S, kps, 8)
            except B.PtError:
                continue
            cfg = B.pt_tune_lookup(n, prec, 0, 5000, 5000)[1]
            check_config(n, pieces, cfg, v=5000, P=5000)
            tried += 1
    B.pt_tune_clear()
    assert tried >= 4
