"""Host-side check of the cluster l1 fit's shared-memory carve-up and index
arithmetic (no GPU), restated from the kernels' layout rules (csrc/pt_rapid.cu:
clu_carve, choose_cluster, the Gauss-Jordan staging, the ADMM share split, the
training update's chunks and the QR apply's R^-1), for every rank 1..128 and sample
counts from r to 20,000:

* the smallest cluster (from 2 for recovery, 16 for the sequential fits) whose
  per-CTA rows fit the shared-memory limit exists up to the documented sizes,
  and r = 50, m = 1750 takes 2 CTAs, r = 100, m = 2100 takes 8;
* the Gauss-Jordan staging (pivot columns, pivot rows, z) fits the cross-warp
  buffer, one pass of CW columns per lane covers the padded columns, the
  rows of a warp cover R, and the vector accesses stay 16- or 8-byte aligned;
* the ADMM share's GS lanes x CH terms cover the padded rank exactly once, in
  whole float4 runs;
* the Gram row groups fit the CTA and the Gram partial only shares the ADMM
  vectors' space when it fits there;
* every pushed vector fits a slot; the bulk copies' byte counts stay below the
  mbarrier transaction limit (2^20 - 1);
* the training update's two buffers and the QR apply's R^-1 fit shared memory.
"""
import pytest

K_MAX_RANK = 128
K_SLOT = K_MAX_RANK + 8
K_CLU_THREADS = 512
K_CLU_WARPS = K_CLU_THREADS // 32
SMEM_LIMIT = 227 * 1024 - 64
OPTIN_MAX = 232448
TX_LIMIT = (1 << 20) - 1


def padded_rank(r):
    return (r + 3) // 4 * 4 if r <= 64 else (r + 7) // 8 * 8


def clu_rs(RP):
    return RP + 4 if (RP // 4) % 2 == 0 else RP


def up4(x):
    return (x + 3) // 4 * 4


def clu_carve(mloc, R, RP, CL, n_pad=0):
    """Floats taken by each region, in the kernels' order; returns (bytes, gp_aliased)."""
    RS, RG = clu_rs(RP), up4(R)
    o = 0
    o += up4(mloc * RS)             # A
    o += 4 * up4(mloc)              # b, s, y, x
    o += up4(mloc)                  # idx
    o += up4(R * RG)                # G
    gp = R * RG
    aliased = gp <= 3 * up4(mloc)
    if not aliased:
        o += up4(gp)                # Gp
    o += up4(2 * CL * K_SLOT)       # xch
    o += up4(K_SLOT)                # stage
    o += up4(K_CLU_WARPS * RP)      # red
    o += up4(K_SLOT)                # vec
    o += up4(RP)                    # wv
    o += up4(8 + K_CLU_WARPS)       # misc
    o += up4(16)                    # pinv
    o += up4(n_pad)                 # Lrow
    return 4 * o, aliased


def choose_cluster(m, R, RP, first):
    CL = first
    while CL <= 16:
        b, _ = clu_carve((m + CL - 1) // CL, R, RP, CL)
        if b <= SMEM_LIMIT:
            return CL, b
        CL *= 2
    return 0, 0


def update_smem(RP):
    coef = up4(3 * RP + 2) * 4
    row = clu_rs(RP) * 4
    ch = 256
    while ch > 32 and coef + 2 * ch * row > SMEM_LIMIT - 4096:
        ch -= 32
    return ch, coef + 2 * ch * row


RANKS = list(range(1, K_MAX_RANK + 1))


@pytest.mark.parametrize("R", RANKS)
def test_fit_layout_for_every_rank(R):
    RP = padded_rank(R)
    RG = up4(R)
    assert RP % 4 == 0 and R <= RG <= RP <= K_MAX_RANK
    # Gauss-Jordan staging in the cross-warp buffer: fac (4R), rowb (4R), z (4 RG);
    # z starts 32R bytes in, a multiple of 16
    assert 8 * R + 4 * RG <= K_CLU_WARPS * RP
    assert (8 * R * 4) % 16 == 0
    CW = 2 if RP <= 64 else 4
    assert CW * 32 >= RP and RG % CW == 0           # one vector pass covers the padded columns
    rows_per_warp = (RP + K_CLU_WARPS - 1) // K_CLU_WARPS
    assert rows_per_warp * K_CLU_WARPS >= R
    # ADMM share of w: GS lanes per column over CH-long float4 runs
    GS = 8 if K_CLU_THREADS // RP >= 8 else (4 if K_CLU_THREADS // RP >= 4 else 2)
    CH = ((RP + GS - 1) // GS + 3) // 4 * 4
    assert CH % 4 == 0 and GS * CH >= RP and 32 % GS == 0
    covered = sorted(d for g in range(GS) for d in range(g * CH, g * CH + CH) if d < RG)
    assert covered == list(range(RG))              # every term once
    # Gram tiles and row groups
    RT = RP // 4
    ntile = RT * (RT + 1) // 2
    ngr = 1 if ntile >= K_CLU_THREADS else K_CLU_THREADS // ntile
    assert ngr >= 1 and (ngr == 1 or ntile * ngr <= K_CLU_THREADS)
    # pushed vectors: A^T r and ||r||^2 (R + 1), shares of w (R)
    assert R + 1 <= K_SLOT
    # training update and QR apply
    ch, ub = update_smem(RP)
    assert 32 <= ch <= 256 and ub <= SMEM_LIMIT - 4096
    assert ch * RP * 4 <= TX_LIMIT
    assert 4 * RP * RP <= OPTIN_MAX - 1024             # R^-1 of the QR apply


@pytest.mark.parametrize("R", [1, 3, 5, 12, 20, 50, 52, 64, 70, 100, 104, 128])
@pytest.mark.parametrize("m", [None, 100, 449, 898, 1750, 2100, 2513, 5000, 20000])
def test_cluster_choice_and_transfer_sizes(R, m):
    m = R if m is None else max(m, R)
    RP = padded_rank(R)
    for first in (2, 16):
        CL, b = choose_cluster(m, R, RP, first)
        if CL == 0:
            # only large problems do not fit a 16-CTA cluster (the library then
            # returns PT_ERR_UNSUPPORTED): r m above 2.5e5 (m > 2,144 at r = 128,
            # 4,480 at r = 100, 13,280 at r = 50)
            assert R * m > 250_000, (R, m, first)
            continue
        assert CL >= first and b <= SMEM_LIMIT
        mloc = (m + CL - 1) // CL
        assert mloc * RP * 4 <= TX_LIMIT                # one bulk-copy phase per relabelling
        bytes_, aliased = clu_carve(mloc, R, RP, CL)
        assert bytes_ == b
        if aliased:                                     # the partial fits in s, y, x
            assert R * up4(R) <= 3 * up4(mloc)
        # the training kernel's launch takes the larger of the fit and the update
        if first == 16:
            assert max(b, update_smem(RP)[1]) <= SMEM_LIMIT


def test_largest_sample_counts():
    """The largest m per rank that fits (documented in include/pt.h)."""
    def largest(R):
        RP, lo, hi = padded_rank(R), R, 200_000
        while lo < hi:
            mid = (lo + hi + 1) // 2
            lo, hi = (mid, hi) if choose_cluster(mid, R, RP, 2)[0] else (lo, mid - 1)
        return lo
    assert [largest(R) for R in (50, 100, 128)] == [13280, 4480, 2144]


def test_workload_cluster_sizes():
    """r = 50, m = 1750 (n = 200 workload): 2-CTA recovery clusters; r = 100,
    m = 2100 (n = 400 workload): 8-CTA clusters (one R x R matrix per CTA since
    the inverse is formed in place); both 16 for the sequential fits."""
    assert choose_cluster(1750, 50, padded_rank(50), 2)[0] == 2
    assert choose_cluster(2100, 100, padded_rank(100), 2)[0] == 8
    assert choose_cluster(1750, 50, padded_rank(50), 16)[0] == 16
    assert choose_cluster(2100, 100, padded_rank(100), 16)[0] == 16
