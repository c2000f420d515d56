// Tensor-core (tcgen05) form of the NaivePT contraction U = L . Xn^T fused
// with the max-null / exceedance-count reduction (Alg. 1; Eq. (5) through the
// monotone map u -> t).
//
// Roles (one CTA per SM, persistent over work items = (voxel tile, block range)):
//   warp 0      TMA producer: the resident Xn tile (BF16 pieces) once per item,
//               then the label matrix L streamed one k-step (128 x 16) per stage.
//   warp 1      MMA issuer: per k-step, one tcgen05.mma per data piece into a
//               128 x NT FP32 accumulator in TMEM (two accumulators, ping-pong).
//   warps 2..17 epilogue (16 warps, 4 per TMEM lane quadrant, each owning NT/4
//               columns): tcgen05.ld rows of the accumulator (lane = relabelling,
//               column = voxel), row max -> packed (u, voxel) atomics, per-voxel
//               exceedance counts in packed 8-bit registers, optional row writes.
//
// Labels are exact in BF16 and FP16; the data enter as hi + mid (+ lo) BF16
// pieces of the unit-norm value (~16 or ~24 bits), or as hi + lo FP16 pieces of
// 2^15 times it (~22 bits; the accumulator then holds 2^15 u, and the observed
// values and written rows are scaled by that power of two, exactly).
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>
#include <algorithm>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {

// ---------------------------------------------------------------------------
// TMA descriptors (also used by pt_recon_tc.cu)
// ---------------------------------------------------------------------------
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                        &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// 2D view [rows][256] of a BF16 buffer, box [box_rows][256], no swizzle.
bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint32_t box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {256, rows};
  cuuint64_t strides[1] = {512};
  cuuint32_t box[2] = {256, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

namespace {

constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // 576
constexpr int kStepBytes = 4096;  // one k-step of labels: 128 relabellings x 16 subjects x BF16
constexpr int kSmemLimit = 232448;
constexpr int kMaxBlocksPerItem = 255;  // per-thread 8-bit exceedance counters
constexpr int kMaxStages = 32;          // label ring stages (4 KB each)
constexpr int kDefaultItemsPerSm = 8;

// One study (one prepared context and its relabellings) of a launch. Launches
// with several studies (pt_maxnull_naive_batched) walk the concatenation of
// their work items; tensor maps live in global memory with the descriptor.
struct TcStudy {  // CUtensorMap members carry their own alignment
  CUtensorMap tmL;  // labels, [P_pad * n_pad / 256][256] BF16 view
  CUtensorMap tmX;  // data pieces, [3 * v_pad * n_pad / 256][256] BF16 view
  int n_pad, ksteps;
  int64_t P, v, v_pad;
  int64_t n_chunks, blocks_per_chunk, nblocks, item_begin;
  const float* u_obs;
  const uint8_t* rowflag;    // per relabelling: 1 = observed group-1 set (not compared)
  const uint8_t* blockflag;  // per 128-row block: holds such a row
  unsigned long long* maxkey;
  uint32_t* cnt;
  float* uout;  // row writes (single-study launches only)
  const float* rowscale;  // covariate-adjusted statistic: per-row factor of the
                          // exceedance test (u * f >= u_obs); NULL for the plain t
  // F of a g-group factor (kernel mode FG > 0): label row r = i FG + h is group h
  // of relabelling i (rows h >= g - 1 are zero), u_obs holds B_obs per voxel,
  // maxkey is indexed by relabelling, and fmat + i fstride is the FG x FG matrix
  // W (zero-padded) with B = u^T W u (fstride 0: one matrix for every row).
  const float* fmat;
  int64_t fstride;
};

struct TcArgs {
  const TcStudy* studies;
  int n_studies, stages, kps;  // ring stages, k-steps per stage
  int n_pad_max;
  int64_t n_items;
  int do_reduce, write_mode;  // write_mode: 0 none, 1 u, 2 t, 3 bits u >= uthr
  int scaled;                 // the studies carry per-row factors (covariate-adjusted t)
  int f16;                    // FP16 operands (labels and 2^15-scaled data pieces)
  float uscale, inv_uscale;   // accumulator = uscale * u (2^15 for FP16 pieces, else 1)
  float k_f, ct_f;
  float uthr;                 // write_mode 3: threshold on the accumulator's scale
  uint32_t* status;
};

__device__ __forceinline__ void epi_bar() {
  asm volatile("bar.sync 1, %0;" ::"n"(32 * kEpiWarps) : "memory");
}

// Sum packed 16-bit column counters over the 32 lanes (each lane holds R
// registers = 2R columns of its relabelling row) and add them to cnt.
// Register k of a lane covers local columns 2k and 2k+1.
template <int R>
__device__ __forceinline__ void flush_counts16(uint32_t (&r)[R], int lane, int64_t col0, int64_t v,
                                               uint32_t* cnt) {
  int base = 0;
#pragma unroll
  for (int rnd = 0; rnd < 5; ++rnd) {
    const int off = 16 >> rnd;
    const int Rb = (R >> rnd) > 0 ? (R >> rnd) : 1;
    if (Rb >= 2) {
      const bool up = (lane & off) != 0;
#pragma unroll
      for (int q = 0; q < Rb / 2; ++q) {
        const uint32_t send = up ? r[q] : r[q + Rb / 2];
        const uint32_t keep = up ? r[q + Rb / 2] : r[q];
        r[q] = keep + __shfl_xor_sync(0xffffffffu, send, off);
      }
      if (up) base += Rb / 2;
    } else {
      r[0] += __shfl_xor_sync(0xffffffffu, r[0], off);
    }
  }
  constexpr int Rf = (R >> 5) > 0 ? (R >> 5) : 1;
  constexpr int dup_mask = (R >= 32) ? 0 : (32 / R - 1);
  if ((lane & dup_mask) != 0) return;
#pragma unroll
  for (int f = 0; f < Rf; ++f) {
    const int kreg = base + f;
    const uint32_t pk = r[f];
    const int64_t c0 = col0 + 2 * kreg;
    const uint32_t lo = pk & 0xffffu, hi = pk >> 16;
    if (lo && c0 < v) atomicAdd(&cnt[c0], lo);
    if (hi && c0 + 1 < v) atomicAdd(&cnt[c0 + 1], hi);
  }
}

// 8-bit counters (register g = local columns 4g..4g+3) -> 16-bit pairs -> flush.
// flush_counts16 over R registers, R not a power of two: the largest power of
// two first, then the rest (2 columns per register).
template <int R>
__device__ __forceinline__ void flush_counts16_any(uint32_t* r, int lane, int64_t col0, int64_t v,
                                                   uint32_t* cnt) {
  constexpr int Pw = (R & (R - 1)) == 0 ? R : (R >= 16 ? 16 : (R >= 8 ? 8 : (R >= 4 ? 4 : 2)));
  flush_counts16<Pw>(*reinterpret_cast<uint32_t(*)[Pw]>(r), lane, col0, v, cnt);
  if constexpr (Pw < R) flush_counts16_any<R - Pw>(r + Pw, lane, col0 + 2 * Pw, v, cnt);
}

template <int CW>
__device__ __forceinline__ void flush_counts8(const uint32_t (&c8)[CW / 4], int lane, int64_t col0,
                                              int64_t v, uint32_t* cnt) {
  uint32_t c16[CW / 2];
#pragma unroll
  for (int g = 0; g < CW / 4; ++g) {
    c16[2 * g] = (c8[g] & 0xffu) | ((c8[g] & 0xff00u) << 8);
    c16[2 * g + 1] = ((c8[g] >> 16) & 0xffu) | ((c8[g] >> 8) & 0xff0000u);
  }
  flush_counts16_any<CW / 2>(c16, lane, col0, v, cnt);
}

template <int CW>
__device__ __forceinline__ void tc_ld_cols(uint32_t taddr, uint32_t (&r)[CW]) {
  if constexpr (CW == 8) {
    tc_ld_32x32b_x8(taddr, r);
  } else if constexpr (CW == 16) {
    tc_ld_32x32b_x16(taddr, r);
  } else {
#pragma unroll
    for (int h = 0; h < CW / 32; ++h)
      tc_ld_32x32b_x32(taddr + 32 * h, *reinterpret_cast<uint32_t(*)[32]>(&r[32 * h]));
  }
}

// Max and exceedance counts over the CW columns of one relabelling row.
// RAGGED: the block has padded relabelling rows, padded voxel columns or a row
// with the observed group-1 set. Padded entries take the value -inf (never
// counted, never a maximum); an observed-set row still competes for the
// maximum but is not compared (its count is added exactly elsewhere).
template <int CW, bool TWO, bool RAGGED, bool SCALE = false>
__device__ __forceinline__ float cols_reduce(const uint32_t (&r)[CW], const float* su_cols,
                                             int64_t gcol0, int64_t v, bool row_ok, bool cnt_ok,
                                             uint32_t (&c8)[CW / 4], float fr = 1.0f) {
  float m0 = -INFINITY, m1 = -INFINITY, m2 = -INFINITY, m3 = -INFINITY;
  const float4* s4 = reinterpret_cast<const float4*>(su_cols);
#pragma unroll
  for (int g = 0; g < CW / 4; ++g) {
    const float4 o = s4[g];
    const float ov[4] = {o.x, o.y, o.z, o.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int jj = g * 4 + e;
      float s = __uint_as_float(r[jj]);
      if (TWO) s = fabsf(s);
      if (RAGGED && (!row_ok || gcol0 + jj >= v)) s = -INFINITY;
      if (e == 0) m0 = fmaxf(m0, s);
      if (e == 1) m1 = fmaxf(m1, s);
      if (e == 2) m2 = fmaxf(m2, s);
      if (e == 3) m3 = fmaxf(m3, s);
      if ((SCALE ? s * fr : s) >= ov[e] && (!RAGGED || cnt_ok)) c8[g] += 1u << (8 * e);
    }
  }
  return fmaxf(fmaxf(m0, m1), fmaxf(m2, m3));
}

// WRITE = false: reduce only (the NaivePT path); true: rows of u or t are
// written (training rows of Alg. 2), optionally also reduced. SCALED: the
// covariate-adjusted statistic (per-row factor in the exceedance test; the
// launch's studies carry rowscale). FG > 0: the F of a g-group factor, the
// g - 1 group sums of a relabelling in FG adjacent lanes (g - 1 <= FG), which
// exchange them by shuffles; B = u^T W u replaces u, and the group's first
// lane takes the maximum and the counts.
template <int NT, bool TWO, int PIECES, bool WRITE, bool SCALED = false, int FG = 0>
__global__ void __launch_bounds__(kThreads, 1)
    tc_contract_kernel(const TcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  // Accumulators per block (NACC), summed in the epilogue. The data pieces'
  // tiles are adjacent in shared memory, so one MMA of width q NT covers q of
  // them: NT = 256 accumulates every piece in one accumulator (one MMA per
  // piece); NT = 128 and 96 keep hi and mid(+lo) apart (one MMA of width 2 NT
  // for hi and mid, one for lo); NT = 64 keeps every piece apart (one MMA of
  // width PIECES x 64 per k-step, so the label operand is read once).
  constexpr int NACC = NT == 256 ? 1 : (NT >= 96 ? 2 : PIECES);
  constexpr int ACC = NACC * NT;             // accumulator columns per buffer
  constexpr int CW = NT / 4;                 // voxel columns per epilogue thread
  constexpr int CHK = NACC > 1 ? (CW % 16 == 0 ? 16 : 8) : (CW < 32 ? CW : 32);  // per load
  constexpr int NCH = CW / CHK;              // loads per block
  const bool do_reduce = !WRITE || a.do_reduce;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.stages;
  const int KPS = a.kps;
  const uint32_t stage_bytes = uint32_t(KPS) * kStepBytes;
  uint8_t* xs = smem;
  uint8_t* ls = smem + PIECES * uint32_t(NT) * a.n_pad_max * 2;
  float* su = reinterpret_cast<float*>(ls + S * stage_bytes);
  uint8_t* sbf = reinterpret_cast<uint8_t*>(su + NT);  // block flags of the current item
  uint64_t* bars = reinterpret_cast<uint64_t*>(sbf + kMaxBlocksPerItem + 1);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7 + 2 * S);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t bar0 = smem_addr(bars);
#define BAR(i) (bar0 + 8u * uint32_t(i))
  // 0 xfull, 1 xempty, 2..3 accfull, 4..5 accempty, 6 mma_done, 7.. lfull[S], 7+S.. lempty[S]
#define LFULL(s) BAR(7 + (s))
#define LEMPTY(s) BAR(7 + S + (s))

  if (threadIdx.x == 0) {
    mbar_init(BAR(0), 1);
    mbar_init(BAR(1), 1);
    mbar_init(BAR(2), 1);
    mbar_init(BAR(3), 1);
    mbar_init(BAR(4), kEpiWarps);
    mbar_init(BAR(5), kEpiWarps);
    mbar_init(BAR(6), 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(LFULL(s), 1);
      mbar_init(LEMPTY(s), 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  constexpr uint32_t kTmemCols = 2 * ACC <= 256 ? (2 * ACC <= 128 ? 128 : 256) : 512;
  if (warp == 1) tmem_alloc(smem_addr(tmem_slot), kTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      uint32_t it = 0;
      int w = 0;
      bool ok = true;
      int x_armed = -1;  // parity of the last armed phase of xfull (-1: none)
      uint32_t ps = 0, pph = 0;  // ring stage and its phase parity
      int sid = 0;
      for (int64_t item = blockIdx.x; item < a.n_items && ok; item += gridDim.x, ++w) {
        while (sid + 1 < a.n_studies && item >= a.studies[sid + 1].item_begin) ++sid;
        const TcStudy& st = a.studies[sid];
        const int64_t local = item - st.item_begin;
        const int64_t vt = local / st.n_chunks, pc = local % st.n_chunks;
        const int64_t b0 = pc * st.blocks_per_chunk;
        const int64_t b1 = min(st.nblocks, b0 + st.blocks_per_chunk);
        const int n_pad = st.n_pad;
        const uint32_t xtile_bytes = uint32_t(NT) * n_pad * 2;
        if (!mbar_wait(BAR(1), (w & 1) ^ 1, a.status, abort_flag)) break;
        mbar_arrive_expect_tx(BAR(0), uint32_t(PIECES) * xtile_bytes);
        x_armed = w & 1;
        for (int q = 0; q < PIECES; ++q) {
          const int64_t row0 = (int64_t(q) * st.v_pad * n_pad + vt * NT * n_pad) / 256;
          tma_load_2d(smem_addr(xs + q * xtile_bytes), &st.tmX, 0, int32_t(row0), BAR(0));
        }
        const int64_t nb = b1 - b0, rot = (int64_t(blockIdx.x) * 17) % nb;
        for (int64_t kb = 0; kb < nb && ok; ++kb) {
          const int64_t b = b0 + (kb + rot) % nb;
          // One stage = KPS consecutive k-steps of the block (one box); the
          // block's last stage may hold fewer, the rest of its box is unused.
          for (int ks = 0; ks < st.ksteps; ks += KPS, ++it) {
            if (!mbar_wait(LEMPTY(ps), pph ^ 1u, a.status, abort_flag)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(LFULL(ps), stage_bytes);
            const int64_t row = b * (n_pad / 2) + ks * 8;
            tma_load_2d(smem_addr(ls + ps * stage_bytes), &st.tmL, 0, int32_t(row), LFULL(ps));
            if (++ps == uint32_t(S)) {
              ps = 0;
              pph ^= 1u;
            }
          }
        }
      }
      // Drain: every copy this thread started has completed before the CTA exits.
      const uint32_t armed = it < uint32_t(S) ? it : uint32_t(S);
      for (uint32_t k = 0; k < armed; ++k) {
        const uint32_t last = it - 1 - k;  // the most recent use of stage last % S
        mbar_wait(LFULL(last % uint32_t(S)), (last / uint32_t(S)) & 1u, a.status, abort_flag,
                  kWaitLimitNs, false);
      }
      if (x_armed >= 0)
        mbar_wait(BAR(0), uint32_t(x_armed), a.status, abort_flag, kWaitLimitNs, false);
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      uint32_t j = 0, ms = 0, mph = 0;  // block counter; ring stage and phase
      int w = 0;
      const uint32_t idesc = a.f16 ? idesc_f16_f32(128, NT) : idesc_bf16_f32(128, NT);
      const int nw = (NACC == 2 ? 2 : PIECES) * NT;
      const uint32_t idesc_w = a.f16 ? idesc_f16_f32(128, nw) : idesc_bf16_f32(128, nw);
      // L stage: k-group major (k-groups 2 KB apart, 8-row groups adjacent);
      // Xn tile: row-group major (k-groups adjacent, 8-row groups n_pad/8 x 128 B apart).
      const uint64_t adesc0 = smem_desc(smem_addr(ls), 16 * 128, 128);
      bool ok = true;
      int sid = 0;
      for (int64_t item = blockIdx.x; item < a.n_items && ok; item += gridDim.x, ++w) {
        while (sid + 1 < a.n_studies && item >= a.studies[sid + 1].item_begin) ++sid;
        const TcStudy& st = a.studies[sid];
        const int64_t local = item - st.item_begin;
        const int64_t pc = local % st.n_chunks;
        const int64_t b0 = pc * st.blocks_per_chunk;
        const int64_t b1 = min(st.nblocks, b0 + st.blocks_per_chunk);
        const int ksteps = st.ksteps;
        const uint32_t xtile_bytes = uint32_t(NT) * st.n_pad * 2;
        uint64_t bdesc0[PIECES];
#pragma unroll
        for (int q = 0; q < PIECES; ++q)
          bdesc0[q] = smem_desc(smem_addr(xs) + q * xtile_bytes, 128, uint32_t(st.n_pad / 8) * 128);
        if (!mbar_wait(BAR(0), w & 1, a.status, abort_flag)) break;
        tc_fence_after();
        for (int64_t b = b0; b < b1 && ok; ++b, ++j) {
          const uint32_t abuf = j & 1u, aph = (j >> 1) & 1u;
          if (!mbar_wait(BAR(4 + abuf), aph ^ 1u, a.status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + abuf * ACC;
          for (int ks0 = 0; ks0 < ksteps; ks0 += KPS) {
            if (!mbar_wait(LFULL(ms), mph, a.status, abort_flag)) {
              ok = false;
              break;
            }
            const int nk = ksteps - ks0 < KPS ? ksteps - ks0 : KPS;
            // descriptor start addresses advance in 16-byte units
            uint64_t adesc = adesc0 + uint64_t(ms * uint32_t(KPS) * (kStepBytes >> 4));
            for (int kk = 0; kk < nk; ++kk, adesc += kStepBytes >> 4) {
              const int ks = ks0 + kk;
              if constexpr (NACC == PIECES && NACC > 1) {
                // piece q -> columns [q NT, (q + 1) NT)
                tc_mma_f16(d, adesc, bdesc0[0] + uint64_t(ks * 16), idesc_w, ks != 0 ? 1u : 0u);
              } else if constexpr (NACC == 2) {
                // hi -> columns [0, NT), mid -> [NT, 2 NT); lo joins mid's accumulator
                tc_mma_f16(d, adesc, bdesc0[0] + uint64_t(ks * 16), idesc_w, ks != 0 ? 1u : 0u);
                tc_mma_f16(d + NT, adesc, bdesc0[2] + uint64_t(ks * 16), idesc, 1u);
              } else {
#pragma unroll
                for (int q = 0; q < PIECES; ++q)
                  tc_mma_f16(d, adesc, bdesc0[q] + uint64_t(ks * 16), idesc,
                             (ks | q) != 0 ? 1u : 0u);
              }
            }
            tc_commit(LEMPTY(ms));
            if (++ms == uint32_t(S)) {
              ms = 0;
              mph ^= 1u;
            }
          }
          if (!ok) break;
          tc_commit(BAR(2 + abuf));
        }
        if (!ok) break;
        tc_commit(BAR(1));
      }
      // Every MMA this thread issued has completed before TMEM is released.
      tc_commit(BAR(6));
      mbar_wait(BAR(6), 0, a.status, abort_flag, kWaitLimitNs, false);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    // The epilogue threads always walk the same items and blocks (so the
    // named barrier stays matched); after a failed wait they only skip work.
    const int ew = warp - 2;
    const int quad = warp & 3;
    const int colbase = (ew >> 2) * CW;
    const int etid = threadIdx.x - 64;
    uint32_t j = 0;
    bool ok = true;
    int sid = 0;
    for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
      while (sid + 1 < a.n_studies && item >= a.studies[sid + 1].item_begin) ++sid;
      const TcStudy& st = a.studies[sid];
      const int64_t local = item - st.item_begin;
      const int64_t vt = local / st.n_chunks, pc = local % st.n_chunks;
      const int64_t b0 = pc * st.blocks_per_chunk;
      const int64_t b1 = min(st.nblocks, b0 + st.blocks_per_chunk);
      const int64_t V = st.v, Pn = st.P;
      const float* u_obs = st.u_obs;
      const uint8_t* rowflag = st.rowflag;
      unsigned long long* maxkey = st.maxkey;
      const int64_t v0 = vt * NT;
      const int64_t gcol0 = v0 + colbase;
      const bool ragged_cols = v0 + NT > V;
      epi_bar();
      for (int c = etid; c < NT; c += 32 * kEpiWarps) {
        float x = INFINITY;
        if (do_reduce && v0 + c < V) {
          if constexpr (FG > 0) {
            x = u_obs[v0 + c];  // B_obs
          } else {
            x = u_obs[v0 + c] * a.uscale;  // power of two: exact
            if (TWO) x = fabsf(x);
          }
        }
        su[c] = x;
      }
      for (int64_t c = etid; c < b1 - b0; c += 32 * kEpiWarps)
        sbf[c] = (do_reduce && st.blockflag && st.blockflag[b0 + c]) || (b0 + c + 1) * 128 > Pn
                     ? 1
                     : 0;
      epi_bar();
      uint32_t c8[CW / 4];
#pragma unroll
      for (int q = 0; q < CW / 4; ++q) c8[q] = 0u;
      const int64_t nb = b1 - b0, rot = (int64_t(blockIdx.x) * 17) % nb;
      // current row maximum (possibly stale), fetched one block ahead
      unsigned long long gkey_next = 0ull;
      {
        const int64_t rowf = (b0 + rot % nb) * 128 + quad * 32 + lane;
        if (do_reduce && rowf < Pn) gkey_next = __ldcg(&maxkey[FG > 0 ? rowf / FG : rowf]);
      }
      for (int64_t kb = 0; kb < nb; ++kb, ++j) {
        // Blocks run in a per-CTA rotated order so that the CTAs do not all
        // stream the same label slab from the same L2 lines at once.
        int64_t bi = kb + rot;
        if (bi >= nb) bi -= nb;
        const int64_t b = b0 + bi;
        const uint32_t abuf = j & 1u, aph = (j >> 1) & 1u;
        const int64_t row = b * 128 + quad * 32 + lane;
        const unsigned long long gkey = gkey_next;
        if (kb + 1 < nb) {
          int64_t bn = bi + 1;
          if (bn >= nb) bn -= nb;
          const int64_t rown = (b0 + bn) * 128 + quad * 32 + lane;
          if (do_reduce && rown < Pn) gkey_next = __ldcg(&maxkey[FG > 0 ? rown / FG : rown]);
        }
        const bool ragged = ragged_cols || sbf[bi];
        if (ok && !mbar_wait(BAR(2 + abuf), aph, a.status, abort_flag)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) continue;
        tc_fence_after();
        const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + abuf * ACC + colbase;
        const bool row_ok = row < Pn;
        const bool lead = FG == 0 || (lane & (FG > 0 ? FG - 1 : 0)) == 0;
        const bool cnt_ok =
            row_ok && (FG > 0 ? lead : !(ragged && do_reduce && rowflag[row]));
        const float fr = SCALED && row_ok ? st.rowscale[row] : 1.0f;
        // F mode: this lane's view of W (rows and columns taken in xor order
        // of its position in the group, so every lane runs the same code)
        float Wp[FG > 0 ? FG : 1][FG > 0 ? FG : 1];
        if constexpr (FG > 0) {
          const int hl = lane & (FG - 1);
          const float* W = st.fmat + (row_ok ? (row / FG) * st.fstride : 0);
#pragma unroll
          for (int m = 0; m < FG; ++m)
#pragma unroll
            for (int m2 = 0; m2 < FG; ++m2)
              Wp[m][m2] = row_ok ? W[(hl ^ m) * FG + (hl ^ m2)] : 0.0f;
        }
        // Running row maximum over the chunks and, for a maximum that can beat
        // the row's current global key, its first column (found while the
        // chunk is still in registers).
        const float gval = gkey != 0ull ? unpack_key_value(gkey) : -INFINITY;
        float best = -INFINITY;
        int64_t bestcol = -1;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
          uint32_t r[CHK];
          tc_ld_cols<CHK>(taddr + c * CHK, r);
          if constexpr (NACC == 2) {
            uint32_t r2[CHK];
            tc_ld_cols<CHK>(taddr + NT + c * CHK, r2);
            tc_wait_ld();
#pragma unroll
            for (int jj = 0; jj < CHK; ++jj)
              r[jj] = __float_as_uint(__uint_as_float(r[jj]) + __uint_as_float(r2[jj]));
          } else if constexpr (NACC == 3) {
            uint32_t r2[CHK], r3[CHK];
            tc_ld_cols<CHK>(taddr + NT + c * CHK, r2);
            tc_ld_cols<CHK>(taddr + 2 * NT + c * CHK, r3);
            tc_wait_ld();
#pragma unroll
            for (int jj = 0; jj < CHK; ++jj)  // hi + (mid + lo)
              r[jj] = __float_as_uint(__uint_as_float(r[jj]) +
                                      (__uint_as_float(r2[jj]) + __uint_as_float(r3[jj])));
          } else {
            tc_wait_ld();
          }
          const int64_t g0 = gcol0 + c * CHK;
          if (WRITE && a.write_mode == 3 && row_ok) {
            // one bit per entry (u >= threshold) in rows of (V + 31) / 32 words,
            // or-ed in: the chunk's columns span at most two words
            uint32_t* bm = reinterpret_cast<uint32_t*>(st.uout) + row * ((V + 31) >> 5);
            const int sh = int(g0 & 31);
            uint32_t w0 = 0u, w1 = 0u;
#pragma unroll
            for (int jj = 0; jj < CHK; ++jj) {
              if (g0 + jj < V && __uint_as_float(r[jj]) >= a.uthr) {
                const int p = sh + jj;
                if (p < 32) w0 |= 1u << p;
                else w1 |= 1u << (p - 32);
              }
            }
            if (w0) atomicOr(bm + (g0 >> 5), w0);
            if (w1) atomicOr(bm + (g0 >> 5) + 1, w1);
          } else if (WRITE && a.write_mode && row_ok) {
            float* dst = st.uout + row * V;
#pragma unroll
            for (int jj = 0; jj < CHK; ++jj) {
              if (g0 + jj < V) {
                const float u = __uint_as_float(r[jj]) * a.inv_uscale;  // exact
                float val = u;
                if (a.write_mode == 2) {
                  const float den = 1.0f - a.k_f * u * u;
                  val = den > 0.0f ? a.ct_f * u * rsqrtf(den) : (u > 0.0f ? INFINITY : -INFINITY);
                }
                dst[g0 + jj] = val;
              }
            }
          }
          if (do_reduce) {
            uint32_t(&cc)[CHK / 4] = *reinterpret_cast<uint32_t(*)[CHK / 4]>(&c8[c * (CHK / 4)]);
            if constexpr (FG > 0) {
              // Lane hl of a group takes the chunk's columns FG j + hl: it gets
              // their u from the group's other lanes (round m: partner hl ^ m
              // sends its u of column FG j + hl), forms B = u^T W u once per
              // column, and keeps that column's maximum and count.
              const int hl = lane & (FG - 1);
              const float* sc = su + colbase + c * CHK;
#pragma unroll
              for (int j = 0; j < CHK / FG; ++j) {
                float own[FG];
#pragma unroll
                for (int m = 0; m < FG; ++m) own[m] = __uint_as_float(r[FG * j + m]) * a.inv_uscale;
                auto pick = [&](int idx) {  // own[idx] without indexing registers at run time
                  float x = own[0];
#pragma unroll
                  for (int m = 1; m < FG; ++m) x = idx == m ? own[m] : x;
                  return x;
                };
                float v[FG];
                v[0] = pick(hl);
#pragma unroll
                for (int m = 1; m < FG; ++m) v[m] = __shfl_xor_sync(0xffffffffu, pick(hl ^ m), m);
                float bq = 0.0f;
#pragma unroll
                for (int m = 0; m < FG; ++m) {
                  float t = 0.0f;
#pragma unroll
                  for (int m2 = 0; m2 < FG; ++m2) t = fmaf(Wp[m][m2], v[m2], t);
                  bq = fmaf(v[m], t, bq);
                }
                const int col = FG * j + hl;
                const bool valid = row_ok && g0 + col < V;
                if (valid && bq > best) {
                  best = bq;
                  bestcol = g0 + col;
                }
                if (valid && bq >= sc[col]) {
                  if constexpr (FG == 2)
                    cc[j >> 1] += 1u << (8 * ((2 * j & 3) + hl));
                  else
                    cc[j] += 1u << (8 * hl);
                }
              }
            } else {
              const float cm =
                  ragged ? cols_reduce<CHK, TWO, true, SCALED>(r, su + colbase + c * CHK, g0, V,
                                                               row_ok, cnt_ok, cc, fr)
                         : cols_reduce<CHK, TWO, false, SCALED>(r, su + colbase + c * CHK, g0,
                                                                V, true, true, cc, fr);
              const bool cand = row_ok && cm > best && cm >= gval && cm > -INFINITY;
              if (cm > best) {
                best = cm;
                bestcol = -1;
              }
              if (__any_sync(0xffffffffu, cand) && cand) {
                int jj_best = -1;
#pragma unroll
                for (int jj = CHK - 1; jj >= 0; --jj) {
                  float sv = __uint_as_float(r[jj]);
                  if (TWO) sv = fabsf(sv);
                  if (sv == cm && g0 + jj < V) jj_best = jj;
                }
                bestcol = jj_best >= 0 ? g0 + jj_best : -1;
              }
            }
          }
        }
        if constexpr (FG > 0) {
          // the group's best (largest B, smallest voxel on ties) to its first lane
#pragma unroll
          for (int o = FG / 2; o > 0; o >>= 1) {
            const float ob = __shfl_xor_sync(0xffffffffu, best, o);
            const int64_t oc = __shfl_xor_sync(0xffffffffu, bestcol, o);
            if (oc >= 0 && (bestcol < 0 || ob > best || (ob == best && oc < bestcol))) {
              best = ob;
              bestcol = oc;
            }
          }
          if (!lead) bestcol = -1;
        }
        if (do_reduce && bestcol >= 0) {
          const unsigned long long key = pack_key(best, uint32_t(bestcol));
          if (key > gkey) atomicMax(&maxkey[FG > 0 ? row / FG : row], key);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(BAR(4 + abuf));
      }
      if (ok && do_reduce) flush_counts8<CW>(c8, lane, gcol0, V, st.cnt);
    }
  }
#undef LFULL
#undef LEMPTY
#undef BAR
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
int smem_bytes(int NT, int n_pad, int pieces, int stages, int kps) {
  return pieces * NT * n_pad * 2 + stages * kps * kStepBytes + NT * 4 + (kMaxBlocksPerItem + 1) +
         (7 + 2 * stages) * 8 + 16;
}

int num_sms(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

template <int NT, bool TWO>
pt_status launch_nt(pt_ctx* ctx, const TcArgs& a, int pieces, int grid, int smem) {
  auto kern = a.write_mode ? (pieces == 2 ? tc_contract_kernel<NT, TWO, 2, true>
                                          : tc_contract_kernel<NT, TWO, 3, true>)
              : a.scaled   ? (pieces == 2 ? tc_contract_kernel<NT, TWO, 2, false, true>
                                          : tc_contract_kernel<NT, TWO, 3, false, true>)
                           : (pieces == 2 ? tc_contract_kernel<NT, TWO, 2, false>
                                          : tc_contract_kernel<NT, TWO, 3, false>);
  PT_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  if (a.do_reduce) prof_begin(ctx);
  kern<<<grid, kThreads, smem, ctx->stream>>>(a);
  if (a.do_reduce) prof_end(ctx);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

// F of a g-group factor (reduce only, one-sided).
template <int NT, int FG>
pt_status launch_f(pt_ctx* ctx, const TcArgs& a, int pieces, int grid, int smem) {
  auto kern = pieces == 2 ? tc_contract_kernel<NT, false, 2, false, false, FG>
                          : tc_contract_kernel<NT, false, 3, false, false, FG>;
  PT_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  kern<<<grid, kThreads, smem, ctx->stream>>>(a);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

template <int FG>
pt_status launch_f_nt(pt_ctx* ctx, const TcArgs& a, int NT, int pieces, int grid, int smem) {
  if (NT == 256) return launch_f<256, FG>(ctx, a, pieces, grid, smem);
  if (NT == 128) return launch_f<128, FG>(ctx, a, pieces, grid, smem);
  if (NT == 96) return launch_f<96, FG>(ctx, a, pieces, grid, smem);
  return launch_f<64, FG>(ctx, a, pieces, grid, smem);
}

// Label-ring stages of kps k-steps each that fit beside the resident data
// tile of NT voxels (0 when fewer than 2 fit or the tile exceeds one TMA box).
int max_stages_fit(int NT, int n_pad, int pieces, int kps) {
  if (int64_t(NT) * n_pad / 256 > 256) return 0;
  int s = kMaxStages;
  while (s >= 2 && smem_bytes(NT, n_pad, pieces, s, kps) > kSmemLimit - 1024) --s;
  return s >= 2 ? s : 0;
}

// Largest voxel tile NT whose resident data tile leaves room for a label ring
// of at least 8 one-k-step stages that also covers at least 2,048 MMA columns
// x k-steps (stages x pieces x NT: about 1,000 cycles of MMA work in flight,
// which the label loads' L2 latency needs), else the largest that leaves at
// least 4 stages. NT = 96 is taken with two data pieces only (one MMA of width
// 192 per k-step; with three its lo piece would take a separate MMA of width
// 96, slower than the 64-voxel tile's single MMA of width 192). Measured on
// 10,000 relabellings: n = 392 FP16x2, 96 voxels 5.04 ms against 128 voxels
// (6 stages) 6.85 ms; n = 200 FP16x2, 128 voxels 3.13 ms against 256 voxels
// (4 stages) 3.30 ms; n = 300 BF16x3, 64 voxels 5.89 ms against 96 voxels
// 6.38 ms.
bool choose_tile(int n_pad, int pieces, int* NT) {
  for (int cand : {256, 128, 96, 64}) {
    if (cand == 96 && pieces != 2) continue;
    const int s = max_stages_fit(cand, n_pad, pieces, 1);
    if (s >= 8 && s * pieces * cand >= 2048) {
      *NT = cand;
      return true;
    }
  }
  for (int cand : {256, 128, 96, 64}) {
    if (cand == 96 && pieces != 2) continue;
    if (max_stages_fit(cand, n_pad, pieces, 1) >= 4) {
      *NT = cand;
      return true;
    }
  }
  return false;
}

// Work split of one study into items (voxel tile x block range) and its
// descriptor; target_items spreads small studies over more block ranges.
bool fill_study(pt_ctx* c, const void* Lb, int64_t P, int NT, int kps, int64_t target_items,
                int64_t item_begin, const float* u_obs, unsigned long long* maxkey, uint32_t* cnt,
                float* uout, TcStudy* st) {
  memset(st, 0, sizeof(*st));
  st->n_pad = c->n_pad;
  st->ksteps = c->n_pad / 16;
  st->P = P;
  st->v = c->v_valid;
  st->v_pad = c->v_pad;
  st->nblocks = (P + 127) / 128;
  const int64_t n_vtiles = (st->v + NT - 1) / NT;
  int64_t chunks = (st->nblocks + kMaxBlocksPerItem - 1) / kMaxBlocksPerItem;
  if (n_vtiles * chunks < target_items) {
    const int64_t want = (target_items + n_vtiles - 1) / n_vtiles;
    if (want > chunks) chunks = want;
  }
  if (chunks > st->nblocks) chunks = st->nblocks;
  if (chunks < 1) chunks = 1;
  st->blocks_per_chunk = (st->nblocks + chunks - 1) / chunks;
  st->n_chunks = (st->nblocks + st->blocks_per_chunk - 1) / st->blocks_per_chunk;
  st->item_begin = item_begin;
  st->u_obs = u_obs;
  st->rowflag = c->rowflag.as<uint8_t>();
  st->blockflag = c->blockflag.as<uint8_t>();
  st->maxkey = maxkey;
  st->cnt = cnt;
  st->uout = uout;
  st->rowscale = c->glm_q1 ? c->rowscale.as<float>() : nullptr;
  const int64_t P_pad = st->nblocks * 128;
  // Label box: kps k-steps of one 128-row block (8 view rows per k-step); a
  // box that runs past the last block reads zero fill.
  return make_map(&st->tmL, Lb, uint64_t(P_pad) * c->n_pad / 256, uint32_t(8 * kps)) &&
         make_map(&st->tmX, c->Xnb.p, uint64_t(3) * c->v_pad * c->n_pad / 256,
                  uint32_t(NT * c->n_pad / 256));
}

// Launch the fused kernel over n studies sharing tile NT, ring shape and piece
// count. descs: device copy of the descriptors (filled by the caller).
pt_status launch_studies(pt_ctx* ctx, const TcStudy* descs, int n, int64_t n_items, int NT,
                         int stages, int kps, int pieces, int n_pad_max, int do_reduce,
                         int write_mode, int two_sided, float kf, float ctf, int scaled = 0,
                         int f16 = 0, int fg = 0, float uthr = 0.0f) {
  if (scaled && (write_mode || !do_reduce)) {
    set_error(ctx, "covariate-adjusted statistic: reduce-only launches");
    return PT_ERR_UNSUPPORTED;
  }
  const int fit = max_stages_fit(NT, n_pad_max, pieces, kps);
  if (!fit || stages < 2 || stages > fit) {
    set_error(ctx, "tensor-core path: n too large for the resident data tile");
    return PT_ERR_UNSUPPORTED;
  }
  TcArgs a;
  a.studies = descs;
  a.n_studies = n;
  a.stages = stages;
  a.kps = kps;
  a.n_pad_max = n_pad_max;
  a.n_items = n_items;
  a.do_reduce = do_reduce;
  a.write_mode = write_mode;
  a.k_f = kf;
  a.ct_f = ctf;
  a.scaled = scaled;
  a.f16 = f16;
  a.uscale = f16 ? kF16Scale : 1.0f;
  a.inv_uscale = f16 ? 1.0f / kF16Scale : 1.0f;
  a.uthr = uthr * a.uscale;  // power of two: exact
  a.status = ctx->status.as<uint32_t>();
  const int sms = num_sms(ctx->device);
  const int grid = int(n_items < sms ? n_items : sms);
  const int smem = smem_bytes(NT, n_pad_max, pieces, stages, kps);
  if (fg) {
    if (two_sided || write_mode || !do_reduce || scaled) {
      set_error(ctx, "F mode: one-sided reduce-only launches");
      return PT_ERR_UNSUPPORTED;
    }
    return fg == 2 ? launch_f_nt<2>(ctx, a, NT, pieces, grid, smem)
                   : launch_f_nt<4>(ctx, a, NT, pieces, grid, smem);
  }
  if (two_sided) {
    if (NT == 256) return launch_nt<256, true>(ctx, a, pieces, grid, smem);
    if (NT == 128) return launch_nt<128, true>(ctx, a, pieces, grid, smem);
    if (NT == 96) return launch_nt<96, true>(ctx, a, pieces, grid, smem);
    return launch_nt<64, true>(ctx, a, pieces, grid, smem);
  }
  if (NT == 256) return launch_nt<256, false>(ctx, a, pieces, grid, smem);
  if (NT == 128) return launch_nt<128, false>(ctx, a, pieces, grid, smem);
  if (NT == 96) return launch_nt<96, false>(ctx, a, pieces, grid, smem);
  return launch_nt<64, false>(ctx, a, pieces, grid, smem);
}

// One study with an explicit launch configuration (already validated).
pt_status tc_launch_cfg(pt_ctx* ctx, const void* Lb, int64_t P, int pieces, int do_reduce,
                        int write_mode, int two_sided, const float* u_obs,
                        unsigned long long* maxkey, uint32_t* cnt, float* uout,
                        const pt_tc_config& cfg, int f16, float uthr = 0.0f) {
  const int NT = cfg.voxel_tile;
  TcStudy st;
  if (!fill_study(ctx, Lb, P, NT, cfg.ksteps_per_stage,
                  int64_t(cfg.items_per_sm) * num_sms(ctx->device), 0, u_obs, maxkey, cnt, uout,
                  &st)) {
    set_error(ctx, "cuTensorMapEncodeTiled failed");
    return PT_ERR_CUDA;
  }
  if (!ctx->tcdesc.ensure(sizeof(TcStudy))) {
    set_error(ctx, "out of device memory (descriptor)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->tcdesc.p, &st, sizeof(TcStudy), cudaMemcpyHostToDevice,
                                   ctx->stream));
  const int64_t items = ((st.v + NT - 1) / NT) * st.n_chunks;
  return launch_studies(ctx, ctx->tcdesc.as<TcStudy>(), 1, items, NT, cfg.stages,
                        cfg.ksteps_per_stage, pieces, ctx->n_pad, do_reduce, write_mode,
                        two_sided, float(ctx->k), float(ctx->c_t),
                        ctx->glm_q1 && do_reduce && !write_mode ? 1 : 0, f16, 0, uthr);
}

pt_status tc_launch(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int do_reduce,
                    int write_mode, int two_sided, const float* u_obs,
                    unsigned long long* maxkey, uint32_t* cnt, float* uout, float uthr = 0.0f) {
  const int pieces = prec_pieces(precision);
  pt_tc_config cfg;
  if (!tc_default_config(ctx->n_pad, pieces, &cfg)) {
    set_error(ctx, "tensor-core path: n too large for the resident data tile");
    return PT_ERR_UNSUPPORTED;
  }
  // The reduce-only launch (NaivePT) takes a tuned configuration when one is
  // recorded for this shape; row-writing launches keep the default.
  if (do_reduce && !write_mode) tune_find(ctx->n_pad, precision, two_sided, ctx->v_valid, P, &cfg);
  return tc_launch_cfg(ctx, Lb, P, pieces, do_reduce, write_mode, two_sided, u_obs, maxkey, cnt,
                       uout, cfg, precision == PT_PREC_FP16X2 ? 1 : 0, uthr);
}

}  // namespace

// The F of a g-group factor fused into the contraction: `rows` label rows of
// groups (FG per relabelling), B_obs per compact voxel, W per relabelling
// (stride fstride), keys per relabelling, counts B >= B_obs per voxel.
pt_status tc_f_reduce(pt_ctx* ctx, const void* Lb, int64_t rows, int precision, int fg,
                      const float* b_obs, const float* fmat, int64_t fstride,
                      unsigned long long* keys, uint32_t* cnt) {
  if (fg != 2 && fg != 4) {
    set_error(ctx, "F mode: 2 or 4 rows per relabelling");
    return PT_ERR_INVALID;
  }
  const int pieces = prec_pieces(precision);
  pt_tc_config cfg;
  if (!tc_default_config(ctx->n_pad, pieces, &cfg)) {
    set_error(ctx, "tensor-core path: n too large for the resident data tile");
    return PT_ERR_UNSUPPORTED;
  }
  const int NT = cfg.voxel_tile;
  TcStudy st;
  if (!fill_study(ctx, Lb, rows, NT, cfg.ksteps_per_stage,
                  int64_t(cfg.items_per_sm) * num_sms(ctx->device), 0, b_obs, keys, cnt, nullptr,
                  &st)) {
    set_error(ctx, "cuTensorMapEncodeTiled failed");
    return PT_ERR_CUDA;
  }
  st.rowflag = nullptr;
  st.blockflag = nullptr;
  st.rowscale = nullptr;
  st.fmat = fmat;
  st.fstride = fstride;
  if (!ctx->tcdesc.ensure(sizeof(TcStudy))) {
    set_error(ctx, "out of device memory (descriptor)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->tcdesc.p, &st, sizeof(TcStudy), cudaMemcpyHostToDevice,
                                   ctx->stream));
  const int64_t items = ((st.v + NT - 1) / NT) * st.n_chunks;
  return launch_studies(ctx, ctx->tcdesc.as<TcStudy>(), 1, items, NT, cfg.stages,
                        cfg.ksteps_per_stage, pieces, ctx->n_pad, 1, 0, 0, float(ctx->k),
                        float(ctx->c_t), 0, precision == PT_PREC_FP16X2 ? 1 : 0, fg);
}


pt_status tc_supported(pt_ctx* ctx) {
  int major = 0, minor = 0;
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, ctx->device);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, ctx->device);
  if (major != 10 || minor != 3) {
    set_error(ctx, "tensor-core path needs an sm_103 (GB300) device; got sm_" +
                       std::to_string(major) + std::to_string(minor));
    return PT_ERR_UNSUPPORTED;
  }
  if (!encode_fn()) {
    set_error(ctx, "cuTensorMapEncodeTiled entry point unavailable");
    return PT_ERR_UNSUPPORTED;
  }
  return PT_OK;
}

pt_status tc_reduce(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int two_sided,
                    const float* u_obs, unsigned long long* maxkey, uint32_t* cnt) {
  return tc_launch(ctx, Lb, P, precision, 1, 0, two_sided, u_obs, maxkey, cnt, nullptr);
}

pt_status tc_rows(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int write_mode,
                  float* out, int do_reduce, int two_sided, const float* u_obs,
                  unsigned long long* maxkey, uint32_t* cnt, float uthr) {
  if (write_mode == 3 && (do_reduce || two_sided)) {
    set_error(ctx, "bit rows: one-sided, without the reduction");
    return PT_ERR_INVALID;
  }
  return tc_launch(ctx, Lb, P, precision, do_reduce, write_mode, two_sided, u_obs, maxkey, cnt,
                   out, uthr);
}

// ---------------------------------------------------------------------------
// Several prepared studies in one persistent launch per tile class
// ---------------------------------------------------------------------------
pt_status tc_batch_plan(pt_ctx* lead, pt_ctx* const* ctxs, const int64_t* P, int n,
                        const pt_naive_opts& o, Buf& descbuf, std::vector<char>& host_desc,
                        std::vector<TcGroup>& groups) {
  const int pieces = prec_pieces(o.precision);
  std::vector<pt_tc_config> cfg(n);
  for (int i = 0; i < n; ++i) {
    if (!tc_default_config(ctxs[i]->n_pad, pieces, &cfg[i])) {
      set_error(lead, "tensor-core path: a study's n is too large for the resident data tile");
      return PT_ERR_UNSUPPORTED;
    }
    tune_find(ctxs[i]->n_pad, o.precision, o.two_sided, ctxs[i]->v_valid, P[i], &cfg[i]);
  }
  host_desc.assign(sizeof(TcStudy) * size_t(n), 0);
  TcStudy* hd = reinterpret_cast<TcStudy*>(host_desc.data());
  groups.clear();
  // One launch per (voxel tile, k-steps per stage) among the studies: the ring
  // is as deep (in k-steps) as its members ask for and fits the largest n of
  // the launch, and every study's blocks are split so that the launch holds
  // about items_per_sm work items per SM, each study by its share of voxels.
  const int sms = num_sms(lead->device);
  int filled = 0;
  for (int NT : {256, 128, 96, 64}) {
    for (int kps : {8, 4, 2, 1}) {
      TcGroup g{NT, filled, 0, 16, 0, 0, kps};
      int ring = 1 << 30, items_per_sm = 1;
      int64_t vsum = 0;
      for (int i = 0; i < n; ++i) {
        if (cfg[i].voxel_tile != NT || cfg[i].ksteps_per_stage != kps || ctxs[i]->v_valid < 1)
          continue;
        ring = std::min(ring, cfg[i].stages * kps);
        items_per_sm = std::max(items_per_sm, cfg[i].items_per_sm);
        g.n_pad_max = std::max(g.n_pad_max, ctxs[i]->n_pad);
        vsum += ctxs[i]->v_valid;
      }
      if (!vsum) continue;
      const int fit = max_stages_fit(NT, g.n_pad_max, pieces, kps);
      g.stages = std::max(2, std::min(fit, ring / kps));
      const double want = double(items_per_sm) * sms;
      for (int i = 0; i < n; ++i) {
        pt_ctx* c = ctxs[i];
        if (cfg[i].voxel_tile != NT || cfg[i].ksteps_per_stage != kps || c->v_valid < 1)
          continue;  // another launch, or nothing to contract
        const int64_t target = int64_t(std::ceil(want * double(c->v_valid) / double(vsum)));
        if (!fill_study(c, c->labels.p, P[i], NT, kps, target, g.items, c->u_obs.as<float>(),
                        c->maxkey.as<unsigned long long>(), c->cnt.as<uint32_t>(), nullptr,
                        &hd[filled])) {
          set_error(lead, "cuTensorMapEncodeTiled failed");
          return PT_ERR_CUDA;
        }
        g.items += ((hd[filled].v + NT - 1) / NT) * hd[filled].n_chunks;
        ++filled;
        ++g.count;
      }
      groups.push_back(g);
    }
  }
  if (!filled) return PT_OK;
  if (!descbuf.ensure(sizeof(TcStudy) * size_t(filled))) {
    set_error(lead, "out of device memory (descriptors)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(lead, cudaMemcpyAsync(descbuf.p, hd, sizeof(TcStudy) * size_t(filled),
                                    cudaMemcpyHostToDevice, lead->stream));
  PT_CUDA_TRY(lead, cudaStreamSynchronize(lead->stream));
  return PT_OK;
}

pt_status tc_batch_launch(pt_ctx* lead, const Buf& descbuf, const std::vector<TcGroup>& groups,
                          int precision, int two_sided) {
  const int pieces = prec_pieces(precision);
  for (const TcGroup& g : groups) {
    pt_status s = launch_studies(lead, static_cast<const TcStudy*>(descbuf.p) + g.first, g.count,
                                 g.items, g.NT, g.stages, g.kps, pieces, g.n_pad_max, 1, 0,
                                 two_sided, 0.0f, 0.0f, 0, precision == PT_PREC_FP16X2 ? 1 : 0);
    if (s != PT_OK) return s;
  }
  return PT_OK;
}

// ---------------------------------------------------------------------------
// Launch configurations and the autotuner's timing loop
// ---------------------------------------------------------------------------
int tc_max_stages(int NT, int n_pad, int pieces, int kps) {
  return max_stages_fit(NT, n_pad, pieces, kps);
}

bool tc_default_config(int n_pad, int pieces, pt_tc_config* out) {
  int NT = 0;
  if (!choose_tile(n_pad, pieces, &NT)) return false;
  // Fewest ring waits: the largest stage (in k-steps) of which two fit, and a
  // ring of about 16 k-steps.
  int kps = 1;
  for (int k : {8, 4, 2})
    if (max_stages_fit(NT, n_pad, pieces, k) >= 2) {
      kps = k;
      break;
    }
  const int fit = max_stages_fit(NT, n_pad, pieces, kps);
  out->voxel_tile = NT;
  out->ksteps_per_stage = kps;
  out->stages = std::max(2, std::min(fit, 16 / kps));
  out->items_per_sm = kDefaultItemsPerSm;
  return true;
}

// The voxel tile fixes how the data pieces' partial sums are combined (one,
// two or three accumulators), so a configuration keeps the default tile for
// its n: the outputs never depend on the configuration.
bool tc_config_valid(const pt_tc_config& c, int n_pad, int pieces) {
  pt_tc_config d;
  if (!tc_default_config(n_pad, pieces, &d)) return false;
  if (c.voxel_tile != d.voxel_tile) return false;
  const int k = c.ksteps_per_stage;
  if (k != 1 && k != 2 && k != 4 && k != 8) return false;
  const int fit = max_stages_fit(c.voxel_tile, n_pad, pieces, k);
  return fit >= 2 && c.stages >= 2 && c.stages <= fit && c.items_per_sm >= 1 &&
         c.items_per_sm <= 64;
}

// Times the reduce-only launch of every candidate configuration on this
// problem (labels already built, operand pieces ready): each candidate runs
// twice after the workspaces are cleared, and its faster run counts.
pt_status tc_autotune(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int two_sided,
                      pt_tc_config* best, double* best_ms, std::vector<TcTrial>* trials) {
  const int pieces = prec_pieces(precision);
  std::vector<pt_tc_config> cand;
  pt_tc_config d;
  if (!tc_default_config(ctx->n_pad, pieces, &d)) {
    set_error(ctx, "tensor-core path: n too large for the resident data tile");
    return PT_ERR_UNSUPPORTED;
  }
  for (int NT : {d.voxel_tile}) {
    for (int kps : {1, 2, 4, 8}) {
      const int fit = max_stages_fit(NT, ctx->n_pad, pieces, kps);
      for (int ring : {8, 16, 32}) {  // ring depth in k-steps
        const int st = std::min(fit, std::max(2, ring / kps));
        const pt_tc_config c{NT, st, kps, kDefaultItemsPerSm};
        if (!tc_config_valid(c, ctx->n_pad, pieces)) continue;
        bool dup = false;
        for (const auto& e : cand)
          dup = dup || (e.voxel_tile == NT && e.stages == st && e.ksteps_per_stage == kps);
        if (!dup) cand.push_back(c);
      }
    }
  }
  if (cand.empty()) {
    set_error(ctx, "tensor-core path: n too large for the resident data tile");
    return PT_ERR_UNSUPPORTED;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  PT_CUDA_TRY(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    set_error(ctx, "cudaEventCreate failed");
    return PT_ERR_CUDA;
  }
  const bool prof = ctx->profile;
  ctx->profile = false;
  pt_status s = PT_OK;
  double bms = 0.0;
  pt_tc_config b{};
  auto time_one = [&](const pt_tc_config& c, double* ms_out) -> pt_status {
    double bestrun = 0.0;
    for (int rep = 0; rep < 2; ++rep) {
      PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->maxkey.p, 0, sizeof(unsigned long long) * P,
                                       ctx->stream));
      PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cnt.p, 0, sizeof(uint32_t) * (ctx->v_valid + 1),
                                       ctx->stream));
      PT_CUDA_TRY(ctx, cudaEventRecord(e0, ctx->stream));
      pt_status r = tc_launch_cfg(ctx, Lb, P, pieces, 1, 0, two_sided, ctx->u_obs.as<float>(),
                                  ctx->maxkey.as<unsigned long long>(), ctx->cnt.as<uint32_t>(),
                                  nullptr, c, precision == PT_PREC_FP16X2 ? 1 : 0);
      if (r != PT_OK) return r;
      PT_CUDA_TRY(ctx, cudaEventRecord(e1, ctx->stream));
      PT_CUDA_TRY(ctx, cudaEventSynchronize(e1));
      float ms = 0.0f;
      PT_CUDA_TRY(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 0 || ms < bestrun) bestrun = ms;
    }
    *ms_out = bestrun;
    if (trials) trials->push_back({c, bestrun});
    return PT_OK;
  };
  // Phase 1: tile and ring shape at the default block split.
  for (size_t i = 0; i < cand.size() && s == PT_OK; ++i) {
    double ms = 0.0;
    s = time_one(cand[i], &ms);
    if (s == PT_OK && (i == 0 || ms < bms)) {
      bms = ms;
      b = cand[i];
    }
  }
  // Phase 2: how finely the relabelling blocks of a voxel tile are split.
  for (int items : {1, 2, 4, 8}) {
    if (s != PT_OK) break;
    if (items == kDefaultItemsPerSm) continue;
    pt_tc_config c = b;
    c.items_per_sm = items;
    double ms = 0.0;
    s = time_one(c, &ms);
    if (s == PT_OK && ms < bms) {
      bms = ms;
      b = c;
    }
  }
  ctx->profile = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != PT_OK) return s;
  *best = b;
  *best_ms = bms;
  return PT_OK;
}

}  // namespace pt
