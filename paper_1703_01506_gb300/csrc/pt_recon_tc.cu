// Reconstruction with noise and row maxima on the tensor cores (Alg. 2
// recovery; Sec. 4.2): for each row i of W (a relabelling's weights) and
// voxel j,  val_ij = (U w_i)_j + sigma z_ij,  z_ij the Philox/Box-Muller normal
// of (tag, voxel j, relabelling label0 + i), and per row the largest val with
// its first voxel, merged into packed keys.
//
// Operands: W (rows x RP) and U (V x RP) FP32, each split into BF16 pieces
// hi + mid + lo (x - hi and x - hi - mid are exact in FP32), stored as 8 x 8
// core matrices (K-major, no swizzle) so that a 128-row (or NT-voxel) tile is
// one contiguous block for a TMA copy. Six products hh, hm, mh, hl, lh, mm
// accumulate in FP32 (the dropped ml, lm, ll are below 2^-24 relative).
//
// Roles (one CTA per SM, persistent over items = (voxel chunk, 128-row block),
// voxel chunk major so that the CTAs running at once share U tiles in L2):
//   warp 0      TMA: the item's W pieces once, then U tiles through an S-stage ring
//   warp 1      MMA: 6 x Kp/16 tcgen05.mma per tile into one of two TMEM accumulators
//   warps 2..17 epilogue: a thread owns one row (TMEM lane) and NT/4 columns;
//               per 4 voxels one Philox call; a Box-Muller pair is evaluated only
//               when its radius can lift the entry to the thread's running
//               maximum M (test on the integer word, exact, below), so almost
//               every entry costs a quarter of a Philox call and a compare.
//
// Skip test. An entry of a pair can reach M only if sigma r >= M - mu, with
// r = sqrt(-2 ln u1) and u1 = (x + 1) 2^-32: i.e. only if
// x + 1 <= 2^32 exp(-D^2 / 2), D = (M - mu) / sigma. The kernel lowers M - mu
// by an absolute guard and raises the word threshold by a relative one, both
// larger than the rounding of u1, logf, sqrtf, sincospif and the final fmaf,
// so every skipped entry evaluates (in this kernel's own arithmetic) strictly
// below M and cannot be a row maximum or tie one.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "pt_draws.h"
#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {
namespace {

constexpr int kEpiWarps = 16;
constexpr int kThreads = 64 + 32 * kEpiWarps;  // 576
constexpr int kSmemLimit = 232448;
constexpr int kNumProducts = 6;
__constant__ uint8_t kProdA[kNumProducts] = {0, 0, 1, 0, 2, 1};  // piece of W
__constant__ uint8_t kProdB[kNumProducts] = {0, 1, 0, 2, 0, 1};  // piece of U

struct ReconTcArgs {
  CUtensorMap tmW;  // W pieces, [3 * rows_pad * Kp / 256][256] BF16 view
  CUtensorMap tmU;  // U pieces, [3 * V_pad * Kp / 256][256] BF16 view
  int64_t rows, rows_pad, V, V_pad;
  int Kp, stages;
  int64_t label0;
  float sigma, inv_sigma;  // inv_sigma = 0: no skipping (sigma <= 0)
  uint32_t tag, k0, k1;
  int64_t n_rb, vtiles, tiles_per_chunk, n_items;
  unsigned long long* maxkey;
  uint32_t* status;
};

// Word threshold of the skip test for the quad (gap = M - max mu, in value
// units): a pair is evaluated iff float(first word) <= thr.
__device__ __forceinline__ float pair_threshold(float gap, float inv_sigma) {
  const float d = gap * inv_sigma;
  if (!(d > 0.0f)) return 4294967296.0f;  // every word
  // 2^32 exp(-d^2/2) = 2^(32 - d^2 / (2 ln 2)), raised by 2^-10 relative + 2
  const float e = fmaf(-0.72134752f * d, d, 32.0f);
  return fmaf(exp2f(e), 1.0009765625f, 2.0f);
}

struct RowBest {
  float best = -INFINITY;
  uint32_t col = 0xffffffffu;
  float M = -INFINITY;
  __device__ __forceinline__ void take(float v, uint32_t c) {
    if (v > best || (v == best && c < col)) {
      best = v;
      col = c;
    }
    M = fmaxf(M, v);
  }
};

template <int NT>
__global__ void __launch_bounds__(kThreads, 1) recon_tc_kernel(const __grid_constant__ ReconTcArgs a) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int CW = NT / 4;  // columns per epilogue thread
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S = a.stages;
  const int Kp = a.Kp;
  const uint32_t abytes = uint32_t(128) * Kp * 2;  // one W piece tile
  const uint32_t bbytes = uint32_t(NT) * Kp * 2;   // one U piece tile
  uint8_t* as = smem;
  uint8_t* bs = smem + 3 * abytes;
  uint64_t* bars = reinterpret_cast<uint64_t*>(bs + size_t(S) * 3 * bbytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 7 + 2 * S);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const uint32_t bar0 = smem_addr(bars);
#define BAR(i) (bar0 + 8u * uint32_t(i))
  // 0 afull, 1 aempty, 2..3 accfull, 4..5 accempty, 6 mma_done, 7.. bfull[S], 7+S.. bempty[S]
#define BFULL(s) BAR(7 + (s))
#define BEMPTY(s) BAR(7 + S + (s))
  if (threadIdx.x == 0) {
    mbar_init(BAR(0), 1);
    mbar_init(BAR(1), 1);
    mbar_init(BAR(2), 1);
    mbar_init(BAR(3), 1);
    mbar_init(BAR(4), kEpiWarps);
    mbar_init(BAR(5), kEpiWarps);
    mbar_init(BAR(6), 1);
    for (int s = 0; s < S; ++s) {
      mbar_init(BFULL(s), 1);
      mbar_init(BEMPTY(s), 1);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 1) tmem_alloc(smem_addr(tmem_slot), 2 * NT);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      uint32_t it = 0, ps = 0, pph = 0;
      int w = 0, a_armed = -1;
      bool ok = true;
      for (int64_t item = blockIdx.x; item < a.n_items && ok; item += gridDim.x, ++w) {
        const int64_t vc = item / a.n_rb, rb = item % a.n_rb;
        const int64_t t0 = vc * a.tiles_per_chunk;
        const int64_t t1 = min(a.vtiles, t0 + a.tiles_per_chunk);
        if (!mbar_wait(BAR(1), (w & 1) ^ 1, a.status, abort_flag)) break;
        mbar_arrive_expect_tx(BAR(0), 3 * abytes);
        a_armed = w & 1;
        for (int q = 0; q < 3; ++q) {
          const int64_t row0 = (int64_t(q) * a.rows_pad + rb * 128) * Kp / 256;
          tma_load_2d(smem_addr(as + q * abytes), &a.tmW, 0, int32_t(row0), BAR(0));
        }
        for (int64_t t = t0; t < t1; ++t, ++it) {
          if (!mbar_wait(BEMPTY(ps), pph ^ 1u, a.status, abort_flag)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(BFULL(ps), 3 * bbytes);
          uint8_t* dst = bs + size_t(ps) * 3 * bbytes;
          for (int q = 0; q < 3; ++q) {
            const int64_t row0 = (int64_t(q) * a.V_pad + t * NT) * Kp / 256;
            tma_load_2d(smem_addr(dst + q * bbytes), &a.tmU, 0, int32_t(row0), BFULL(ps));
          }
          if (++ps == uint32_t(S)) {
            ps = 0;
            pph ^= 1u;
          }
        }
      }
      // Drain: every copy this thread started has completed before the CTA exits.
      const uint32_t armed = it < uint32_t(S) ? it : uint32_t(S);
      for (uint32_t k = 0; k < armed; ++k) {
        const uint32_t last = it - 1 - k;
        mbar_wait(BFULL(last % uint32_t(S)), (last / uint32_t(S)) & 1u, a.status, abort_flag,
                  kWaitLimitNs, false);
      }
      if (a_armed >= 0)
        mbar_wait(BAR(0), uint32_t(a_armed), a.status, abort_flag, kWaitLimitNs, false);
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      uint32_t j = 0, ms = 0, mph = 0;
      int w = 0;
      bool ok = true;
      const uint32_t idesc = idesc_bf16_f32(128, NT);
      const uint32_t sbo = uint32_t(Kp) * 16;  // 8-row groups; K-adjacent core matrices 128 B apart
      uint64_t adesc[3];
      for (int q = 0; q < 3; ++q) adesc[q] = smem_desc(smem_addr(as + q * abytes), 128, sbo);
      const int ksteps = Kp / 16;
      for (int64_t item = blockIdx.x; item < a.n_items && ok; item += gridDim.x, ++w) {
        const int64_t vc = item / a.n_rb;
        const int64_t t0 = vc * a.tiles_per_chunk;
        const int64_t t1 = min(a.vtiles, t0 + a.tiles_per_chunk);
        if (!mbar_wait(BAR(0), w & 1, a.status, abort_flag)) break;
        tc_fence_after();
        for (int64_t t = t0; t < t1 && ok; ++t, ++j) {
          const uint32_t abuf = j & 1u, aph = (j >> 1) & 1u;
          if (!mbar_wait(BAR(4 + abuf), aph ^ 1u, a.status, abort_flag) ||
              !mbar_wait(BFULL(ms), mph, a.status, abort_flag)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t bst = smem_addr(bs + size_t(ms) * 3 * bbytes);
          const uint32_t d = tmem + abuf * NT;
          for (int pr = 0; pr < kNumProducts; ++pr) {
            const uint64_t ad = adesc[kProdA[pr]];
            const uint64_t bd = smem_desc(bst + kProdB[pr] * bbytes, 128, sbo);
            for (int ks = 0; ks < ksteps; ++ks)
              tc_mma_f16(d, ad + uint64_t(ks * 16), bd + uint64_t(ks * 16), idesc,
                         (pr | ks) != 0 ? 1u : 0u);
          }
          tc_commit(BEMPTY(ms));
          if (++ms == uint32_t(S)) {
            ms = 0;
            mph ^= 1u;
          }
          tc_commit(BAR(2 + abuf));
        }
        if (!ok) break;
        tc_commit(BAR(1));
      }
      tc_commit(BAR(6));
      mbar_wait(BAR(6), 0, a.status, abort_flag, kWaitLimitNs, false);
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int ew = warp - 2;
    const int quad = warp & 3;  // TMEM lane quadrant this warp may read
    const int colbase = (ew >> 2) * CW;
    const int rl = quad * 32 + lane;
    const float sigma = a.sigma, inv_sigma = a.inv_sigma;
    uint32_t j = 0;
    bool ok = true;
    for (int64_t item = blockIdx.x; item < a.n_items; item += gridDim.x) {
      const int64_t vc = item / a.n_rb, rb = item % a.n_rb;
      const int64_t t0 = vc * a.tiles_per_chunk;
      const int64_t t1 = min(a.vtiles, t0 + a.tiles_per_chunk);
      const int64_t row = rb * 128 + rl;
      const bool row_ok = row < a.rows;
      const uint32_t label = uint32_t(a.label0 + row);
      RowBest rbst;
      unsigned long long gkey = 0ull;
      if (row_ok) {
        gkey = __ldcg(&a.maxkey[row]);
        if (gkey) rbst.M = unpack_key_value(gkey);
      }
      for (int64_t t = t0; t < t1; ++t, ++j) {
        const uint32_t abuf = j & 1u, aph = (j >> 1) & 1u;
        if (ok && !mbar_wait(BAR(2 + abuf), aph, a.status, abort_flag)) ok = false;
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) continue;
        tc_fence_after();
        uint32_t r[CW];
        const uint32_t taddr = tmem + (uint32_t(quad * 32) << 16) + abuf * NT + colbase;
        if constexpr (CW == 32) {
          tc_ld_32x32b_x32(taddr, r);
        } else {
          tc_ld_32x32b_x16(taddr, r);
        }
        tc_wait_ld();
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(BAR(4 + abuf));  // accumulator free: values in registers
        if (!row_ok) continue;
        const int64_t c0 = t * NT + colbase;
#pragma unroll
        for (int g = 0; g < CW / 4; ++g) {  // unrolled: r stays in registers
          const int64_t c = c0 + 4 * g;
          if (c >= a.V) break;
          float mu[4];
#pragma unroll
          for (int h = 0; h < 4; ++h)
            mu[h] = c + h < a.V ? __uint_as_float(r[4 * g + h]) : -INFINITY;
          const float mq = fmaxf(fmaxf(mu[0], mu[1]), fmaxf(mu[2], mu[3]));
          // rounding guard of the skip test (absolute, in value units)
          const float guard = fmaf(2e-6f, fabsf(rbst.M) + fabsf(mq), 1e-3f * sigma) + 1e-30f;
          const float gap = rbst.M - mq - guard;
          if (gap * inv_sigma >= kNoiseBound) continue;  // no draw reaches M
          const uint4 o = philox(make_uint4(uint32_t(c >> 2), label, 0u, a.tag), a.k0, a.k1);
          const float thr = inv_sigma > 0.0f ? pair_threshold(gap, inv_sigma) : 4294967296.0f;
          if (__uint2float_rz(o.x) <= thr) {
            float z0, z1;
            bm_pair(o.x, o.y, z0, z1);
            rbst.take(fmaf(sigma, z0, mu[0]), uint32_t(c));
            if (c + 1 < a.V) rbst.take(fmaf(sigma, z1, mu[1]), uint32_t(c + 1));
          }
          if (c + 2 < a.V && __uint2float_rz(o.z) <= thr) {
            float z2, z3;
            bm_pair(o.z, o.w, z2, z3);
            rbst.take(fmaf(sigma, z2, mu[2]), uint32_t(c + 2));
            if (c + 3 < a.V) rbst.take(fmaf(sigma, z3, mu[3]), uint32_t(c + 3));
          }
        }
      }
      if (ok && row_ok && rbst.col != 0xffffffffu) {
        const unsigned long long key = pack_key(rbst.best, rbst.col);
        if (key > __ldcg(&a.maxkey[row])) atomicMax(&a.maxkey[row], key);
      }
    }
  }
#undef BFULL
#undef BEMPTY
#undef BAR
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, 2 * NT);
}

// Pieces hi, mid, lo of src (rows x RP, FP32) in core-matrix order, zero
// padded to rows_pad x Kp: element (i, k) of piece q at
// q rows_pad Kp + ((i / 8) (Kp / 8) + k / 8) 64 + (i % 8) 8 + k % 8.
__global__ void split3_tiled_kernel(const float* __restrict__ src, int64_t rows, int RP, int Kp,
                                    int64_t rows_pad, __nv_bfloat16* __restrict__ dst) {
  const int64_t total = rows_pad * Kp;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / Kp;
    const int k = int(e - i * Kp);
    const float x = (i < rows && k < RP) ? src[i * RP + k] : 0.0f;
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const float rx = x - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(rx);
    const __nv_bfloat16 l = __float2bfloat16_rn(rx - __bfloat162float(m));
    const int64_t off = ((i >> 3) * (Kp >> 3) + (k >> 3)) * 64 + (i & 7) * 8 + (k & 7);
    dst[off] = h;
    dst[total + off] = m;
    dst[2 * total + off] = l;
  }
}

int grid_for(int64_t work, int threads) {
  return int(std::max<int64_t>(1, std::min<int64_t>((work + threads - 1) / threads, 152 * 16)));
}

int smem_bytes(int NT, int Kp, int stages) {
  return 3 * 128 * Kp * 2 + stages * 3 * NT * Kp * 2 + (7 + 2 * stages) * 8 + 16;
}

}  // namespace

pt_status recon_tc(pt_ctx* ctx, const float* W, int64_t rows, int64_t label0, const float* U,
                   int64_t V, int RP, float sigma, uint32_t tag, uint32_t k0, uint32_t k1,
                   unsigned long long* keys) {
  if (rows <= 0 || V <= 0) return PT_OK;
  const int Kp = (RP + 15) / 16 * 16;
  const int NT = Kp <= 64 ? 128 : 64;
  int S = 8;
  while (S > 2 && smem_bytes(NT, Kp, S) > kSmemLimit - 1024) --S;
  const int smem = smem_bytes(NT, Kp, S);
  if (Kp > 128 || smem > kSmemLimit - 1024) {
    set_error(ctx, "RapidPT reconstruction: rank too large for the tensor-core tile");
    return PT_ERR_UNSUPPORTED;
  }
  const int64_t rows_pad = (rows + 127) / 128 * 128;
  const int64_t V_pad = (V + NT - 1) / NT * NT;
  if (3 * std::max(rows_pad, V_pad) * Kp / 256 >= (int64_t(1) << 31)) {
    set_error(ctx, "RapidPT reconstruction: too many rows or voxels for one tensor map");
    return PT_ERR_UNSUPPORTED;
  }
  Buf wp, up;
  struct Rel {
    Buf *a, *b;
    ~Rel() {
      a->release();
      b->release();
    }
  } rel{&wp, &up};
  if (!wp.ensure(sizeof(__nv_bfloat16) * 3 * size_t(rows_pad) * Kp) ||
      !up.ensure(sizeof(__nv_bfloat16) * 3 * size_t(V_pad) * Kp)) {
    set_error(ctx, "out of device memory (RapidPT reconstruction pieces)");
    return PT_ERR_NOMEM;
  }
  cudaStream_t st = ctx->stream;
  split3_tiled_kernel<<<grid_for(rows_pad * Kp, 256), 256, 0, st>>>(
      W, rows, RP, Kp, rows_pad, wp.as<__nv_bfloat16>());
  PT_LAUNCH_CHECK(ctx);
  split3_tiled_kernel<<<grid_for(V_pad * Kp, 256), 256, 0, st>>>(U, V, RP, Kp, V_pad,
                                                                up.as<__nv_bfloat16>());
  PT_LAUNCH_CHECK(ctx);

  ReconTcArgs a;
  memset(&a, 0, sizeof(a));
  if (!make_map(&a.tmW, wp.p, uint64_t(3) * rows_pad * Kp / 256, uint32_t(128 * Kp / 256)) ||
      !make_map(&a.tmU, up.p, uint64_t(3) * V_pad * Kp / 256, uint32_t(NT * Kp / 256))) {
    set_error(ctx, "cuTensorMapEncodeTiled failed (RapidPT reconstruction)");
    return PT_ERR_CUDA;
  }
  a.rows = rows;
  a.rows_pad = rows_pad;
  a.V = V;
  a.V_pad = V_pad;
  a.Kp = Kp;
  a.stages = S;
  a.label0 = label0;
  a.sigma = sigma;
  a.inv_sigma = sigma > 0.0f ? 1.0f / sigma : 0.0f;
  a.tag = tag;
  a.k0 = k0;
  a.k1 = k1;
  a.n_rb = rows_pad / 128;
  a.vtiles = V_pad / NT;
  // voxel chunks: enough items for ~16 per SM, each at least a few tiles
  const int sms = 152;
  int64_t n_vc = std::max<int64_t>(1, (int64_t(sms) * 16 + a.n_rb - 1) / a.n_rb);
  n_vc = std::min<int64_t>(n_vc, std::max<int64_t>(1, a.vtiles / 4));
  a.tiles_per_chunk = (a.vtiles + n_vc - 1) / n_vc;
  n_vc = (a.vtiles + a.tiles_per_chunk - 1) / a.tiles_per_chunk;
  a.n_items = n_vc * a.n_rb;
  a.maxkey = keys;
  a.status = ctx->status.as<uint32_t>();
  int dev = 0, nsm = sms;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int grid = int(std::min<int64_t>(a.n_items, nsm));
  auto kern = NT == 128 ? recon_tc_kernel<128> : recon_tc_kernel<64>;
  PT_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  prof_begin(ctx);
  kern<<<grid, kThreads, smem, st>>>(a);
  prof_end(ctx);
  PT_LAUNCH_CHECK(ctx);
  // the piece buffers are released (on return) only after the kernel ran
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return PT_OK;
}

}  // namespace pt
