// NaivePT (Alg. 1) on the GPU: relabelling rows -> 0/1 label matrix L, the
// contraction U = L . Xn^T (u = group-1 sum of unit-norm centred data), and
// the fused reduction to the max-null and per-voxel exceedance counts.
//
// Because t = sqrt(k(n-2)) u / sqrt(1 - k u^2) is the same strictly
// increasing function of u at every voxel, max_j t_ij = f(max_j u_ij), and
// t_ij >= t_obs_j  <=>  u_ij >= u_obs_j. The kernels therefore reduce u and
// convert only the P row maxima to t (in FP64) at the end.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {

// ---------------------------------------------------------------------------
// Labels: one warp per relabelling row. Validates the row (entries in range
// and distinct), then writes L[i][s] = 1 for the subjects of group 1.
// layout 0: float [P_pad][n_pad];  layout 1: bf16 8x8 core matrices (tensor-core A).
// ---------------------------------------------------------------------------
__global__ void labels_kernel(const int32_t* __restrict__ perms, int64_t P, int64_t P_pad, int n,
                              int n1, int n_pad, int layout, void* __restrict__ Lout,
                              uint8_t* __restrict__ rowflag, uint8_t* __restrict__ blockflag,
                              uint32_t* __restrict__ ident_count, uint32_t* __restrict__ status) {
  __shared__ uint32_t seen_all[8][32];
  __shared__ uint32_t g1_all[8][32];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* seen = seen_all[wib];
  uint32_t* g1 = g1_all[wib];
  const int64_t i = int64_t(blockIdx.x) * 8 + wib;
  if (i >= P_pad) return;
  seen[lane] = 0u;
  g1[lane] = 0u;
  __syncwarp();
  bool bad = false;
  if (i < P) {
    const int32_t* row = perms + i * n;
    for (int q = lane; q < n; q += 32) {
      const int32_t e = row[q];
      if (e < 0 || e >= n) {
        bad = true;
        continue;
      }
      const uint32_t bit = 1u << (e & 31);
      const uint32_t old = atomicOr(&seen[e >> 5], bit);
      if (old & bit) bad = true;
      if (q < n1) atomicOr(&g1[e >> 5], bit);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kErrBadPerm);
  __syncwarp();
  // Same group-1 set as the observed labelling (subjects 0..n1-1)? Such a row
  // ties the observed statistic exactly at every voxel; it is counted exactly
  // (once per voxel) instead of through a rounded comparison.
  const int lo = lane * 32;
  uint32_t want = 0u;
  if (n1 >= lo + 32) want = 0xffffffffu;
  else if (n1 > lo) want = (1u << (n1 - lo)) - 1u;
  const bool ident = (i < P) && __all_sync(0xffffffffu, g1[lane] == want);
  if (lane == 0) {
    rowflag[i] = ident ? 1 : 0;
    if (ident) {
      atomicAdd(ident_count, 1u);
      blockflag[i >> 7] = 1;
    }
  }
  for (int s = lane; s < n_pad; s += 32) {
    const bool in = (i < P) && s < n && ((g1[s >> 5] >> (s & 31)) & 1u);
    if (layout == 0) {
      static_cast<float*>(Lout)[i * n_pad + s] = in ? 1.0f : 0.0f;
    } else {
      // 128-row blocks, inside a block k-group major: core matrix (row group rg,
      // k group kg) of 8x8 elements at (kg * 16 + rg) * 64 -> one k-step of 16
      // subjects is a contiguous 4 KB slab (one TMA stage).
      const int64_t off = (i >> 7) * int64_t(128) * n_pad +
                          ((s >> 3) * 16 + ((i & 127) >> 3)) * 64 + (i & 7) * 8 + (s & 7);
      if (layout == 1)
        static_cast<__nv_bfloat16*>(Lout)[off] = __float2bfloat16(in ? 1.0f : 0.0f);
      else  // layout 2: FP16 labels for the FP16 data pieces
        static_cast<__half*>(Lout)[off] = __float2half(in ? 1.0f : 0.0f);
    }
  }
}

// ---------------------------------------------------------------------------
// Plain FP32 CUDA-core contraction with the fused epilogue.
// CTA tile 128 relabellings x 128 voxels, K step 16, 256 threads, 8x8 per thread.
// mode 0: reduce (row max -> packed key atomics, counts -> cnt)
// mode 1: write u rows to uout[row][voxel]
// ---------------------------------------------------------------------------
constexpr int BM = 128, BN = 128, BK = 16;

__global__ void __launch_bounds__(256, 2)
    simt_contract_kernel(const float* __restrict__ L, const float* __restrict__ Xn, int n_pad,
                         int64_t P, int64_t v, int tiles_per_cta, int mode, int two_sided,
                         const float* __restrict__ u_obs, const uint8_t* __restrict__ rowflag,
                         unsigned long long* __restrict__ maxkey, uint32_t* __restrict__ cnt,
                         float* __restrict__ uout) {
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Bs[2][BK][BN];
  __shared__ uint32_t scnt[BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int64_t v0 = int64_t(blockIdx.x) * BN;
  const int64_t ptiles = (P + BM - 1) / BM;
  const int64_t t_begin = int64_t(blockIdx.y) * tiles_per_cta;
  const int64_t t_end = min(ptiles, t_begin + tiles_per_cta);
  if (tid < BN) scnt[tid] = 0u;

  // loader mapping: row = tid >> 1 (0..127), k offset (tid & 1) * 8
  const int lrow = tid >> 1, lk = (tid & 1) * 8;
  const int ksteps = n_pad / BK;

  float uo[8];
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const int col = (b < 4) ? (tx * 4 + b) : (64 + tx * 4 + b - 4);
    const int64_t gc = v0 + col;
    float x = (mode == 0 && gc < v) ? u_obs[gc] : 0.0f;
    uo[b] = two_sided ? fabsf(x) : x;
  }

  for (int64_t pt = t_begin; pt < t_end; ++pt) {
    const int64_t p0 = pt * BM;
    float acc[8][8];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int b = 0; b < 8; ++b) acc[a][b] = 0.0f;

    const float* Lrow = L + (p0 + lrow) * n_pad + lk;      // L is padded to whole tiles
    const float* Xrow = Xn + (v0 + lrow) * n_pad + lk;     // Xn is padded to 256 voxels
    float4 ra0 = *reinterpret_cast<const float4*>(Lrow);
    float4 ra1 = *reinterpret_cast<const float4*>(Lrow + 4);
    float4 rb0 = *reinterpret_cast<const float4*>(Xrow);
    float4 rb1 = *reinterpret_cast<const float4*>(Xrow + 4);
    __syncthreads();
    for (int ks = 0; ks < ksteps; ++ks) {
      const int buf = ks & 1;
      As[buf][lk + 0][lrow] = ra0.x; As[buf][lk + 1][lrow] = ra0.y;
      As[buf][lk + 2][lrow] = ra0.z; As[buf][lk + 3][lrow] = ra0.w;
      As[buf][lk + 4][lrow] = ra1.x; As[buf][lk + 5][lrow] = ra1.y;
      As[buf][lk + 6][lrow] = ra1.z; As[buf][lk + 7][lrow] = ra1.w;
      Bs[buf][lk + 0][lrow] = rb0.x; Bs[buf][lk + 1][lrow] = rb0.y;
      Bs[buf][lk + 2][lrow] = rb0.z; Bs[buf][lk + 3][lrow] = rb0.w;
      Bs[buf][lk + 4][lrow] = rb1.x; Bs[buf][lk + 5][lrow] = rb1.y;
      Bs[buf][lk + 6][lrow] = rb1.z; Bs[buf][lk + 7][lrow] = rb1.w;
      __syncthreads();
      if (ks + 1 < ksteps) {
        const int ko = (ks + 1) * BK;
        ra0 = *reinterpret_cast<const float4*>(Lrow + ko);
        ra1 = *reinterpret_cast<const float4*>(Lrow + ko + 4);
        rb0 = *reinterpret_cast<const float4*>(Xrow + ko);
        rb1 = *reinterpret_cast<const float4*>(Xrow + ko + 4);
      }
#pragma unroll
      for (int k = 0; k < BK; ++k) {
        const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
        const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
        const float4 b0 = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
        const float4 b1 = *reinterpret_cast<const float4*>(&Bs[buf][k][64 + tx * 4]);
        const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
        const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int a = 0; a < 8; ++a)
#pragma unroll
          for (int b = 0; b < 8; ++b) acc[a][b] = fmaf(av[a], bv[b], acc[a][b]);
      }
    }

    if (mode == 1) {
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t row = p0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
        if (row >= P) continue;
#pragma unroll
        for (int b = 0; b < 8; ++b) {
          const int64_t col = v0 + ((b < 4) ? (tx * 4 + b) : (64 + tx * 4 + b - 4));
          if (col < v) uout[row * v + col] = acc[a][b];
        }
      }
      continue;
    }

    // ---- fused epilogue: row max (with smallest-index ties) and counts ----
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      const int64_t row = p0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
      float best = -INFINITY;
      uint32_t bj = 0xffffffffu;
#pragma unroll
      for (int b = 0; b < 8; ++b) {
        const int64_t col = v0 + ((b < 4) ? (tx * 4 + b) : (64 + tx * 4 + b - 4));
        const float s = two_sided ? fabsf(acc[a][b]) : acc[a][b];
        if (col < v && (s > best || (s == best && uint32_t(col) < bj))) {
          best = s;
          bj = uint32_t(col);
        }
      }
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) {
        const float ob = __shfl_xor_sync(0xffffffffu, best, o);
        const uint32_t oj = __shfl_xor_sync(0xffffffffu, bj, o);
        if (ob > best || (ob == best && oj < bj)) {
          best = ob;
          bj = oj;
        }
      }
      if (tx == 0 && row < P && bj != 0xffffffffu) {
        const unsigned long long key = pack_key(best, bj);
        if (key > maxkey[row]) atomicMax(&maxkey[row], key);
      }
    }
#pragma unroll
    for (int b = 0; b < 8; ++b) {
      const int colo = (b < 4) ? (tx * 4 + b) : (64 + tx * 4 + b - 4);
      uint32_t c = 0;
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const int64_t row = p0 + ((a < 4) ? (ty * 4 + a) : (64 + ty * 4 + a - 4));
        const float s = two_sided ? fabsf(acc[a][b]) : acc[a][b];
        c += (row < P && s >= uo[b] && !rowflag[row]) ? 1u : 0u;
      }
      // reduce over the two ty rows of this warp, then shared atomics
      c += __shfl_xor_sync(0xffffffffu, c, 16);
      if ((tid & 16) == 0 && c) atomicAdd(&scnt[colo], c);
    }
  }
  if (mode == 0) {
    __syncthreads();
    if (tid < BN) {
      const int64_t col = v0 + tid;
      if (col < v && scnt[tid]) atomicAdd(&cnt[col], scnt[tid]);
    }
  }
}

// ---------------------------------------------------------------------------
// Finalise: packed keys -> t (FP64 from u), masked argmax; counts -> masked order.
// ---------------------------------------------------------------------------
// Sixteen lanes per relabelling row (two rows per warp, kFinRowsPerBlock rows
// per 256-thread CTA, so a 10,000-row call fits in one wave of the GPU). The
// contraction only selects the winning voxel (u orders voxels exactly as t
// does); its statistic is then recomputed here in FP64 from the input values,
// two-pass, as Eq. (5) defines it, so the reported maximum carries no
// FP32/BF16 error even where t = f(u) is ill-conditioned (few degrees of
// freedom, very unequal groups).
__global__ void __launch_bounds__(256)
    finalize_max_kernel(const unsigned long long* __restrict__ maxkey, int64_t P,
                        const int32_t* __restrict__ valid_map, const float* __restrict__ Xraw,
                        int n, int n1, int n_pad, const int32_t* __restrict__ perms,
                        int two_sided, float* __restrict__ maxnull, int32_t* __restrict__ argmax) {
  constexpr int L = 256 / kFinRowsPerBlock;  // lanes per row
  __shared__ uint32_t g1_all[kFinRowsPerBlock][32];
  __shared__ double rc[3];  // 1/n1, 1/n2, (1/n1 + 1/n2)/(n - 2)
  const int grp = threadIdx.x / L, gl = threadIdx.x % L;
  const unsigned gmask = ((1u << L) - 1u) << (threadIdx.x & 31 & ~(L - 1));
  uint32_t* g1 = g1_all[grp];
  if (threadIdx.x == 0) {
    rc[0] = __drcp_rn(double(n1));
    rc[1] = __drcp_rn(double(n - n1));
    rc[2] = (rc[0] + rc[1]) * __drcp_rn(double(n - 2));
  }
  __syncthreads();
  for (int64_t i = int64_t(blockIdx.x) * kFinRowsPerBlock + grp; i < P;
       i += int64_t(gridDim.x) * kFinRowsPerBlock) {
    const unsigned long long key = maxkey[i];
    if (key == 0ull) {
      if (gl == 0) {
        maxnull[i] = -INFINITY;
        argmax[i] = -1;
      }
      continue;
    }
    const uint32_t c = unpack_key_index(key);
    for (int q = gl; q < 32; q += L) g1[q] = 0u;
    __syncwarp(gmask);
    const int32_t* row = perms + i * n;
    for (int q = gl; q < n1; q += L) {
      const int32_t e = row[q];
      if (e >= 0 && e < n) atomicOr(&g1[e >> 5], 1u << (e & 31));  // others: reported by labels
    }
    __syncwarp(gmask);
    const float* x = Xraw + int64_t(valid_map[c]) * n_pad;  // Xraw is in masked order
    // Two-pass group sums in float-float (FP32 pipes; ~44 significant bits) of
    // the values scaled by the power of two that puts max |x| in [1, 2) (exact;
    // squares cannot overflow; t does not depend on the scale), the means and
    // the statistic in FP64.
    float amax = 0.0f;
    for (int s = gl; s < n; s += L) amax = fmaxf(amax, fabsf(x[s]));
    for (int o = L / 2; o > 0; o >>= 1) amax = fmaxf(amax, __shfl_xor_sync(gmask, amax, o));
    int ex = int((__float_as_uint(amax) >> 23) & 0xffu) - 127;
    ex = ex < -126 ? -126 : (ex > 126 ? 126 : ex);
    const float scale = __uint_as_float(uint32_t(127 - ex) << 23);
    float s1h = 0.0f, s1l = 0.0f, s2h = 0.0f, s2l = 0.0f;
    for (int s = gl; s < n; s += L) {
      const float xs = x[s] * scale;
      if ((g1[s >> 5] >> (s & 31)) & 1u) ff_acc(s1h, s1l, xs, 0.0f);
      else ff_acc(s2h, s2l, xs, 0.0f);
    }
    for (int o = L / 2; o > 0; o >>= 1) {  // two-sum is exact, so every lane ends with the same sums
      const float a = __shfl_xor_sync(gmask, s1h, o), b = __shfl_xor_sync(gmask, s1l, o);
      const float c2 = __shfl_xor_sync(gmask, s2h, o), d = __shfl_xor_sync(gmask, s2l, o);
      ff_acc(s1h, s1l, a, b);
      ff_acc(s2h, s2l, c2, d);
    }
    const double m1 = ff_d(s1h, s1l) * rc[0], m2 = ff_d(s2h, s2l) * rc[1];
    const float m1h = float(m1), m1l = float(m1 - double(m1h));
    const float m2h = float(m2), m2l = float(m2 - double(m2h));
    float ssh = 0.0f, ssl = 0.0f;
    for (int s = gl; s < n; s += L) {
      const bool in1 = (g1[s >> 5] >> (s & 31)) & 1u;
      float dh, dl;
      two_sum(x[s] * scale, in1 ? -m1h : -m2h, dh, dl);
      dl -= in1 ? m1l : m2l;
      const float tt = dh + dl;
      dl = dl - (tt - dh);
      dh = tt;
      const float p = dh * dh;
      ff_acc(ssh, ssl, p, fmaf(2.0f * dh, dl, fmaf(dh, dh, -p)));
    }
    for (int o = L / 2; o > 0; o >>= 1) {
      const float a = __shfl_xor_sync(gmask, ssh, o), b = __shfl_xor_sync(gmask, ssl, o);
      ff_acc(ssh, ssl, a, b);
    }
    const double ss = ff_d(ssh, ssl);
    if (gl == 0) {
      const double t = (m1 - m2) * rsqrt(ss * rc[2]);
      maxnull[i] = float(two_sided ? fabs(t) : t);
      argmax[i] = valid_map[c];
    }
    __syncwarp(gmask);
  }
}

// counts[masked voxel] = comparisons counted by the contraction + relabellings
// whose group-1 set equals the observed one (cnt[v_valid]).
__global__ void scatter_counts_kernel(const uint32_t* __restrict__ cnt, int64_t v_valid,
                                      const int32_t* __restrict__ valid_map,
                                      uint32_t* __restrict__ counts, int accumulate) {
  const uint32_t ties = cnt[v_valid];
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < v_valid;
       c += int64_t(gridDim.x) * blockDim.x) {
    const int32_t j = valid_map[c];
    counts[j] = (accumulate ? counts[j] : 0u) + cnt[c] + ties;
  }
}

// FWER-corrected p-values: p_j = (1 + #{i : m_i >= T_j}) / (P + 1) over the
// max-null, T_j the voxel's observed statistic (float32 on both sides of the
// comparison). Brute force: each thread one voxel, the maxima streamed through
// shared memory in tiles.
constexpr int kPvalTile = 4096;
__global__ void __launch_bounds__(256) fwer_pvalues_kernel(const float* __restrict__ maxnull,
                                                           int64_t P,
                                                           const double* __restrict__ t_obs64,
                                                           int64_t v, int two_sided,
                                                           float* __restrict__ p_out) {
  __shared__ float tile[kPvalTile];
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  float T = NAN;
  if (j < v) {
    T = float(t_obs64[j]);
    if (two_sided) T = fabsf(T);
  }
  uint32_t cnt = 0;
  for (int64_t i0 = 0; i0 < P; i0 += kPvalTile) {
    const int len = int(P - i0 < kPvalTile ? P - i0 : kPvalTile);
    __syncthreads();
    for (int k = threadIdx.x; k < len; k += blockDim.x) tile[k] = maxnull[i0 + k];
    __syncthreads();
    int k = 0;
    uint32_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    for (; k + 3 < len; k += 4) {
      c0 += tile[k] >= T;
      c1 += tile[k + 1] >= T;
      c2 += tile[k + 2] >= T;
      c3 += tile[k + 3] >= T;
    }
    for (; k < len; ++k) c0 += tile[k] >= T;
    cnt += c0 + c1 + c2 + c3;
  }
  if (j < v) p_out[j] = isnan(T) ? NAN : float((1.0 + double(cnt)) / (double(P) + 1.0));
}

static int grid_1d(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return int(b);
}

// Build labels for P rows into ctx->labels (layout per path), with the
// observed-set flags; ctx->cnt must already hold v_valid + 1 zeroed words.
pt_status build_labels(pt_ctx* ctx, const int32_t* perms, int64_t P, int layout, int64_t* P_pad_out) {
  const int64_t P_pad = (P + 127) / 128 * 128;
  const size_t elem = layout == 0 ? sizeof(float) : sizeof(__nv_bfloat16);  // BF16 / FP16: 2 B
  if (!ctx->labels.ensure(elem * size_t(P_pad) * ctx->n_pad) || !ctx->rowflag.ensure(P_pad) ||
      !ctx->blockflag.ensure(P_pad / 128)) {
    set_error(ctx, "out of device memory (labels)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->blockflag.p, 0, P_pad / 128, ctx->stream));
  labels_kernel<<<unsigned((P_pad + 7) / 8), 256, 0, ctx->stream>>>(
      perms, P, P_pad, ctx->n, ctx->n1, ctx->n_pad, layout, ctx->labels.p,
      ctx->rowflag.as<uint8_t>(), ctx->blockflag.as<uint8_t>(),
      ctx->cnt.as<uint32_t>() + ctx->v_valid, ctx->status.as<uint32_t>());
  PT_LAUNCH_CHECK(ctx);
  if (ctx->glm_q1 && layout != 0) {
    pt_status s = glm_rowscale(ctx, perms, P, P_pad);
    if (s != PT_OK) return s;
  }
  *P_pad_out = P_pad;
  return PT_OK;
}

// SIMT launch: grid (voxel tiles, relabelling chunks).
static pt_status launch_simt(pt_ctx* ctx, const float* L, int64_t P, int mode, int two_sided,
                             const float* u_obs, unsigned long long* maxkey, uint32_t* cnt,
                             float* uout) {
  const int64_t vt = (ctx->v_valid + BN - 1) / BN;
  const int64_t ptiles = (P + BM - 1) / BM;
  int64_t chunks = (152 * 2 * 4 + vt - 1) / vt;
  if (chunks > ptiles) chunks = ptiles;
  if (chunks < 1) chunks = 1;
  if (chunks > 65535) chunks = 65535;
  const int per = int((ptiles + chunks - 1) / chunks);
  chunks = (ptiles + per - 1) / per;
  const dim3 grid{unsigned(vt), unsigned(chunks), 1u};
  if (mode == 0) prof_begin(ctx);
  simt_contract_kernel<<<grid, 256, 0, ctx->stream>>>(
      L, ctx->Xn32.as<float>(), ctx->n_pad, P, ctx->v_valid, per, mode, two_sided, u_obs,
      ctx->rowflag.as<uint8_t>(), maxkey, cnt, uout);
  if (mode == 0) prof_end(ctx);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

pt_status naive_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, const pt_naive_opts& o,
                     float* maxnull, int32_t* argmax, uint32_t* counts) {
  cudaStream_t st = ctx->stream;
  const bool tc = o.precision != PT_PREC_FP32;
  if (ctx->glm_q1 && !tc) {
    set_error(ctx, "the covariate-adjusted statistic runs on the tensor-core path (BF16X2/X3)");
    return PT_ERR_UNSUPPORTED;
  }
  pt_status s = tc ? tc_supported(ctx) : PT_OK;
  if (s != PT_OK) return s;
  if (!ctx->maxkey.ensure(sizeof(unsigned long long) * P) ||
      !ctx->cnt.ensure(sizeof(uint32_t) * (ctx->v_valid + 1))) {
    set_error(ctx, "out of device memory (workspace)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->maxkey.p, 0, sizeof(unsigned long long) * P, st));
  PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cnt.p, 0, sizeof(uint32_t) * (ctx->v_valid + 1), st));
  if (counts && !o.accumulate_counts)
    PT_CUDA_TRY(ctx, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ctx->v, st));
  int64_t P_pad = 0;
  s = build_labels(ctx, perms, P, prec_label_layout(o.precision), &P_pad);
  if (s != PT_OK) return s;
  if (ctx->v_valid > 0) {
    if (!tc) {
      s = ensure_xn32(ctx);
      if (s == PT_OK)
        s = launch_simt(ctx, ctx->labels.as<float>(), P, 0, o.two_sided, ctx->u_obs.as<float>(),
                        ctx->maxkey.as<unsigned long long>(), ctx->cnt.as<uint32_t>(), nullptr);
    } else {
      s = ensure_xnb(ctx, o.precision);
      if (s == PT_OK)
        s = tc_reduce(ctx, ctx->labels.p, P, o.precision, o.two_sided, ctx->u_obs.as<float>(),
                      ctx->maxkey.as<unsigned long long>(), ctx->cnt.as<uint32_t>());
    }
    if (s != PT_OK) return s;
  }
  if (ctx->glm_q1) {
    s = glm_finalize(ctx, perms, P, o.two_sided, maxnull, argmax);
    if (s != PT_OK) return s;
  } else {
    const int fin_blocks = grid_1d((P + kFinRowsPerBlock - 1) / kFinRowsPerBlock, 1);
    finalize_max_kernel<<<fin_blocks, 256, 0, st>>>(
        ctx->maxkey.as<unsigned long long>(), P, ctx->valid_map.as<int32_t>(),
        ctx->Xraw.as<float>(), ctx->n, ctx->n1, ctx->n_pad, perms, o.two_sided, maxnull, argmax);
    PT_LAUNCH_CHECK(ctx);
  }
  if (counts && ctx->v_valid > 0) {
    scatter_counts_kernel<<<grid_1d(ctx->v_valid, 256), 256, 0, st>>>(
        ctx->cnt.as<uint32_t>(), ctx->v_valid, ctx->valid_map.as<int32_t>(), counts,
        o.accumulate_counts);
    PT_LAUNCH_CHECK(ctx);
  }
  return PT_OK;
}

pt_status fwer_pvalues_impl(pt_ctx* ctx, const float* maxnull, int64_t P, int two_sided,
                            float* p_out) {
  if (ctx->v < 1) return PT_OK;
  const int64_t blocks = (ctx->v + 255) / 256;
  fwer_pvalues_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(
      maxnull, P, ctx->t_obs64.as<double>(), ctx->v, two_sided, p_out);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

// ---------------------------------------------------------------------------
// pt_maxnull_naive_batched: every study's labels, one persistent fused launch
// per tile class over all studies of that class, then every study's
// finalisation. The sequence is captured once into a CUDA graph on a private
// stream and replayed on the caller's stream while the arguments repeat.
// ---------------------------------------------------------------------------
namespace {
struct BatchGraph {
  std::vector<const void*> key;
  cudaGraphExec_t exec = nullptr;
  int device = -1;
  cudaStream_t capture = nullptr;
  int64_t launches = 0;  // kernels in the graph
  Buf desc;
  std::vector<char> host_desc;
  std::vector<TcGroup> groups;
  std::vector<const pt_ctx*> members;
};
std::mutex g_batch_mu;
BatchGraph g_batch;

void drop_graph_locked() {
  if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
  g_batch.exec = nullptr;
  g_batch.key.clear();
  g_batch.members.clear();
}
}  // namespace

// Called when the tuned configurations change: the next batched call replans.
void batch_drop_graph() {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  drop_graph_locked();
}

// Called by pt_destroy: a cached graph must not outlive the buffers it names.
bool batch_forget(const pt_ctx* ctx) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (const pt_ctx* m : g_batch.members)
    if (m == ctx) {
      drop_graph_locked();
      return true;
    }
  return false;
}

static pt_status batched_enqueue(pt_ctx* lead, pt_ctx* const* ctxs, int n,
                                 const int32_t* const* perms, const int64_t* P,
                                 const pt_naive_opts& o, float* const* maxnull,
                                 int32_t* const* argmax, uint32_t* const* counts) {
  cudaStream_t st = lead->stream;
  for (int i = 0; i < n; ++i) {
    pt_ctx* c = ctxs[i];
    PT_CUDA_TRY(lead, cudaMemsetAsync(c->maxkey.p, 0, sizeof(unsigned long long) * P[i], st));
    PT_CUDA_TRY(lead, cudaMemsetAsync(c->cnt.p, 0, sizeof(uint32_t) * (c->v_valid + 1), st));
    if (counts && counts[i] && !o.accumulate_counts)
      PT_CUDA_TRY(lead, cudaMemsetAsync(counts[i], 0, sizeof(uint32_t) * c->v, st));
    int64_t P_pad = 0;
    pt_status s = build_labels(c, perms[i], P[i], prec_label_layout(o.precision), &P_pad);
    if (s != PT_OK) return s;
  }
  pt_status s = tc_batch_launch(lead, g_batch.desc, g_batch.groups, o.precision, o.two_sided);
  if (s != PT_OK) return s;
  for (int i = 0; i < n; ++i) {
    pt_ctx* c = ctxs[i];
    const int fin_blocks = grid_1d((P[i] + kFinRowsPerBlock - 1) / kFinRowsPerBlock, 1);
    finalize_max_kernel<<<fin_blocks, 256, 0, st>>>(
        c->maxkey.as<unsigned long long>(), P[i], c->valid_map.as<int32_t>(), c->Xraw.as<float>(),
        c->n, c->n1, c->n_pad, perms[i], o.two_sided, maxnull[i], argmax[i]);
    PT_LAUNCH_CHECK(lead);
    if (counts && counts[i] && c->v_valid > 0) {
      scatter_counts_kernel<<<grid_1d(c->v_valid, 256), 256, 0, st>>>(
          c->cnt.as<uint32_t>(), c->v_valid, c->valid_map.as<int32_t>(), counts[i],
          o.accumulate_counts);
      PT_LAUNCH_CHECK(lead);
    }
  }
  return PT_OK;
}

// Everything a captured batch names: replay only while all of it is unchanged.
static std::vector<const void*> batch_key(pt_ctx* const* ctxs, int n, const int32_t* const* perms,
                                          const int64_t* P, const pt_naive_opts& o,
                                          float* const* maxnull, int32_t* const* argmax,
                                          uint32_t* const* counts) {
  std::vector<const void*> key;
  key.push_back(reinterpret_cast<const void*>(intptr_t(n)));
  key.push_back(
      reinterpret_cast<const void*>(intptr_t((o.precision * 2 + o.two_sided) * 2 +
                                             o.accumulate_counts)));
  key.push_back(reinterpret_cast<const void*>(intptr_t(ctxs[0]->device)));
  for (int i = 0; i < n; ++i) {
    key.push_back(ctxs[i]);
    key.push_back(perms[i]);
    key.push_back(reinterpret_cast<const void*>(intptr_t(P[i])));
    key.push_back(maxnull[i]);
    key.push_back(argmax[i]);
    key.push_back(counts ? counts[i] : nullptr);
    // workspaces named by the graph (a single-study call may have regrown them)
    for (const Buf* b : {&ctxs[i]->labels, &ctxs[i]->maxkey, &ctxs[i]->cnt, &ctxs[i]->rowflag,
                         &ctxs[i]->blockflag, &ctxs[i]->Xnb}) {
      key.push_back(b->p);
      key.push_back(reinterpret_cast<const void*>(b->bytes));
    }
  }
  return key;
}

pt_status naive_batched_impl(pt_ctx* const* ctxs, int n, const int32_t* const* perms,
                             const int64_t* P, const pt_naive_opts& o, float* const* maxnull,
                             int32_t* const* argmax, uint32_t* const* counts) {
  pt_ctx* lead = ctxs[0];
  if (o.precision == PT_PREC_FP32) {
    set_error(lead, "pt_maxnull_naive_batched runs the tensor-core path (BF16x2/x3, FP16x2)");
    return PT_ERR_UNSUPPORTED;
  }
  pt_status s = tc_supported(lead);
  if (s != PT_OK) return s;
  for (int i = 0; i < n; ++i)
    if (ctxs[i]->glm_q1) {
      set_error(lead, "pt_maxnull_naive_batched: covariate-adjusted contexts run one at a time");
      return PT_ERR_UNSUPPORTED;
    }

  const std::vector<const void*> key = batch_key(ctxs, n, perms, P, o, maxnull, argmax, counts);
  std::lock_guard<std::mutex> lk(g_batch_mu);
  if (g_batch.exec && g_batch.key == key) {
    PT_CUDA_TRY(lead, cudaGraphLaunch(g_batch.exec, lead->stream));
    for (int64_t k = 0; k < g_batch.launches; ++k) count_launch();
    return PT_OK;
  }
  drop_graph_locked();

  // Everything that allocates or copies from the host happens before capture.
  for (int i = 0; i < n; ++i) {
    pt_ctx* c = ctxs[i];
    if (c->device != lead->device) {
      set_error(lead, "pt_maxnull_naive_batched: all contexts must be on one device");
      return PT_ERR_INVALID;
    }
    if (c->v_valid > 0) {
      s = ensure_xnb(c, o.precision);
      if (s != PT_OK) return s;
    }
    const int64_t P_pad = (P[i] + 127) / 128 * 128;
    if (!c->maxkey.ensure(sizeof(unsigned long long) * P[i]) ||
        !c->cnt.ensure(sizeof(uint32_t) * (c->v_valid + 1)) ||
        !c->labels.ensure(sizeof(__nv_bfloat16) * size_t(P_pad) * c->n_pad) ||
        !c->rowflag.ensure(P_pad) || !c->blockflag.ensure(P_pad / 128)) {
      set_error(lead, "out of device memory (batched workspaces)");
      return PT_ERR_NOMEM;
    }
    PT_CUDA_TRY(lead, cudaStreamSynchronize(c->stream));
  }
  s = tc_batch_plan(lead, ctxs, P, n, o, g_batch.desc, g_batch.host_desc, g_batch.groups);
  if (s != PT_OK) return s;
  if (g_batch.device != lead->device) {
    if (g_batch.capture) cudaStreamDestroy(g_batch.capture);
    g_batch.capture = nullptr;
    g_batch.device = lead->device;
  }
  if (!g_batch.capture)
    PT_CUDA_TRY(lead, cudaStreamCreateWithFlags(&g_batch.capture, cudaStreamNonBlocking));

  // Capture on the private stream (the caller's may be the legacy default stream).
  std::vector<cudaStream_t> saved(n);
  std::vector<bool> saved_prof(n);
  for (int i = 0; i < n; ++i) {
    saved[i] = ctxs[i]->stream;
    saved_prof[i] = ctxs[i]->profile;
    ctxs[i]->stream = g_batch.capture;
    ctxs[i]->profile = false;
  }
  const cudaStream_t user = saved[0];
  const int64_t before = launch_counter();
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamBeginCapture(g_batch.capture, cudaStreamCaptureModeThreadLocal);
  if (ce == cudaSuccess) {
    s = batched_enqueue(lead, ctxs, n, perms, P, o, maxnull, argmax, counts);
    ce = cudaStreamEndCapture(g_batch.capture, &graph);
  }
  for (int i = 0; i < n; ++i) {
    ctxs[i]->stream = saved[i];
    ctxs[i]->profile = saved_prof[i];
  }
  const int64_t captured = launch_counter() - before;
  add_launch_count(-captured);  // counted when the graph runs
  if (s != PT_OK || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (s == PT_OK) {
      set_error(lead, std::string("graph capture: ") + cudaGetErrorString(ce));
      s = PT_ERR_CUDA;
    }
    return s;
  }
  cudaGraphExec_t exec = nullptr;
  ce = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ce != cudaSuccess) {
    set_error(lead, std::string("graph instantiate: ") + cudaGetErrorString(ce));
    return PT_ERR_CUDA;
  }
  g_batch.exec = exec;
  g_batch.key = batch_key(ctxs, n, perms, P, o, maxnull, argmax, counts);
  g_batch.launches = captured;
  g_batch.members.assign(ctxs, ctxs + n);
  PT_CUDA_TRY(lead, cudaGraphLaunch(exec, user));
  add_launch_count(captured);
  return PT_OK;
}

}  // namespace pt
