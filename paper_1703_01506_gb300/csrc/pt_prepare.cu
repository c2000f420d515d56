// pt_prepare: mask compaction, per-voxel moments, observed t, a raw
// voxel-major copy of the data; and, on first use, the unit-norm centred data
// Xn in FP32 rows or as BF16 pieces (8x8 core-matrix layout read by the
// tensor-core kernel).
//
// With x the n values of a voxel, mean and SS = sum (x - mean)^2 (see Moments):
//   Xn_s = (x_s - mean) / sqrt(SS),      so sum_s Xn_s = 0 and sum_s Xn_s^2 = 1.
// For a relabelling with group-1 sum u = sum_{s in G1} Xn_s the pooled t of
// Eq. (5) is t = sqrt(k (n-2)) u / sqrt(1 - k u^2), k = 1/n1 + 1/n2, because
// mean1 - mean2 = k s1 and the within-group SS = SS - k s1^2 with s1 = u sqrt(SS).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include <cmath>
#include <string>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPerThread = 16;
constexpr int kScanChunk = kScanThreads * kScanPerThread;

__device__ __forceinline__ bool flag_at(const uint8_t* f, int64_t i, int64_t N) {
  return i < N && f[i] != 0;
}

__global__ void scan_count_kernel(const uint8_t* __restrict__ flags, int64_t N,
                                  uint32_t* __restrict__ block_counts) {
  const int64_t base = int64_t(blockIdx.x) * kScanChunk + int64_t(threadIdx.x) * kScanPerThread;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kScanPerThread; ++e) c += flag_at(flags, base + e, N) ? 1u : 0u;
  __shared__ uint32_t red[kScanThreads / 32];
  for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t t = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) t += red[w];
    block_counts[blockIdx.x] = t;
  }
}

// Single-block exclusive scan of block counts (in place), total at [nb].
__global__ void scan_blocks_kernel(uint32_t* __restrict__ counts, int64_t nb) {
  __shared__ uint64_t carry;
  __shared__ uint32_t warp_tot[32];
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t b0 = 0; b0 < nb; b0 += blockDim.x) {
    const int64_t b = b0 + threadIdx.x;
    const uint32_t x = b < nb ? counts[b] : 0u;
    uint32_t incl = x;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      const int nw = blockDim.x >> 5;
      uint32_t t = lane < nw ? warp_tot[lane] : 0u;
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      if (lane < nw) warp_tot[lane] = t;  // inclusive over warps
    }
    __syncthreads();
    const uint32_t before_warp = w > 0 ? warp_tot[w - 1] : 0u;
    const uint64_t excl = carry + before_warp + incl - x;
    if (b < nb) counts[b] = uint32_t(excl);
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + x;
    __syncthreads();
  }
  if (threadIdx.x == 0) counts[nb] = uint32_t(carry);
}

template <class IdxT>
__global__ void scan_write_kernel(const uint8_t* __restrict__ flags, int64_t N,
                                  const uint32_t* __restrict__ block_offsets,
                                  IdxT* __restrict__ out) {
  const int64_t base = int64_t(blockIdx.x) * kScanChunk + int64_t(threadIdx.x) * kScanPerThread;
  uint32_t c = 0;
#pragma unroll
  for (int e = 0; e < kScanPerThread; ++e) c += flag_at(flags, base + e, N) ? 1u : 0u;
  // block exclusive scan of per-thread counts (thread order = index order)
  __shared__ uint32_t warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t incl = c;
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  uint32_t before = 0;
  for (int q = 0; q < w; ++q) before += warp_tot[q];
  uint32_t pos = block_offsets[blockIdx.x] + before + incl - c;
#pragma unroll
  for (int e = 0; e < kScanPerThread; ++e)
    if (flag_at(flags, base + e, N)) out[pos++] = IdxT(base + e);
}

__global__ void iota64_kernel(int64_t* __restrict__ out, int64_t N) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < N;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = i;
}

// ---------------------------------------------------------------------------
// Moments. A CTA takes 32 consecutive mask voxels (lane = voxel); warp w holds
// subjects w, w + 8, ... of them in a shared-memory tile (reads of X along a
// grid row are coalesced), and the tile is written out as voxel-major rows of
// Xraw. Per voxel:
//   pass 1: FP32 sum of x (a seed mean m), max |x|, the flags;
//   pass 2: with y = x s and s the power of two that brings max |x| into
//           [1, 2) (exact; squares cannot overflow for any finite input),
//           d = y - m s exactly as a pair (two-sum), and per group the sums
//           D_g = sum_{G_g} d and Q_g = sum_{G_g} d^2 as float-float pairs
//           (an unevaluated h + l, about 44 significant bits);
// then finished in float-float (FP64 issues at a small fraction of the FP32
// rate on this part; only the three outputs are widened to FP64):
//   delta = (D_1 + D_2)/n,  SS = Q_1 + Q_2 - (D_1 + D_2) delta  (the corrected
//   two-pass formula: the seed mean's rounding cancels),
//   A_1 = sum_{G_1} (y - mean(y)) = (n_2 D_1 - n_1 D_2)/n,
//   SS_w = SS - k A_1^2     (between-group SS = A_1^2/n_1 + A_2^2/n_2, A_2 = -A_1),
//   t_obs = sqrt(k (n-2)) A_1 / sqrt(SS_w)                        (Eq. (5)),
//   u_obs = A_1 / sqrt(SS),
// with 1/sqrt from the FP32 estimate and one Newton step carried in
// float-float (relative error about 2^-43). t and u do not depend on s; the
// mean and 1/sqrt(SS) are unscaled exactly. A voxel is degenerate (no t)
// exactly when all its values are equal.
constexpr int kMV = 32;  // voxels per CTA (one per lane)
constexpr int kMW = 8;   // warps per CTA; warp w holds subjects s = w, w + 8, ...
constexpr int kMU = 4;   // subject loads in flight per warp (host-memory X)
constexpr float kFltMax = 3.402823466e38f;

// Float-float values: h + l with |l| <= ulp(h)/2.
struct FF {
  float h, l;
};
__device__ __forceinline__ FF ff_norm(float s, float e) {  // needs |s| >= |e|
  const float h = s + e;
  return {h, e - (h - s)};
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s, e;
  two_sum(a.h, b.h, s, e);
  return ff_norm(s, e + (a.l + b.l));
}
__device__ __forceinline__ FF ff_sub(FF a, FF b) { return ff_add(a, FF{-b.h, -b.l}); }
__device__ __forceinline__ FF ff_mul(FF a, FF b) {
  const float p = a.h * b.h;
  const float e = fmaf(a.h, b.h, -p);  // the product's rounding error, exact
  return ff_norm(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
__device__ __forceinline__ FF ff_mulf(FF a, float b) {
  const float p = a.h * b;
  return ff_norm(p, fmaf(a.l, b, fmaf(a.h, b, -p)));
}
__device__ __forceinline__ double ff_d(FF a) { return double(a.h) + double(a.l); }
// 1/sqrt(x), x > 0 (normal): r = rsqrtf(x.h) is within a few ulp, so y = x r^2
// lies within 2^-20 of 1 and 1 - y.h is exact; one Newton step
// r (1 + (1 - y)/2) squares the relative error (about 2^-43 after it).
__device__ __forceinline__ FF ff_rsqrt(FF x) {
  const float r = rsqrtf(x.h);
  const float r2 = r * r;
  const FF y = ff_mul(x, FF{r2, fmaf(r, r, -r2)});
  const float e = (1.0f - y.h) - y.l;
  return ff_norm(r, 0.5f * r * e);
}

// 1/n, k = 1/n_1 + 1/n_2 and sqrt(k (n - 2)) as float-float pairs (host), n_1, n_2.
struct MomentRecips {
  FF rn, k, ct;
  float n1f, n2f;
};

struct MomentOut {
  double* mean;
  double* inv_norm;
  double* t_obs;
  float* u_obs_m;
  uint8_t* valid;
  float* Xraw;
  uint32_t* status;
};

__device__ __forceinline__ void cp_async_f32(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// Adds d = y - m (exact pair) and d^2 (pair) to the running (high, low) sums.
__device__ __forceinline__ void moment_add(float y, float m, float& Dh, float& Dl, float& Qh,
                                           float& Ql) {
  float dh, dl, sh, se;
  two_sum(y, -m, dh, dl);
  const float p = dh * dh;
  const float pe = fmaf(2.0f * dh, dl, fmaf(dh, dh, -p));
  two_sum(Dh, dh, sh, se);
  Dh = sh;
  Dl += se + dl;
  two_sum(Qh, p, sh, se);
  Qh = sh;
  Ql += se + pe;
}

// One tile of kMV mask voxels starting at j0 (all threads of the CTA enter;
// only warp 0 finishes the per-voxel part).
template <bool kAsync>
__device__ __forceinline__ void moments_tile(const float* __restrict__ X, int64_t n_grid, int n,
                                             int n1, int n_pad, const MomentRecips& rc,
                                             const int64_t* __restrict__ vox_grid, int64_t v,
                                             int64_t j0, const MomentOut& o, float* tile,
                                             float (*part)[8][kMV]) {
  constexpr int LD = kMV + 1;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t j = j0 + lane;
  const int64_t g = j < v ? vox_grid[j] : -1;

  // Load: lane = voxel. From device memory every value of the tile is copied
  // with cp.async at once (n x 32 x 4 bytes in flight per CTA, no registers
  // held); from host memory (read over the host link) kMU subjects per warp
  // go through registers. Each thread reads back only the values it copied.
  const float x0f = g >= 0 ? __ldcs(X + g) : 0.0f;
  const float* xp = X + (g >= 0 ? g : 0);
  if constexpr (kAsync) {
#pragma unroll 4
    for (int s = warp; s < n; s += kMW) {
      float* dst = &tile[s * LD + lane];
      if (g >= 0) cp_async_f32(dst, xp + int64_t(s) * n_grid);
      else *dst = 0.0f;
    }
    cp_async_wait_all();
  } else {
    for (int s0 = warp; s0 < n; s0 += kMU * kMW) {
      float xv[kMU];
#pragma unroll
      for (int q = 0; q < kMU; ++q) {
        const int s = s0 + q * kMW;
        xv[q] = (g >= 0 && s < n) ? __ldcs(xp + int64_t(s) * n_grid) : 0.0f;
      }
#pragma unroll
      for (int q = 0; q < kMU; ++q) {
        const int s = s0 + q * kMW;
        if (s < n) tile[s * LD + lane] = xv[q];
      }
    }
  }

  // Pass 1: FP32 sum (only the seed of the centring: the two-pass correction
  // removes its rounding), minimum, maximum, and sum of x * 0, which is NaN
  // exactly when some x is NaN or infinite. The flags follow at the end (bit
  // 0: NaN or Inf seen, bit 1: not all values equal). A sum that overflows
  // while every value is finite (|x| near the FP32 limit) is retaken on the
  // scaled values.
  float S = 0.0f, fin = 0.0f, xmin = x0f, xmax = x0f;
  {
    const float* col = tile + lane;
#pragma unroll 4
    for (int s = warp; s < n; s += kMW) {
      const float x = col[s * LD];
      S += x;
      fin = fmaf(x, 0.0f, fin);
      xmin = fminf(xmin, x);
      xmax = fmaxf(xmax, x);
    }
  }
  part[warp][0][lane] = xmin;
  part[warp][1][lane] = S;
  part[warp][2][lane] = xmax;
  part[warp][3][lane] = fin;
  __syncthreads();
  // Voxel-major copy: warp w writes rows l = w, w + 8, ... (lane = subject;
  // tile reads at stride LD = 33 words fall in distinct banks).
  for (int l = warp; l < kMV && j0 + l < v; l += kMW) {
    float* dst = o.Xraw + (j0 + l) * n_pad;
    for (int s = lane; s < n_pad; s += 32) dst[s] = s < n ? tile[s * LD + l] : 0.0f;
  }
  S = 0.0f;
  fin = 0.0f;
#pragma unroll
  for (int w = 0; w < kMW; ++w) {
    xmin = fminf(xmin, part[w][0][lane]);
    S += part[w][1][lane];
    xmax = fmaxf(xmax, part[w][2][lane]);
    fin += part[w][3][lane];
  }
  uint32_t fl = fin != fin ? 1u : 0u;
  if (xmin != xmax) fl |= 2u;
  float amax = fmaxf(fabsf(xmin), fabsf(xmax));
  if (fl & 1u) amax = 1.0f;  // reported below; keep the arithmetic finite
  int ex = int((__float_as_uint(amax) >> 23) & 0xffu) - 127;
  ex = ex < -126 ? -126 : (ex > 126 ? 126 : ex);
  const float scale = __uint_as_float(uint32_t(127 - ex) << 23);  // 2^-ex, exact
  const float inv_n = 1.0f / float(n);
  float ms = (S * inv_n) * scale;  // seed mean of the scaled values
  if (__syncthreads_or(!(fabsf(S) <= kFltMax) && !(fl & 1u))) {
    float Ss = 0.0f;  // overflowed sums only: the scaled sum (cannot overflow)
    for (int s = warp; s < n; s += kMW) Ss += tile[s * LD + lane] * scale;
    part[warp][4][lane] = Ss;
    __syncthreads();
    Ss = 0.0f;
#pragma unroll
    for (int w = 0; w < kMW; ++w) Ss += part[w][4][lane];
    if (!(fabsf(S) <= kFltMax)) ms = Ss * inv_n;
  }
  if (fl & 1u) ms = 0.0f;

  // Pass 2: d = y - m exactly as a pair, its square as a pair, and per group
  // D_g and Q_g as (high, accumulated low) pairs: each addition's rounding
  // error is exact (two-sum) and goes into the low word with the value's own
  // low part.
  float D1h = 0.f, D1l = 0.f, D2h = 0.f, D2l = 0.f, Q1h = 0.f, Q1l = 0.f, Q2h = 0.f, Q2l = 0.f;
  const float* col = tile + lane;
  int s = warp;
#pragma unroll 4
  for (; s < n1; s += kMW) moment_add(col[s * LD] * scale, ms, D1h, D1l, Q1h, Q1l);
#pragma unroll 4
  for (; s < n; s += kMW) moment_add(col[s * LD] * scale, ms, D2h, D2l, Q2h, Q2l);
  __syncthreads();  // everyone has read the pass-1 partials (and the tile)
  float* pp = &part[warp][0][0];
  pp[0 * kMV + lane] = D1h;
  pp[1 * kMV + lane] = D1l;
  pp[2 * kMV + lane] = D2h;
  pp[3 * kMV + lane] = D2l;
  pp[4 * kMV + lane] = Q1h;
  pp[5 * kMV + lane] = Q1l;
  pp[6 * kMV + lane] = Q2h;
  pp[7 * kMV + lane] = Q2l;
  __syncthreads();
  if (warp != 0) return;
  D1h = D1l = D2h = D2l = Q1h = Q1l = Q2h = Q2l = 0.0f;
#pragma unroll
  for (int w = 0; w < kMW; ++w) {
    ff_acc(D1h, D1l, part[w][0][lane], part[w][1][lane]);
    ff_acc(D2h, D2l, part[w][2][lane], part[w][3][lane]);
    ff_acc(Q1h, Q1l, part[w][4][lane], part[w][5][lane]);
    ff_acc(Q2h, Q2l, part[w][6][lane], part[w][7][lane]);
  }
  if (j >= v) return;
  if (fl & 1u) {
    atomicOr(o.status, kErrBadData);
    o.valid[j] = 0;
    o.t_obs[j] = nan("");
    return;
  }
  // Finish in float-float; only the outputs are widened to FP64.
  const FF D1{D1h, D1l}, D2{D2h, D2l};
  const FF Dt = ff_add(D1, D2);
  const FF delta = ff_mul(Dt, rc.rn);
  const FF SS = ff_sub(ff_add(FF{Q1h, Q1l}, FF{Q2h, Q2l}), ff_mul(Dt, delta));
  const FF A1 = ff_mul(ff_sub(ff_mulf(D1, rc.n2f), ff_mulf(D2, rc.n1f)), rc.rn);
  // 1/s = 2^ex exactly (ex in [-126, 126])
  const double unscale = __longlong_as_double(int64_t(1023 + ex) << 52);
  const bool ok = (fl & 2u) && SS.h > 0.0f;
  o.valid[j] = ok ? 1 : 0;
  o.mean[j] = ff_d(ff_add(FF{ms, 0.0f}, delta)) * unscale;
  if (!ok) {
    o.inv_norm[j] = 0.0;
    o.t_obs[j] = nan("");
    o.u_obs_m[j] = 0.0f;
    return;
  }
  const FF rs = ff_rsqrt(SS);
  o.inv_norm[j] = ff_d(rs) * double(scale);
  const FF SSw = ff_sub(SS, ff_mul(rc.k, ff_mul(A1, A1)));
  // perfectly separated groups (SS_w = 0): t = +-infinity
  o.t_obs[j] = SSw.h > 0.0f ? ff_d(ff_mul(ff_mul(rc.ct, A1), ff_rsqrt(SSw)))
                            : copysign(double(INFINITY), double(A1.h));
  o.u_obs_m[j] = ff_mul(A1, rs).h;
}

// Persistent over the tiles of the v mask voxels. v comes from the device
// (v_dev, the mask compaction's count) when it is not known on the host; the
// grid is then sized for the largest possible v.
template <bool kAsync>
__global__ void __launch_bounds__(32 * kMW, kAsync ? 8 : 6)
    moments_kernel(const float* __restrict__ X, int64_t n_grid, int n, int n1, int n_pad,
                   const MomentRecips rc, const int64_t* __restrict__ vox_grid, int64_t v_host,
                   const uint32_t* __restrict__ v_dev, const MomentOut o) {
  extern __shared__ float tile[];  // [n][kMV + 1]
  __shared__ float part[kMW][8][kMV];
  const int64_t v = v_dev ? int64_t(*v_dev) : v_host;
  const int64_t tiles = (v + kMV - 1) / kMV;
  for (int64_t t = blockIdx.x; t < tiles; t += gridDim.x) {
    moments_tile<kAsync>(X, n_grid, n, n1, n_pad, rc, vox_grid, v, t * kMV, o, tile, part);
    __syncthreads();  // the tile and the partials are reused
  }
}

// Per compact voxel: the FP64 mean and 1/sqrt(SS) as float pairs (hi + lo),
// and the observed u in compact order.
__global__ void compact_stats_kernel(const int32_t* __restrict__ valid_map, int64_t v_valid,
                                     int64_t v_pad, const double* __restrict__ mean,
                                     const double* __restrict__ inv_norm,
                                     const float* __restrict__ u_obs_m, float4* __restrict__ vstat,
                                     float* __restrict__ u_obs) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < v_pad;
       c += int64_t(gridDim.x) * blockDim.x) {
    float4 st = make_float4(0.f, 0.f, 0.f, 0.f);
    float uo = INFINITY;
    if (c < v_valid) {
      const int32_t j = valid_map[c];
      const double m = mean[j], iv = inv_norm[j];
      st.x = float(m);
      st.y = float(m - double(st.x));
      st.z = float(iv);
      st.w = float(iv - double(st.z));
      uo = u_obs_m[j];
    }
    vstat[c] = st;
    u_obs[c] = uo;
  }
}

// (x - mean) / sqrt(SS) from an FP32 input and float-pair constants, with the
// subtraction exact (two-sum) and the product carried to ~2^-40 before the
// final rounding to FP32.
__device__ __forceinline__ float unit_centre(float x, float4 st) {
  const float s = x - st.x;
  const float bb = s - x;
  const float e = (x - (s - bb)) + (-st.x - bb);  // s + e == x - mean_hi exactly
  const float dl = e - st.y;                      // + low part of -mean
  const float p = s * st.z;
  const float pe = fmaf(s, st.z, -p);             // exact product error
  return p + (pe + fmaf(s, st.w, dl * st.z));
}

__global__ void build_xn32_kernel(const float* __restrict__ Xraw, int n, int n_pad,
                                  const int32_t* __restrict__ valid_map, int64_t v_valid,
                                  int64_t v_pad, const float4* __restrict__ vstat,
                                  float* __restrict__ Xn32) {
  const int64_t total = v_pad * n_pad;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e / n_pad;
    const int s = int(e - c * n_pad);
    float y = 0.0f;
    if (c < v_valid && s < n) y = unit_centre(Xraw[int64_t(valid_map[c]) * n_pad + s], vstat[c]);
    Xn32[e] = y;
  }
}

// BF16 pieces: hi = bf16(y), mid = bf16(y - hi), lo = bf16(y - hi - mid)
// (each residual exact in FP32), stored as 8x8 core matrices, row-group major.
// A CTA takes one row group (8 consecutive compact voxels); a thread builds one
// core-matrix row (8 consecutive subjects of one voxel), so the 8 threads of a
// core matrix store its 128 contiguous bytes together (16-byte stores).
__global__ void build_xnb_kernel(const float* __restrict__ Xraw, int n, int n_pad,
                                 const int32_t* __restrict__ valid_map, int64_t v_valid,
                                 int64_t v_pad, const float4* __restrict__ vstat,
                                 __nv_bfloat16* __restrict__ Xnb) {
  const int kg_n = n_pad >> 3;
  const int64_t piece = v_pad * n_pad;
  const int64_t cg = blockIdx.x;  // row group
  for (int idx = threadIdx.x; idx < kg_n * 8; idx += blockDim.x) {
    const int r = idx & 7, kg = idx >> 3;
    const int64_t c = cg * 8 + r;
    float y[8];
    if (c < v_valid) {
      const float4 st = vstat[c];
      const float4* src =
          reinterpret_cast<const float4*>(Xraw + int64_t(valid_map[c]) * n_pad + kg * 8);
      const float4 a = src[0], b = src[1];
      const float xv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 8; ++q) y[q] = (kg * 8 + q < n) ? unit_centre(xv[q], st) : 0.0f;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) y[q] = 0.0f;
    }
    __align__(16) __nv_bfloat16 hi[8], mid[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      hi[q] = __float2bfloat16_rn(y[q]);
      const float r1 = y[q] - __bfloat162float(hi[q]);
      mid[q] = __float2bfloat16_rn(r1);
      lo[q] = __float2bfloat16_rn(r1 - __bfloat162float(mid[q]));
    }
    const int64_t off = (cg * kg_n + kg) * 64 + r * 8;
    *reinterpret_cast<uint4*>(Xnb + off) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(Xnb + piece + off) = *reinterpret_cast<const uint4*>(mid);
    *reinterpret_cast<uint4*>(Xnb + 2 * piece + off) = *reinterpret_cast<const uint4*>(lo);
  }
}

// FP16 pieces of the scaled value ys = 2^15 y: hi = fp16(ys), lo = fp16(ys - hi)
// (the residual is exact in FP32), same core-matrix layout as the BF16 pieces.
// |y| < 1, so |ys| < 32768 lies in FP16 range; lo carries the next 11 bits.
__global__ void build_xnh_kernel(const float* __restrict__ Xraw, int n, int n_pad,
                                 const int32_t* __restrict__ valid_map, int64_t v_valid,
                                 int64_t v_pad, const float4* __restrict__ vstat,
                                 __half* __restrict__ Xnh) {
  const int kg_n = n_pad >> 3;
  const int64_t piece = v_pad * n_pad;
  const int64_t cg = blockIdx.x;  // row group
  for (int idx = threadIdx.x; idx < kg_n * 8; idx += blockDim.x) {
    const int r = idx & 7, kg = idx >> 3;
    const int64_t c = cg * 8 + r;
    float y[8];
    if (c < v_valid) {
      const float4 st = vstat[c];
      const float4* src =
          reinterpret_cast<const float4*>(Xraw + int64_t(valid_map[c]) * n_pad + kg * 8);
      const float4 a = src[0], b = src[1];
      const float xv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int q = 0; q < 8; ++q)
        y[q] = (kg * 8 + q < n) ? unit_centre(xv[q], st) * kF16Scale : 0.0f;
    } else {
#pragma unroll
      for (int q = 0; q < 8; ++q) y[q] = 0.0f;
    }
    __align__(16) __half hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      hi[q] = __float2half_rn(y[q]);
      lo[q] = __float2half_rn(y[q] - __half2float(hi[q]));
    }
    const int64_t off = (cg * kg_n + kg) * 64 + r * 8;
    *reinterpret_cast<uint4*>(Xnh + off) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(Xnh + piece + off) = *reinterpret_cast<const uint4*>(lo);
  }
}

__global__ void t_obs_to_float_kernel(const double* __restrict__ t64, float* __restrict__ out,
                                      int64_t v) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < v;
       i += int64_t(gridDim.x) * blockDim.x)
    out[i] = float(t64[i]);
}

int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return int(b);
}

FF to_ff(double d) {
  const float h = float(d);
  return FF{h, float(d - double(h))};
}

int sm_count(int dev) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

pt_status nomem(pt_ctx* ctx, const char* what) {
  set_error(ctx, std::string("out of device memory (") + what + ")");
  return PT_ERR_NOMEM;
}

// Positions of nonzero flags, in index order, and (optionally, device) their count.
template <class IdxT>
pt_status compact(pt_ctx* ctx, const uint8_t* flags, int64_t N, IdxT* out, uint32_t** total_dev,
                  Buf& tmp) {
  const int64_t nb = (N + kScanChunk - 1) / kScanChunk;
  if (!tmp.ensure(sizeof(uint32_t) * (nb + 1))) return nomem(ctx, "scan");
  uint32_t* bc = tmp.as<uint32_t>();
  scan_count_kernel<<<unsigned(nb), kScanThreads, 0, ctx->stream>>>(flags, N, bc);
  PT_LAUNCH_CHECK(ctx);
  scan_blocks_kernel<<<1, 1024, 0, ctx->stream>>>(bc, nb);
  PT_LAUNCH_CHECK(ctx);
  if (out) {
    scan_write_kernel<IdxT><<<unsigned(nb), kScanThreads, 0, ctx->stream>>>(flags, N, bc, out);
    PT_LAUNCH_CHECK(ctx);
  }
  *total_dev = bc + nb;
  return PT_OK;
}

}  // namespace

pt_status prepare_impl(pt_ctx* ctx, const float* X, const uint8_t* mask) {
  cudaStream_t st = ctx->stream;
  Buf& tmp = ctx->scratch;  // scan scratch, kept by the context (kernels may still read it)
  Buf tmp2;
  struct Guard {
    Buf* b;
    ~Guard() { b->release(); }
  } guard{&tmp2};
  Buf& mom = ctx->moments;
  if (!ctx->status.ensure(4 * sizeof(uint32_t))) return nomem(ctx, "status");
  PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->status.p, 0, 4 * sizeof(uint32_t), st));

  // 1. masked voxel list (raster order). Its length v stays on the device: the
  //    buffers up to the validity compaction are sized for the whole grid and
  //    the moments kernel reads v itself, so the stream is waited on once, at
  //    the end (the covariate fit sizes its launch by v and waits here).
  const uint32_t* v_dev = nullptr;
  int64_t v_hi = ctx->n_grid;  // v, or an upper bound of it while v_dev is set
  if (!ctx->vox_grid.ensure(sizeof(int64_t) * ctx->n_grid)) return nomem(ctx, "mask");
  if (mask) {
    uint32_t* tot = nullptr;
    pt_status s = compact<int64_t>(ctx, mask, ctx->n_grid, ctx->vox_grid.as<int64_t>(), &tot, tmp);
    if (s != PT_OK) return s;
    if (ctx->glm_q1) {
      uint32_t vh = 0;
      PT_CUDA_TRY(ctx, cudaMemcpyAsync(&vh, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
      PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
      v_hi = vh;
    } else {
      v_dev = tot;
      PT_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->status.as<uint32_t>() + 2, tot, sizeof(uint32_t),
                                       cudaMemcpyDeviceToDevice, st));
    }
  } else {
    iota64_kernel<<<grid_for(ctx->n_grid, 256), 256, 0, st>>>(ctx->vox_grid.as<int64_t>(),
                                                              ctx->n_grid);
    PT_LAUNCH_CHECK(ctx);
  }
  ctx->v = v_hi;  // the covariate fit reads it; replaced by the count below
  const int64_t vv = v_hi > 0 ? v_hi : 1;
  const int n_pad = ctx->n_pad;

  // 2. moments, observed t and u, validity, raw voxel-major copy
  if (!mom.ensure(vv * (2 * sizeof(double) + sizeof(float) + 1) + 64) ||
      !ctx->t_obs64.ensure(sizeof(double) * vv) || !ctx->Xraw.ensure(sizeof(float) * vv * n_pad))
    return nomem(ctx, "moments");
  double* mean = mom.as<double>();
  double* inv_norm = mean + vv;
  float* u_obs_m = reinterpret_cast<float*>(inv_norm + vv);
  uint8_t* valid = reinterpret_cast<uint8_t*>(u_obs_m + vv);
  if (v_hi > 0) {
    // flags past v stay 0 for the compaction over the upper bound
    if (v_dev) PT_CUDA_TRY(ctx, cudaMemsetAsync(valid, 0, size_t(v_hi), st));
    // device-resident X: cp.async tile loads; host memory: register loads
    cudaPointerAttributes pa{};
    const bool on_device = cudaPointerGetAttributes(&pa, X) == cudaSuccess &&
                           (pa.type == cudaMemoryTypeDevice || pa.type == cudaMemoryTypeManaged);
    cudaGetLastError();
    auto kern = on_device ? moments_kernel<true> : moments_kernel<false>;
    // dynamic tile plus 8 KB of static partials: the opt-in is needed from
    // well below 48 KB of dynamic memory, so it is always set
    const int smem = ctx->n * (kMV + 1) * int(sizeof(float));
    PT_CUDA_TRY(ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    int per_sm = 0;
    PT_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * kMW, smem));
    const int64_t tiles = (v_hi + kMV - 1) / kMV;
    const int64_t grid =
        std::min<int64_t>(tiles, int64_t(std::max(per_sm, 1)) * sm_count(ctx->device));
    kern<<<unsigned(grid), 32 * kMW, smem, st>>>(
        X, ctx->n_grid, ctx->n, ctx->n1, n_pad,
        MomentRecips{to_ff(1.0 / ctx->n), to_ff(ctx->k), to_ff(ctx->c_t), float(ctx->n1),
                     float(ctx->n2)},
        ctx->vox_grid.as<int64_t>(), v_hi, v_dev,
        MomentOut{mean, inv_norm, ctx->t_obs64.as<double>(), u_obs_m, valid,
                  ctx->Xraw.as<float>(), ctx->status.as<uint32_t>()});
    PT_LAUNCH_CHECK(ctx);
    if (ctx->glm_q1) {  // covariate-adjusted statistic: residual fit, validity, u/t_obs
      pt_status s = glm_moments(ctx, valid, u_obs_m);
      if (s != PT_OK) return s;
    }
  }

  // 3. compact list of voxels with a defined t (the count, v and the error
  //    bits are read at the single wait below)
  if (!ctx->valid_map.ensure(sizeof(int32_t) * vv)) return nomem(ctx, "valid map");
  uint32_t* vtot = nullptr;
  if (v_hi > 0) {
    pt_status s = compact<int32_t>(ctx, valid, v_hi, ctx->valid_map.as<int32_t>(), &vtot, tmp2);
    if (s != PT_OK) return s;
    PT_CUDA_TRY(ctx, cudaMemcpyAsync(ctx->status.as<uint32_t>() + 1, vtot, sizeof(uint32_t),
                                     cudaMemcpyDeviceToDevice, st));
  }
  uint32_t hb[4] = {0, 0, 0, 0};
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(hb, ctx->status.p, sizeof(hb), cudaMemcpyDeviceToHost, st));
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (v_dev) ctx->v = hb[2];
  if (hb[0] & kErrBadData) {
    set_error(ctx, "pt_prepare: X holds NaN or Inf in a mask voxel");
    return PT_ERR_INVALID;
  }
  ctx->v_valid = hb[1];
  ctx->v_pad = (ctx->v_valid + 255) / 256 * 256;
  if (ctx->v_pad == 0) ctx->v_pad = 256;
  PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->status.as<uint32_t>() + 1, 0, 3 * sizeof(uint32_t), st));

  // 4. per compact voxel constants for the operand builders
  if (!ctx->vstat.ensure(sizeof(float4) * ctx->v_pad) ||
      !ctx->u_obs.ensure(sizeof(float) * ctx->v_pad))
    return nomem(ctx, "voxel constants");
  compact_stats_kernel<<<grid_for(ctx->v_pad, 256), 256, 0, st>>>(
      ctx->valid_map.as<int32_t>(), ctx->v_valid, ctx->v_pad, mean, inv_norm, u_obs_m,
      ctx->vstat.as<float4>(), ctx->u_obs.as<float>());
  PT_LAUNCH_CHECK(ctx);
  ctx->have_xn32 = ctx->have_xnb = false;
  return PT_OK;
}

pt_status ensure_xn32(pt_ctx* ctx) {
  if (ctx->have_xn32) return PT_OK;
  const size_t elems = size_t(ctx->v_pad) * ctx->n_pad;
  if (!ctx->Xn32.ensure(sizeof(float) * elems)) return nomem(ctx, "Xn32");
  build_xn32_kernel<<<grid_for(int64_t(elems), 256), 256, 0, ctx->stream>>>(
      ctx->Xraw.as<float>(), ctx->n, ctx->n_pad, ctx->valid_map.as<int32_t>(), ctx->v_valid,
      ctx->v_pad, ctx->vstat.as<float4>(), ctx->Xn32.as<float>());
  PT_LAUNCH_CHECK(ctx);
  ctx->have_xn32 = true;
  return PT_OK;
}

pt_status ensure_xnb(pt_ctx* ctx, int precision) {
  const bool f16 = precision == PT_PREC_FP16X2;
  if (ctx->have_xnb && ctx->xnb_f16 == f16) return PT_OK;
  ctx->have_xnb = false;
  const size_t elems = size_t(ctx->v_pad) * ctx->n_pad;
  if (!ctx->Xnb.ensure(sizeof(__nv_bfloat16) * 3 * elems)) return nomem(ctx, "Xnb");
  const int xnb_threads = std::min(256, (ctx->n_pad + 31) / 32 * 32);
  if (f16) {
    if (ctx->glm_q1) {
      set_error(ctx, "PT_PREC_FP16X2 is not available with covariates (use BF16X2/X3)");
      return PT_ERR_UNSUPPORTED;
    }
    build_xnh_kernel<<<unsigned(ctx->v_pad / 8), xnb_threads, 0, ctx->stream>>>(
        ctx->Xraw.as<float>(), ctx->n, ctx->n_pad, ctx->valid_map.as<int32_t>(), ctx->v_valid,
        ctx->v_pad, ctx->vstat.as<float4>(), ctx->Xnb.as<__half>());
    PT_LAUNCH_CHECK(ctx);
    ctx->have_xnb = ctx->xnb_f16 = true;
    return PT_OK;
  }
  ctx->xnb_f16 = false;
  if (ctx->glm_q1) {
    pt_status s = glm_build_xnb(ctx);
    if (s == PT_OK) ctx->have_xnb = true;
    return s;
  }
  build_xnb_kernel<<<unsigned(ctx->v_pad / 8), xnb_threads, 0, ctx->stream>>>(
      ctx->Xraw.as<float>(), ctx->n, ctx->n_pad, ctx->valid_map.as<int32_t>(), ctx->v_valid,
      ctx->v_pad, ctx->vstat.as<float4>(), ctx->Xnb.as<__nv_bfloat16>());
  PT_LAUNCH_CHECK(ctx);
  ctx->have_xnb = true;
  return PT_OK;
}

}  // namespace pt

extern "C" pt_status pt_t_obs(pt_ctx* ctx, float* t_obs) {
  if (!ctx || !t_obs) {
    pt::set_error(ctx, "pt_t_obs: NULL argument");
    return PT_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  if (ctx->v > 0) {
    pt::t_obs_to_float_kernel<<<pt::grid_for(ctx->v, 256), 256, 0, ctx->stream>>>(
        ctx->t_obs64.as<double>(), t_obs, ctx->v);
    PT_LAUNCH_CHECK(ctx);
  }
  return PT_OK;
}
