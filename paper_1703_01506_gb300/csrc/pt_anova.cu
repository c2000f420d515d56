// One-way F statistic of g groups under relabellings: the general "stat"
// input of Alg. 1 with several group columns (Sec. 3.2 instantiates it as the
// two-sample t, the case g = 2, where F = t^2).
//
// With the unit-norm centred data Xn of a voxel (mean 0, sum of squares 1) and
// u_h = sum over group h of Xn, SS_between / SS_total = B = sum_h u_h^2 / n_h,
// and because the u_h of all g groups sum to 0, u_g = -(u_1 + ... + u_{g-1}):
//
//   F = (B / (g - 1)) / ((1 - B) / (n - g)),
//
// strictly increasing in B and the same map at every voxel. So the row maximum
// of F is at the row maximum of B, and F >= F_obs <=> B >= B_obs. The g - 1
// group sums come out of the NaivePT contraction as rows (one label row per
// relabelling and group, written as u rows a batch at a time); a reduction
// kernel forms B, the per-row maximum (packed keys) and the exceedance counts;
// the winner's F is recomputed in FP64 from the input values.
//
// With nuisance covariates Z (a context from pt_prepare_glm: Q an orthonormal
// basis of [1, Z], q1 columns, and the unit-norm residual r^ of every voxel on
// it), the statistic is the factor's F in  y = E beta + [1, Z] gamma + e  (E the
// indicators of groups 1..g-1 of the relabelling): with u = E^T r^ (the same
// contraction, on the residual) and M = E^T (I - Q Q^T) E (per relabelling),
//
//   B = u^T M^-1 u = (RSS_reduced - RSS_full) / RSS_reduced,
//   F = (B / (g - 1)) / ((1 - B) / (n - g - q1 + 1)).
//
// M^-1 is formed per relabelling in FP64 (Cholesky); a relabelling whose group
// columns are not independent of [1, Z] has no statistic (error bit).
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>
#include <vector>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {

__global__ void simt_contract_kernel(const float* L, const float* Xn, int n_pad, int64_t P,
                                     int64_t v, int tiles_per_cta, int mode, int two_sided,
                                     const float* u_obs, const uint8_t* rowflag,
                                     unsigned long long* maxkey, uint32_t* cnt, float* uout);

namespace {

constexpr int kMaxGroups = 16;

struct Groups {
  int g;
  int start[kMaxGroups + 1];  // group h = positions [start[h], start[h+1]) of a relabelling row
  float inv_n[kMaxGroups];    // 1 / n_h
};

int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return int(b);
}

// Label rows of relabellings [i0, i0 + nb): row r = (i - i0) rs + h holds a 1
// for every subject of group h (h < g - 1; rows g - 1 <= h < rs are zero).
// layout 0: FP32 rows of n_pad; 1 / 2: BF16 / FP16 core matrices in 128-row
// blocks (as the NaivePT labels). One warp per relabelling; a row that is not
// a permutation sets kErrBadPerm.
__global__ void anova_labels_kernel(const int32_t* __restrict__ perms, int64_t i0, int64_t nb,
                                    int64_t rows_pad, int n, int n_pad, Groups gr, int rs,
                                    int layout, void* __restrict__ Lout,
                                    uint32_t* __restrict__ status) {
  __shared__ uint32_t seen_all[4][32];
  __shared__ uint16_t grp_all[4][1024];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t k = int64_t(blockIdx.x) * 4 + wib;
  const int G1 = gr.g - 1;
  if (k * rs >= rows_pad) return;
  uint32_t* seen = seen_all[wib];
  uint16_t* grp = grp_all[wib];
  seen[lane] = 0u;
  for (int s = lane; s < n; s += 32) grp[s] = 0xffffu;
  __syncwarp();
  bool bad = false;
  if (k < nb) {
    const int32_t* row = perms + (i0 + k) * n;
    for (int q = lane; q < n; q += 32) {
      const int32_t e = row[q];
      if (e < 0 || e >= n) {
        bad = true;
        continue;
      }
      const uint32_t bit = 1u << (e & 31);
      if (atomicOr(&seen[e >> 5], bit) & bit) bad = true;
      int h = 0;
      while (q >= gr.start[h + 1]) ++h;
      grp[e] = uint16_t(h);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kErrBadPerm);
  __syncwarp();
  for (int h = 0; h < rs; ++h) {
    const int64_t r = k * rs + h;
    if (r >= rows_pad) break;
    for (int s = lane; s < n_pad; s += 32) {
      const bool in = k < nb && s < n && h < G1 && grp[s] == h;
      if (layout == 0) {
        static_cast<float*>(Lout)[r * n_pad + s] = in ? 1.0f : 0.0f;
      } else {
        const int64_t off = (r >> 7) * int64_t(128) * n_pad +
                            ((s >> 3) * 16 + ((r & 127) >> 3)) * 64 + (r & 7) * 8 + (s & 7);
        if (layout == 1)
          static_cast<__nv_bfloat16*>(Lout)[off] = __float2bfloat16(in ? 1.0f : 0.0f);
        else
          static_cast<__half*>(Lout)[off] = __float2half(in ? 1.0f : 0.0f);
      }
    }
  }
}

__device__ __forceinline__ float b_of(const float* __restrict__ U, int64_t base, int64_t stride,
                                      const Groups& gr) {
  float tot = 0.0f, b = 0.0f;
  for (int h = 0; h < gr.g - 1; ++h) {
    const float u = U[base + h * stride];
    tot += u;
    b = fmaf(u * u, gr.inv_n[h], b);
  }
  return fmaf(tot * tot, gr.inv_n[gr.g - 1], b);
}

__device__ __forceinline__ double warp_sum_d(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// M^-1 (FP64, (g-1) x (g-1), row-major) of relabellings [0, P) of `perms`, one
// warp per relabelling: S[h][k] = sum over group h of Q[s][k], M = diag(n_h) -
// S S^T, Cholesky M = L L^T on lane 0, M^-1 = L^-T L^-1. A non-positive pivot
// (group columns dependent on [1, Z]) sets kErrGlmSpan and leaves zeros.
__global__ void ancova_minv_kernel(const int32_t* __restrict__ perms, int64_t P, int n,
                                   const double* __restrict__ Q, int q1, Groups gr,
                                   double* __restrict__ Minv, float* __restrict__ wout, int FG,
                                   uint32_t* __restrict__ status) {
  __shared__ double sm[4][kMaxGroups * kMaxGroups];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t i = int64_t(blockIdx.x) * 4 + wib;
  if (i >= P) return;
  const int G1 = gr.g - 1;
  const int32_t* row = perms + i * n;
  bool bad = false;
  for (int q = lane; q < n; q += 32) bad |= row[q] < 0 || row[q] >= n;
  double* M = sm[wib];
  double* out = Minv + i * G1 * G1;
  float* wo = wout ? wout + i * FG * FG : nullptr;
  if (wo)
    for (int e = lane; e < FG * FG; e += 32) wo[e] = 0.0f;
  if (__any_sync(0xffffffffu, bad)) {  // reported by the labels kernel
    for (int e = lane; e < G1 * G1; e += 32) out[e] = 0.0;
    return;
  }
  for (int e = lane; e < G1 * G1; e += 32) M[e] = 0.0;
  __syncwarp();
  for (int k = 0; k < q1; ++k) {
    double S[kMaxGroups - 1];
    for (int h = 0; h < G1; ++h) {
      double acc = 0.0;
      for (int q = gr.start[h] + lane; q < gr.start[h + 1]; q += 32)
        acc += Q[int64_t(row[q]) * q1 + k];
      S[h] = warp_sum_d(acc);
    }
    for (int e = lane; e < G1 * G1; e += 32) {
      const int h = e / G1, c = e - h * G1;
      M[e] -= S[h] * S[c];
    }
    __syncwarp();
  }
  if (lane != 0) return;
  for (int h = 0; h < G1; ++h) M[h * G1 + h] += double(gr.start[h + 1] - gr.start[h]);
  // Cholesky in place (lower triangle), then the inverse into out
  double scale = 0.0;
  for (int h = 0; h < G1; ++h) scale = fmax(scale, M[h * G1 + h]);
  for (int c = 0; c < G1; ++c) {
    double d = M[c * G1 + c];
    for (int k = 0; k < c; ++k) d -= M[c * G1 + k] * M[c * G1 + k];
    if (!(d > 1e-12 * scale)) {
      atomicOr(status, kErrGlmSpan);
      for (int e = 0; e < G1 * G1; ++e) out[e] = 0.0;
      return;
    }
    const double l = sqrt(d);
    M[c * G1 + c] = l;
    for (int r = c + 1; r < G1; ++r) {
      double t = M[r * G1 + c];
      for (int k = 0; k < c; ++k) t -= M[r * G1 + k] * M[c * G1 + k];
      M[r * G1 + c] = t / l;
    }
  }
  // column c of M^-1: solve L y = e_c, then L^T x = y
  for (int c = 0; c < G1; ++c) {
    double y[kMaxGroups - 1];
    for (int r = 0; r < G1; ++r) {
      double t = r == c ? 1.0 : 0.0;
      for (int k = 0; k < r; ++k) t -= M[r * G1 + k] * y[k];
      y[r] = t / M[r * G1 + r];
    }
    for (int r = G1 - 1; r >= 0; --r) {
      double t = y[r];
      for (int k = r + 1; k < G1; ++k) t -= M[k * G1 + r] * y[k];
      y[r] = t / M[r * G1 + r];
    }
    for (int r = 0; r < G1; ++r) {
      out[r * G1 + c] = y[r];
      if (wo) wo[r * FG + c] = float(y[r]);
    }
  }
}

// B_obs per compact voxel from the FG rows of u of the observed labelling, with
// the fused kernel's arithmetic (f_quad), W for the observed labelling.
template <int FG>
__global__ void f_bobs_kernel(const float* __restrict__ U, int64_t V, const float* __restrict__ W,
                              float* __restrict__ bobs) {
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < V;
       j += int64_t(gridDim.x) * blockDim.x) {
    float u[FG];
#pragma unroll
    for (int m = 0; m < FG; ++m) u[m] = U[m * V + j];
    bobs[j] = f_quad<FG>(u, W);
  }
}

// B = u^T M^-1 u over the g - 1 rows (M^-1 of the row's relabelling, FP64 in
// memory, the same for every voxel of the row).
__device__ __forceinline__ float b_of_cov(const float* __restrict__ U, int64_t base,
                                          int64_t stride, int G1, const double* __restrict__ Mi) {
  float u[kMaxGroups - 1];
  for (int h = 0; h < G1; ++h) u[h] = U[base + h * stride];
  float b = 0.0f;
  for (int h = 0; h < G1; ++h) {
    float t = 0.0f;
    for (int k = 0; k < G1; ++k) t = fmaf(float(Mi[h * G1 + k]), u[k], t);
    b = fmaf(u[h], t, b);
  }
  return b;
}

// B of relabellings [0, nb) of the batch over compact voxels: per-row maxima
// (keys[i0 + i]: orderable B << 32 | ~voxel) and counts B >= B_obs (B_obs NULL:
// write B of row 0 to bobs instead). Block = 256 voxels x 16 relabellings.
__global__ void anova_reduce_kernel(const float* __restrict__ U, int64_t nb, int64_t V, Groups gr,
                                    const double* __restrict__ Minv,
                                    const float* __restrict__ b_obs, float* __restrict__ bobs_out,
                                    int64_t i0, unsigned long long* __restrict__ keys,
                                    uint32_t* __restrict__ cnt) {
  __shared__ unsigned long long wk[8];
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  const int64_t r0 = int64_t(blockIdx.y) * 16;
  const int G1 = gr.g - 1;
  const float bo = (j < V && b_obs) ? b_obs[j] : 0.0f;
  uint32_t c = 0;
  for (int q = 0; q < 16; ++q) {
    const int64_t i = r0 + q;
    if (i >= nb) break;
    unsigned long long key = 0ull;
    if (j < V) {
      const float b = Minv ? b_of_cov(U, i * G1 * V + j, V, G1, Minv + (i0 + i) * G1 * G1)
                           : b_of(U, i * G1 * V + j, V, gr);
      if (!b_obs) {
        if (i == 0) bobs_out[j] = b;
      } else {
        if (b >= bo) ++c;
        key = pack_key(b, uint32_t(j));
      }
    }
    if (!b_obs) continue;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long other = __shfl_xor_sync(0xffffffffu, key, o);
      key = other > key ? other : key;
    }
    if ((threadIdx.x & 31) == 0) wk[threadIdx.x >> 5] = key;
    __syncthreads();
    if (threadIdx.x == 0) {
      unsigned long long m = 0ull;
      for (int w = 0; w < int(blockDim.x >> 5); ++w) m = wk[w] > m ? wk[w] : m;
      if (m) atomicMax(keys + i0 + i, m);
    }
    __syncthreads();
  }
  if (b_obs && j < V && c) atomicAdd(cnt + j, c);
}

// Winner's F in FP64 from the input values (two passes per group), one warp
// per relabelling; maxnull = F, argmax = masked voxel index.
__global__ void anova_finalize_kernel(const unsigned long long* __restrict__ keys, int64_t P,
                                      const int32_t* __restrict__ valid_map,
                                      const float* __restrict__ Xraw, int n, int n_pad,
                                      const int32_t* __restrict__ perms, Groups gr,
                                      float* __restrict__ maxnull, int32_t* __restrict__ argmax) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t i = int64_t(blockIdx.x) * 8 + wib; i < P; i += int64_t(gridDim.x) * 8) {
    const unsigned long long key = keys[i];
    if (key == 0ull) {
      if (lane == 0) {
        maxnull[i] = -INFINITY;
        argmax[i] = -1;
      }
      continue;
    }
    const int32_t j = valid_map[unpack_key_index(key)];
    const float* x = Xraw + int64_t(j) * n_pad;
    const int32_t* row = perms + i * n;
    double tot = 0.0;
    for (int q = lane; q < n; q += 32) tot += double(x[q]);
    for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
    const double mean = tot / n;
    double ssb = 0.0, ssw = 0.0;
    for (int h = 0; h < gr.g; ++h) {
      const int a = gr.start[h], b = gr.start[h + 1];
      double s1 = 0.0;
      for (int q = a + lane; q < b; q += 32) {
        const int32_t e = row[q];
        s1 += (e >= 0 && e < n) ? double(x[e]) : 0.0;
      }
      for (int o = 16; o > 0; o >>= 1) s1 += __shfl_xor_sync(0xffffffffu, s1, o);
      const double mh = s1 / double(b - a);
      double s2 = 0.0;
      for (int q = a + lane; q < b; q += 32) {
        const int32_t e = row[q];
        const double d = (e >= 0 && e < n) ? double(x[e]) - mh : 0.0;
        s2 = fma(d, d, s2);
      }
      for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
      ssb += double(b - a) * (mh - mean) * (mh - mean);
      ssw += s2;
    }
    if (lane == 0) {
      maxnull[i] = float((ssb / (gr.g - 1)) / (ssw / (n - gr.g)));
      argmax[i] = j;
    }
  }
}

// With covariates: the winner's F in FP64 from the input values, one warp per
// relabelling: the voxel's residual on [1, Z], its group sums b (groups
// 1..g-1), B = b^T M^-1 b / ||r||^2, F = (B / (g-1)) / ((1 - B) / df).
__global__ void ancova_finalize_kernel(const unsigned long long* __restrict__ keys, int64_t P,
                                       const int32_t* __restrict__ valid_map,
                                       const float* __restrict__ Xraw, int n, int n_pad,
                                       const int32_t* __restrict__ perms, Groups gr,
                                       const double* __restrict__ Q, int q1,
                                       const double* __restrict__ coef,
                                       const double* __restrict__ Minv, double df,
                                       float* __restrict__ maxnull, int32_t* __restrict__ argmax) {
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int G1 = gr.g - 1;
  for (int64_t i = int64_t(blockIdx.x) * 8 + wib; i < P; i += int64_t(gridDim.x) * 8) {
    const unsigned long long key = keys[i];
    if (key == 0ull) {
      if (lane == 0) {
        maxnull[i] = -INFINITY;
        argmax[i] = -1;
      }
      continue;
    }
    const int32_t j = valid_map[unpack_key_index(key)];
    const float* x = Xraw + int64_t(j) * n_pad;
    const double* cj = coef + int64_t(j) * q1;
    const int32_t* row = perms + i * n;
    auto resid = [&](int s) {
      double r = double(x[s]);
      for (int k = 0; k < q1; ++k) r -= Q[int64_t(s) * q1 + k] * cj[k];
      return r;
    };
    double ss = 0.0;
    for (int s = lane; s < n; s += 32) {
      const double r = resid(s);
      ss = fma(r, r, ss);
    }
    ss = warp_sum_d(ss);
    double b[kMaxGroups - 1];
    for (int h = 0; h < G1; ++h) {
      double acc = 0.0;
      for (int q = gr.start[h] + lane; q < gr.start[h + 1]; q += 32) {
        const int32_t e = row[q];
        acc += (e >= 0 && e < n) ? resid(e) : 0.0;
      }
      b[h] = warp_sum_d(acc);
    }
    if (lane != 0) continue;
    const double* Mi = Minv + i * G1 * G1;
    double B = 0.0;
    for (int h = 0; h < G1; ++h) {
      double t = 0.0;
      for (int k = 0; k < G1; ++k) t += Mi[h * G1 + k] * b[k];
      B += b[h] * t;
    }
    B /= ss;
    maxnull[i] = B < 1.0 ? float((B / G1) / ((1.0 - B) / df)) : INFINITY;
    argmax[i] = j;
  }
}

__global__ void anova_scatter_counts_kernel(const uint32_t* __restrict__ cnt, int64_t V,
                                            const int32_t* __restrict__ valid_map,
                                            uint32_t* __restrict__ counts) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < V;
       c += int64_t(gridDim.x) * blockDim.x)
    counts[valid_map[c]] = cnt[c];
}

}  // namespace

pt_status anova_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, const int32_t* sizes, int g,
                     int precision, float* maxnull, int32_t* argmax, uint32_t* counts) {
  const bool cov = ctx->glm_q1 > 0;
  if (cov && precision != PT_PREC_BF16X2 && precision != PT_PREC_BF16X3) {
    set_error(ctx, "pt_maxnull_anova with covariates runs on the BF16X2 / BF16X3 paths");
    return PT_ERR_UNSUPPORTED;
  }
  if (g < 2 || g > kMaxGroups) {
    set_error(ctx, "pt_maxnull_anova: need 2 <= g <= 16 groups");
    return PT_ERR_INVALID;
  }
  Groups gr;
  gr.g = g;
  gr.start[0] = 0;
  for (int h = 0; h < g; ++h) {
    if (sizes[h] < 1) {
      set_error(ctx, "pt_maxnull_anova: every group needs at least one subject");
      return PT_ERR_INVALID;
    }
    gr.start[h + 1] = gr.start[h] + sizes[h];
    gr.inv_n[h] = float(1.0 / sizes[h]);
  }
  // residual degrees of freedom of the full model (g group levels, q1 - 1 covariates)
  const int df = ctx->n - g - (cov ? ctx->glm_q1 - 1 : 0);
  if (gr.start[g] != ctx->n || df < 1) {
    set_error(ctx, "pt_maxnull_anova: group sizes must add up to n, and n - g - q >= 1");
    return PT_ERR_INVALID;
  }
  cudaStream_t st = ctx->stream;
  const int64_t V = ctx->v_valid;
  const int G1 = g - 1;
  if (counts) PT_CUDA_TRY(ctx, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ctx->v, st));
  if (V == 0) {
    std::vector<float> ninf(1, -INFINITY);
    for (int64_t i = 0; i < P; ++i) {
      PT_CUDA_TRY(ctx, cudaMemcpyAsync(maxnull + i, ninf.data(), sizeof(float),
                                       cudaMemcpyHostToDevice, st));
    }
    PT_CUDA_TRY(ctx, cudaMemsetAsync(argmax, 0xFF, sizeof(int32_t) * size_t(P), st));
    return cudaStreamSynchronize(st) == cudaSuccess ? PT_OK : PT_ERR_CUDA;
  }
  const bool tc = precision != PT_PREC_FP32;
  pt_status s = tc ? tc_supported(ctx) : PT_OK;
  if (s == PT_OK) s = tc ? ensure_xnb(ctx, precision) : ensure_xn32(ctx);
  if (s != PT_OK) return s;
  // g - 1 <= 4 on the tensor cores: B formed in the contraction's epilogue
  // (FG label rows per relabelling, adjacent lanes), no rows of u in memory;
  // otherwise rows of u a batch at a time and a reduction kernel.
  const int FG = (tc && G1 <= 4) ? (G1 <= 2 ? 2 : 4) : 0;
  const int rs = FG ? FG : G1;  // label rows per relabelling
  // batch: relabellings whose g - 1 u rows take about 512 MB (all of them when fused)
  int64_t Bp = FG ? (P + 127) / 128 * 128
                  : std::max<int64_t>(128, (int64_t(1) << 27) / (V * G1) / 128 * 128);
  Bp = std::min<int64_t>(Bp, (P + 127) / 128 * 128);
  const int64_t rows_pad_max = (Bp * rs + 127) / 128 * 128;
  const int64_t urows = FG ? 128 : rows_pad_max;  // u rows held at once
  Buf lab, ub, keys, cnt, bobs, ident, minv, minv_id, wall, wid;
  struct Gd {
    std::vector<Buf*> v;
    ~Gd() {
      for (Buf* b : v) b->release();
    }
  } guard{{&lab, &ub, &keys, &cnt, &bobs, &ident, &minv, &minv_id, &wall, &wid}};
  const size_t lab_elem = tc ? 2 : 4;
  if (!lab.ensure(lab_elem * size_t(rows_pad_max) * ctx->n_pad) ||
      !ub.ensure(sizeof(float) * size_t(urows) * V) ||
      !keys.ensure(sizeof(unsigned long long) * size_t(P)) ||
      !cnt.ensure(sizeof(uint32_t) * size_t(V)) || !bobs.ensure(sizeof(float) * size_t(V)) ||
      !ident.ensure(sizeof(int32_t) * ctx->n) ||
      (cov && (!minv.ensure(sizeof(double) * size_t(P) * G1 * G1) ||
               !minv_id.ensure(sizeof(double) * G1 * G1))) ||
      (FG && (!wall.ensure(sizeof(float) * (cov ? size_t(P) : 1) * FG * FG) ||
              !wid.ensure(sizeof(float) * FG * FG)))) {
    set_error(ctx, "out of device memory (one-way F)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemsetAsync(keys.p, 0, sizeof(unsigned long long) * size_t(P), st));
  PT_CUDA_TRY(ctx, cudaMemsetAsync(cnt.p, 0, sizeof(uint32_t) * size_t(V), st));
  {
    std::vector<int32_t> id(ctx->n);
    for (int q = 0; q < ctx->n; ++q) id[q] = q;
    PT_CUDA_TRY(ctx, cudaMemcpyAsync(ident.p, id.data(), sizeof(int32_t) * ctx->n,
                                     cudaMemcpyHostToDevice, st));
  }
  if (cov) {  // M^-1 per relabelling and for the observed labelling (and W = M^-1 padded)
    ancova_minv_kernel<<<unsigned((P + 3) / 4), 128, 0, st>>>(
        perms, P, ctx->n, ctx->glmQ.as<double>(), ctx->glm_q1, gr, minv.as<double>(),
        FG ? wall.as<float>() : nullptr, FG, ctx->status.as<uint32_t>());
    PT_LAUNCH_CHECK(ctx);
    ancova_minv_kernel<<<1, 128, 0, st>>>(ident.as<int32_t>(), 1, ctx->n, ctx->glmQ.as<double>(),
                                          ctx->glm_q1, gr, minv_id.as<double>(),
                                          FG ? wid.as<float>() : nullptr, FG,
                                          ctx->status.as<uint32_t>());
    PT_LAUNCH_CHECK(ctx);
  } else if (FG) {  // W = diag(1/n_h) + (1/n_g) 1 1^T over groups 1..g-1, zero-padded
    std::vector<float> w(size_t(FG) * FG, 0.0f);
    for (int h = 0; h < G1; ++h)
      for (int k = 0; k < G1; ++k)
        w[h * FG + k] = float((h == k ? 1.0 / sizes[h] : 0.0) + 1.0 / sizes[g - 1]);
    PT_CUDA_TRY(ctx, cudaMemcpyAsync(wall.p, w.data(), sizeof(float) * w.size(),
                                     cudaMemcpyHostToDevice, st));
    PT_CUDA_TRY(ctx, cudaMemcpyAsync(wid.p, w.data(), sizeof(float) * w.size(),
                                     cudaMemcpyHostToDevice, st));
  }
  const int layout = prec_label_layout(precision);
  auto labels_of = [&](const int32_t* rp, int64_t i0, int64_t nb) -> int64_t {
    const int64_t rows = nb * rs, rows_pad = (rows + 127) / 128 * 128;
    anova_labels_kernel<<<unsigned((rows_pad / rs + 4) / 4 + 1), 128, 0, st>>>(
        rp, i0, nb, rows_pad, ctx->n, ctx->n_pad, gr, rs, layout, lab.p,
        ctx->status.as<uint32_t>());
    return rows;
  };
  // rows of u for relabellings [i0, i0 + nb) of `rp`
  auto rows_of = [&](const int32_t* rp, int64_t i0, int64_t nb) -> pt_status {
    const int64_t rows = labels_of(rp, i0, nb);
    PT_LAUNCH_CHECK(ctx);
    if (tc) return tc_rows(ctx, lab.p, rows, precision, 1, ub.as<float>(), 0, 0, nullptr, nullptr,
                           nullptr);
    const dim3 grid{unsigned((V + 127) / 128), unsigned((rows + 127) / 128), 1u};
    simt_contract_kernel<<<grid, 256, 0, st>>>(lab.as<float>(), ctx->Xn32.as<float>(), ctx->n_pad,
                                               rows, V, 1, 1, 0, nullptr, nullptr, nullptr,
                                               nullptr, ub.as<float>());
    PT_LAUNCH_CHECK(ctx);
    return PT_OK;
  };
  // observed B: the identity labelling
  s = rows_of(ident.as<int32_t>(), 0, 1);
  if (s != PT_OK) return s;
  if (FG) {
    if (FG == 2)
      f_bobs_kernel<2><<<grid_for(V, 256), 256, 0, st>>>(ub.as<float>(), V, wid.as<float>(),
                                                           bobs.as<float>());
    else
      f_bobs_kernel<4><<<grid_for(V, 256), 256, 0, st>>>(ub.as<float>(), V, wid.as<float>(),
                                                           bobs.as<float>());
    PT_LAUNCH_CHECK(ctx);
    const int64_t rows = labels_of(perms, 0, P);
    PT_LAUNCH_CHECK(ctx);
    s = tc_f_reduce(ctx, lab.p, rows, precision, FG, bobs.as<float>(), wall.as<float>(),
                    cov ? int64_t(FG) * FG : 0, keys.as<unsigned long long>(),
                    cnt.as<uint32_t>());
    if (s != PT_OK) return s;
  } else {
    anova_reduce_kernel<<<dim3(unsigned((V + 255) / 256), 1u, 1u), 256, 0, st>>>(
        ub.as<float>(), 1, V, gr, cov ? minv_id.as<double>() : nullptr, nullptr,
        bobs.as<float>(), 0, nullptr, nullptr);
    PT_LAUNCH_CHECK(ctx);
    for (int64_t i0 = 0; i0 < P; i0 += Bp) {
      const int64_t nb = std::min(Bp, P - i0);
      s = rows_of(perms, i0, nb);
      if (s != PT_OK) return s;
      anova_reduce_kernel<<<dim3(unsigned((V + 255) / 256), unsigned((nb + 15) / 16), 1u), 256,
                            0, st>>>(ub.as<float>(), nb, V, gr,
                                     cov ? minv.as<double>() : nullptr, bobs.as<float>(),
                                     nullptr, i0, keys.as<unsigned long long>(),
                                     cnt.as<uint32_t>());
      PT_LAUNCH_CHECK(ctx);
    }
  }
  if (cov)
    ancova_finalize_kernel<<<grid_for((P + 7) / 8, 1), 256, 0, st>>>(
        keys.as<unsigned long long>(), P, ctx->valid_map.as<int32_t>(), ctx->Xraw.as<float>(),
        ctx->n, ctx->n_pad, perms, gr, ctx->glmQ.as<double>(), ctx->glm_q1,
        ctx->glm_coef.as<double>(), minv.as<double>(), double(df), maxnull, argmax);
  else
    anova_finalize_kernel<<<grid_for((P + 7) / 8, 1), 256, 0, st>>>(
        keys.as<unsigned long long>(), P, ctx->valid_map.as<int32_t>(), ctx->Xraw.as<float>(),
        ctx->n, ctx->n_pad, perms, gr, maxnull, argmax);
  PT_LAUNCH_CHECK(ctx);
  if (counts) {
    anova_scatter_counts_kernel<<<grid_for(V, 256), 256, 0, st>>>(
        cnt.as<uint32_t>(), V, ctx->valid_map.as<int32_t>(), counts);
    PT_LAUNCH_CHECK(ctx);
  }
  // the workspaces are released on return: wait for the kernels that use them
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return PT_OK;
}

}  // namespace pt

extern "C" pt_status pt_maxnull_anova(pt_ctx* ctx, const int32_t* perms, int64_t P,
                                      const int32_t* group_sizes, int32_t g, int32_t precision,
                                      float* maxnull, int32_t* argmax, uint32_t* counts) {
  pt::NvtxRange nvtx_range("pt_maxnull_anova");
  if (!ctx || !perms || !group_sizes || !maxnull || !argmax) {
    pt::set_error(ctx, "pt_maxnull_anova: NULL argument");
    return PT_ERR_INVALID;
  }
  if (P < 1 || P > INT32_MAX || precision < PT_PREC_FP32 || precision > PT_PREC_FP16X2) {
    pt::set_error(ctx, "pt_maxnull_anova: need 1 <= P <= 2^31-1 and a valid precision");
    return PT_ERR_INVALID;
  }
  try {
    cudaSetDevice(ctx->device);
    return pt::anova_impl(ctx, perms, P, group_sizes, g, precision, maxnull, argmax, counts);
  } catch (...) {
    pt::set_error(ctx, "pt_maxnull_anova: internal error");
    return PT_ERR_CUDA;
  }
}
