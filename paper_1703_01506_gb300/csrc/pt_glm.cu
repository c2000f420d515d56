// The two-group statistic with nuisance covariates (the general-contrast
// form of the per-voxel "stat" of Alg. 1; Sec. 3.2 uses the plain two-sample t
// as its instance). For a relabelling with group-1 indicator l and covariates
// Z (intercept added), t is the least-squares t of beta in
//     y = beta l + [1, Z] gamma + e.
// With Q an orthonormal basis of [1, Z] (n x q1), the voxel's residual
// r = y - Q Q^T y, its unit-norm r^ = r / ||r||, and a(l) = ||l||^2 - ||Q^T l||^2:
//     u = l . r^,   w = u / sqrt(a(l)),   t = sqrt(df) w / sqrt(1 - w^2),
// df = n - q1 - 1. For one relabelling t is strictly increasing in u, so the
// fused kernel's row maximum of u is the row maximum of t; the exceedance test
// t >= t_obs becomes u sqrt(a_obs / a(l)) >= u_obs, one multiply by a
// per-relabelling factor. The contraction itself is unchanged: 0/1 labels
// times the BF16 pieces of r^.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {

namespace {

__device__ __forceinline__ double warp_sum(double x) {
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// One warp per masked voxel: coefficients c = Q^T x, residual sums, validity,
// observed u and t (FP64 throughout).
__global__ void glm_moments_kernel(const float* __restrict__ Xraw, int n, int n1, int n_pad,
                                   const double* __restrict__ Q, int q1, int64_t v,
                                   double a_obs, double df, uint8_t* __restrict__ valid,
                                   double* __restrict__ coef, double* __restrict__ inv_r,
                                   float* __restrict__ u_obs_m, double* __restrict__ t_obs) {
  const int lane = threadIdx.x & 31;
  const int64_t j = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (j >= v) return;
  const float* x = Xraw + j * n_pad;
  double sx = 0.0;
  for (int s = lane; s < n; s += 32) sx += double(x[s]);
  const double mean = warp_sum(sx) / double(n);
  double ssc = 0.0;
  for (int s = lane; s < n; s += 32) {
    const double d = double(x[s]) - mean;
    ssc += d * d;
  }
  ssc = warp_sum(ssc);
  double c[kGlmMaxQ1];
  for (int k = 0; k < q1; ++k) {
    double acc = 0.0;
    for (int s = lane; s < n; s += 32) acc += Q[s * q1 + k] * double(x[s]);
    c[k] = warp_sum(acc);
  }
  double ssr = 0.0, g1 = 0.0;
  for (int s = lane; s < n; s += 32) {
    double r = double(x[s]);
    for (int k = 0; k < q1; ++k) r -= Q[s * q1 + k] * c[k];
    ssr += r * r;
    if (s < n1) g1 += r;
  }
  ssr = warp_sum(ssr);
  g1 = warp_sum(g1);
  if (lane != 0) return;
  for (int k = 0; k < q1; ++k) coef[j * q1 + k] = c[k];
  const bool ok = valid[j] && ssr > 1e-24 * ssc;
  valid[j] = ok ? 1 : 0;
  if (!ok) {
    inv_r[j] = 0.0;
    u_obs_m[j] = 0.0f;
    t_obs[j] = nan("");
    return;
  }
  const double ir = 1.0 / sqrt(ssr);
  inv_r[j] = ir;
  const double u = g1 * ir;
  u_obs_m[j] = float(u);
  const double w = u / sqrt(a_obs);
  t_obs[j] = w * w < 1.0 ? sqrt(df) * w / sqrt(1.0 - w * w) : (w > 0.0 ? INFINITY : -INFINITY);
}

// BF16 pieces of the unit-norm residual, 8x8 core matrices, row-group major
// (the layout of build_xnb_kernel): one CTA per row group of 8 compact voxels,
// one thread per core-matrix row.
__global__ void glm_build_xnb_kernel(const float* __restrict__ Xraw, int n, int n_pad,
                                     const int32_t* __restrict__ valid_map, int64_t v_valid,
                                     int64_t v_pad, const double* __restrict__ Q, int q1,
                                     const double* __restrict__ coef,
                                     const double* __restrict__ inv_r,
                                     __nv_bfloat16* __restrict__ Xnb) {
  const int kg_n = n_pad >> 3;
  const int64_t piece = v_pad * n_pad;
  const int64_t cg = blockIdx.x;
  for (int idx = threadIdx.x; idx < kg_n * 8; idx += blockDim.x) {
    const int r8 = idx & 7, kg = idx >> 3;
    const int64_t c = cg * 8 + r8;
    float y[8];
    if (c < v_valid) {
      const int64_t j = valid_map[c];
      const float* x = Xraw + j * n_pad;
      const double ir = inv_r[j];
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const int s = kg * 8 + e;
        double r = 0.0;
        if (s < n) {
          r = double(x[s]);
          for (int k = 0; k < q1; ++k) r -= Q[s * q1 + k] * coef[j * q1 + k];
        }
        y[e] = float(r * ir);
      }
    } else {
#pragma unroll
      for (int e = 0; e < 8; ++e) y[e] = 0.0f;
    }
    __align__(16) __nv_bfloat16 hi[8], mid[8], lo[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      hi[e] = __float2bfloat16_rn(y[e]);
      const float r1 = y[e] - __bfloat162float(hi[e]);
      mid[e] = __float2bfloat16_rn(r1);
      lo[e] = __float2bfloat16_rn(r1 - __bfloat162float(mid[e]));
    }
    const int64_t off = (cg * kg_n + kg) * 64 + r8 * 8;
    *reinterpret_cast<uint4*>(Xnb + off) = *reinterpret_cast<const uint4*>(hi);
    *reinterpret_cast<uint4*>(Xnb + piece + off) = *reinterpret_cast<const uint4*>(mid);
    *reinterpret_cast<uint4*>(Xnb + 2 * piece + off) = *reinterpret_cast<const uint4*>(lo);
  }
}

// a(l) = n1 - ||Q^T l||^2 for the group-1 set of one relabelling row, summed by
// one warp (every lane returns the same value).
__device__ double glm_scale_a(const int32_t* row, int n1, const double* Q, int q1, int lane) {
  double a = double(n1);
  for (int k = 0; k < q1; ++k) {
    double acc = 0.0;
    for (int e = lane; e < n1; e += 32) acc += Q[int64_t(row[e]) * q1 + k];
    acc = warp_sum(acc);
    a -= acc * acc;
  }
  return a;
}

// One warp per relabelling row: the factor sqrt(a_obs / a(l)) of the
// exceedance test (1 for padded rows). A row whose group column lies in the
// span of the covariates has no statistic: error bit, factor 1.
__global__ void glm_rowscale_kernel(const int32_t* __restrict__ perms, int64_t P, int64_t P_pad,
                                    int n, int n1, const double* __restrict__ Q, int q1,
                                    double a_obs, float* __restrict__ scale,
                                    uint32_t* __restrict__ status) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (i >= P_pad) return;
  if (i >= P) {
    if (lane == 0) scale[i] = 1.0f;
    return;
  }
  const int32_t* row = perms + i * n;
  bool bad = false;
  for (int e = lane; e < n1; e += 32) bad |= row[e] < 0 || row[e] >= n;
  if (__any_sync(0xffffffffu, bad)) {  // reported by the labels kernel
    if (lane == 0) scale[i] = 1.0f;
    return;
  }
  const double a = glm_scale_a(row, n1, Q, q1, lane);
  if (lane != 0) return;
  if (!(a > 1e-12 * double(n1))) {
    atomicOr(status, kErrGlmSpan);
    scale[i] = 1.0f;
    return;
  }
  scale[i] = float(sqrt(a_obs / a));
}

// Winner statistic of every row in FP64 from the input values (one warp per
// row): residual of the winning voxel, u over the row's group 1, a(l), t.
__global__ void glm_finalize_kernel(const unsigned long long* __restrict__ maxkey, int64_t P,
                                    const int32_t* __restrict__ valid_map,
                                    const float* __restrict__ Xraw, int n, int n1, int n_pad,
                                    const int32_t* __restrict__ perms, int two_sided,
                                    const double* __restrict__ Q, int q1,
                                    const double* __restrict__ coef,
                                    const double* __restrict__ inv_r, double df,
                                    float* __restrict__ maxnull, int32_t* __restrict__ argmax) {
  const int lane = threadIdx.x & 31;
  const int64_t i = (int64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (i >= P) return;
  const unsigned long long key = maxkey[i];
  if (key == 0ull) {
    if (lane == 0) {
      maxnull[i] = -INFINITY;
      argmax[i] = -1;
    }
    return;
  }
  const int64_t j = valid_map[unpack_key_index(key)];
  const float* x = Xraw + j * n_pad;
  const int32_t* row = perms + i * n;
  bool bad = false;
  for (int e = lane; e < n1; e += 32) bad |= row[e] < 0 || row[e] >= n;
  if (__any_sync(0xffffffffu, bad)) {  // reported by the labels kernel
    if (lane == 0) {
      maxnull[i] = nanf("");
      argmax[i] = -1;
    }
    return;
  }
  double g = 0.0;
  for (int e = lane; e < n1; e += 32) {
    const int s = row[e];
    double r = double(x[s]);
    for (int k = 0; k < q1; ++k) r -= Q[int64_t(s) * q1 + k] * coef[j * q1 + k];
    g += r;
  }
  g = warp_sum(g);
  const double a = glm_scale_a(row, n1, Q, q1, lane);
  if (lane != 0) return;
  const double w = g * inv_r[j] / sqrt(a);
  double t = w * w < 1.0 ? sqrt(df) * w / sqrt(1.0 - w * w) : (w > 0.0 ? INFINITY : -INFINITY);
  maxnull[i] = float(two_sided ? fabs(t) : t);
  argmax[i] = int32_t(j);
}

}  // namespace

// Orthonormal basis of [1, Z] (modified Gram-Schmidt, each column
// orthogonalised twice), its rank check, and a(observed group).
pt_status glm_setup(pt_ctx* ctx, const double* Z, int q) {
  const int n = ctx->n, q1 = q + 1;
  std::vector<double> B(size_t(n) * q1);
  for (int s = 0; s < n; ++s) {
    B[size_t(s) * q1] = 1.0;
    for (int k = 0; k < q; ++k) {
      const double z = Z[size_t(s) * q + k];
      if (!std::isfinite(z)) {
        set_error(ctx, "pt_prepare_glm: Z holds NaN or Inf");
        return PT_ERR_INVALID;
      }
      B[size_t(s) * q1 + 1 + k] = z;
    }
  }
  for (int k = 0; k < q1; ++k) {
    double n0 = 0.0;
    for (int s = 0; s < n; ++s) n0 += B[size_t(s) * q1 + k] * B[size_t(s) * q1 + k];
    for (int pass = 0; pass < 2; ++pass)
      for (int m = 0; m < k; ++m) {
        double d = 0.0;
        for (int s = 0; s < n; ++s) d += B[size_t(s) * q1 + m] * B[size_t(s) * q1 + k];
        for (int s = 0; s < n; ++s) B[size_t(s) * q1 + k] -= d * B[size_t(s) * q1 + m];
      }
    double nk = 0.0;
    for (int s = 0; s < n; ++s) nk += B[size_t(s) * q1 + k] * B[size_t(s) * q1 + k];
    if (!(nk > 1e-20 * n0) || !(n0 > 0.0)) {
      set_error(ctx, "pt_prepare_glm: [1, Z] does not have full column rank");
      return PT_ERR_INVALID;
    }
    const double inv = 1.0 / std::sqrt(nk);
    for (int s = 0; s < n; ++s) B[size_t(s) * q1 + k] *= inv;
  }
  double a = double(ctx->n1);
  for (int k = 0; k < q1; ++k) {
    double acc = 0.0;
    for (int s = 0; s < ctx->n1; ++s) acc += B[size_t(s) * q1 + k];
    a -= acc * acc;
  }
  if (!(a > 1e-12 * ctx->n1)) {
    set_error(ctx, "pt_prepare_glm: the observed group column lies in the span of [1, Z]");
    return PT_ERR_INVALID;
  }
  if (!ctx->glmQ.ensure(sizeof(double) * B.size())) {
    set_error(ctx, "out of device memory (covariate basis)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemcpy(ctx->glmQ.p, B.data(), sizeof(double) * B.size(),
                              cudaMemcpyHostToDevice));
  ctx->glm_q1 = q1;
  ctx->glm_a_obs = a;
  ctx->glm_df = double(n - q1 - 1);
  return PT_OK;
}

pt_status glm_moments(pt_ctx* ctx, uint8_t* valid, float* u_obs_m) {
  const int64_t v = ctx->v;
  if (v < 1) return PT_OK;
  if (!ctx->glm_coef.ensure(sizeof(double) * size_t(v) * ctx->glm_q1) ||
      !ctx->glm_inv.ensure(sizeof(double) * size_t(v))) {
    set_error(ctx, "out of device memory (covariate fit)");
    return PT_ERR_NOMEM;
  }
  const int64_t blocks = (v * 32 + 255) / 256;
  glm_moments_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(
      ctx->Xraw.as<float>(), ctx->n, ctx->n1, ctx->n_pad, ctx->glmQ.as<double>(), ctx->glm_q1,
      v, ctx->glm_a_obs, ctx->glm_df, valid, ctx->glm_coef.as<double>(),
      ctx->glm_inv.as<double>(), u_obs_m, ctx->t_obs64.as<double>());
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

pt_status glm_build_xnb(pt_ctx* ctx) {
  const int threads = std::min(256, (ctx->n_pad + 31) / 32 * 32);
  glm_build_xnb_kernel<<<unsigned(ctx->v_pad / 8), threads, 0, ctx->stream>>>(
      ctx->Xraw.as<float>(), ctx->n, ctx->n_pad, ctx->valid_map.as<int32_t>(), ctx->v_valid,
      ctx->v_pad, ctx->glmQ.as<double>(), ctx->glm_q1, ctx->glm_coef.as<double>(),
      ctx->glm_inv.as<double>(), ctx->Xnb.as<__nv_bfloat16>());
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

pt_status glm_rowscale(pt_ctx* ctx, const int32_t* perms, int64_t P, int64_t P_pad) {
  if (!ctx->rowscale.ensure(sizeof(float) * size_t(P_pad))) {
    set_error(ctx, "out of device memory (relabelling scales)");
    return PT_ERR_NOMEM;
  }
  const int64_t blocks = (P_pad * 32 + 255) / 256;
  glm_rowscale_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(
      perms, P, P_pad, ctx->n, ctx->n1, ctx->glmQ.as<double>(), ctx->glm_q1, ctx->glm_a_obs,
      ctx->rowscale.as<float>(), ctx->status.as<uint32_t>());
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

pt_status glm_finalize(pt_ctx* ctx, const int32_t* perms, int64_t P, int two_sided,
                       float* maxnull, int32_t* argmax) {
  const int64_t blocks = (P * 32 + 255) / 256;
  glm_finalize_kernel<<<unsigned(blocks), 256, 0, ctx->stream>>>(
      ctx->maxkey.as<unsigned long long>(), P, ctx->valid_map.as<int32_t>(),
      ctx->Xraw.as<float>(), ctx->n, ctx->n1, ctx->n_pad, perms, two_sided,
      ctx->glmQ.as<double>(), ctx->glm_q1, ctx->glm_coef.as<double>(), ctx->glm_inv.as<double>(),
      ctx->glm_df, maxnull, argmax);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

}  // namespace pt
