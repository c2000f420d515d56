// pt_prepare: mask compaction, FP64 per-voxel moments, observed t, and the
// unit-norm centred data Xn in FP32 and as BF16 pieces (blocked 8x8 layout
// consumed directly by the tensor-core kernel).
//
// With x the n values of a voxel, mean and SS = sum (x - mean)^2 in FP64:
//   Xn_s = (x_s - mean) / sqrt(SS),      so sum_s Xn_s = 0 and sum_s Xn_s^2 = 1.
// For a relabelling with group-1 sum u = sum_{s in G1} Xn_s the pooled t of
// Eq. (5) is t = sqrt(k (n-2)) u / sqrt(1 - k u^2), k = 1/n1 + 1/n2, because
// mean1 - mean2 = k s1 and the within-group SS = SS - k s1^2 with s1 = u sqrt(SS).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <string>

#include "pt_internal.h"

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

// One thread per masked voxel: FP64 two-pass moments, observed t, validity.
__global__ void moments_kernel(const float* __restrict__ X, int64_t n_grid, int n, int n1,
                               const int64_t* __restrict__ vox_grid, int64_t v,
                               double* __restrict__ mean_out, double* __restrict__ inv_norm_out,
                               double* __restrict__ t_obs, uint8_t* __restrict__ valid,
                               uint32_t* __restrict__ status) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= v) return;
  const int64_t g = vox_grid[j];
  const float* x = X + g;
  double sum = 0.0, sum1 = 0.0;
  bool finite = true;
  for (int s = 0; s < n; ++s) {
    const float xs = x[int64_t(s) * n_grid];
    finite = finite && isfinite(xs);
    sum += double(xs);
    if (s < n1) sum1 += double(xs);
  }
  if (!finite) {
    atomicOr(status, kErrBadData);
    valid[j] = 0;
    t_obs[j] = nan("");
    return;
  }
  const double mean = sum / n;
  const double sum2 = sum - sum1;  // not used for t (two-pass below keeps subject order)
  (void)sum2;
  double ss = 0.0, s1 = 0.0, s2 = 0.0;
  for (int s = 0; s < n; ++s) {
    const double xs = double(x[int64_t(s) * n_grid]);
    const double d = xs - mean;
    ss += d * d;
    if (s < n1) s1 += xs;
    else s2 += xs;
  }
  const bool ok = ss > 0.0;
  valid[j] = ok ? 1 : 0;
  mean_out[j] = mean;
  inv_norm_out[j] = ok ? 1.0 / sqrt(ss) : 0.0;
  if (!ok) {
    t_obs[j] = nan("");
    return;
  }
  // Observed statistic, Eq. (5) with pooled variances, identity labelling.
  const int n2 = n - n1;
  const double m1 = s1 / n1, m2 = s2 / n2;
  double ssw = 0.0;
  for (int s = 0; s < n; ++s) {
    const double d = double(x[int64_t(s) * n_grid]) - (s < n1 ? m1 : m2);
    ssw += d * d;
  }
  const double sp2 = ssw / double(n - 2);
  t_obs[j] = (m1 - m2) / sqrt(sp2 * (1.0 / n1 + 1.0 / n2));
}

// Element (c, s) of the compact unit-norm data: FP32 copy and BF16 pieces.
__global__ void normalize_kernel(const float* __restrict__ X, int64_t n_grid, int n, int n_pad,
                                 const int64_t* __restrict__ vox_grid,
                                 const int32_t* __restrict__ valid_map, int64_t v_valid,
                                 int64_t v_pad, const double* __restrict__ mean,
                                 const double* __restrict__ inv_norm, float* __restrict__ Xn32,
                                 __nv_bfloat16* __restrict__ Xnb, float* __restrict__ Xraw) {
  const int64_t total = v_pad * n_pad;
  const int64_t piece = v_pad * n_pad;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e / n_pad;
    const int s = int(e - c * n_pad);
    double xd = 0.0;
    float xr = 0.0f;
    if (c < v_valid && s < n) {
      const int32_t j = valid_map[c];
      const int64_t g = vox_grid[j];
      xr = X[int64_t(s) * n_grid + g];
      xd = (double(xr) - mean[j]) * inv_norm[j];
    }
    Xraw[e] = xr;
    Xn32[e] = float(xd);
    const __nv_bfloat16 hi = __double2bfloat16(xd);
    const double r1 = xd - double(__bfloat162float(hi));
    const __nv_bfloat16 mid = __double2bfloat16(r1);
    const double r2 = r1 - double(__bfloat162float(mid));
    const __nv_bfloat16 lo = __double2bfloat16(r2);
    const int64_t off = ((c >> 3) * (n_pad >> 3) + (s >> 3)) * 64 + (c & 7) * 8 + (s & 7);
    Xnb[off] = hi;
    Xnb[piece + off] = mid;
    Xnb[2 * piece + off] = lo;
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
  if (b > 148 * 64) b = 148 * 64;
  return int(b);
}

// Positions of nonzero flags, in index order. Synchronises to read the total.
template <class IdxT>
pt_status compact(pt_ctx* ctx, const uint8_t* flags, int64_t N, IdxT* out, int64_t* total,
                  Buf& tmp) {
  const int64_t nb = (N + kScanChunk - 1) / kScanChunk;
  if (!tmp.ensure(sizeof(uint32_t) * (nb + 1))) {
    set_error(ctx, "pt_prepare: out of device memory");
    return PT_ERR_NOMEM;
  }
  uint32_t* bc = tmp.as<uint32_t>();
  scan_count_kernel<<<unsigned(nb), kScanThreads, 0, ctx->stream>>>(flags, N, bc);
  PT_LAUNCH_CHECK(ctx);
  scan_blocks_kernel<<<1, 1024, 0, ctx->stream>>>(bc, nb);
  PT_LAUNCH_CHECK(ctx);
  if (out) {
    scan_write_kernel<IdxT><<<unsigned(nb), kScanThreads, 0, ctx->stream>>>(flags, N, bc, out);
    PT_LAUNCH_CHECK(ctx);
  }
  uint32_t tot = 0;
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(&tot, bc + nb, sizeof(uint32_t), cudaMemcpyDeviceToHost,
                                   ctx->stream));
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  *total = tot;
  return PT_OK;
}

}  // namespace

pt_status prepare_impl(pt_ctx* ctx, const float* X, const uint8_t* mask) {
  cudaStream_t st = ctx->stream;
  Buf tmp;
  struct Guard {
    Buf* b;
    ~Guard() { b->release(); }
  } guard{&tmp};
  if (!ctx->status.ensure(sizeof(uint32_t))) {
    set_error(ctx, "pt_prepare: out of device memory");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->status.p, 0, sizeof(uint32_t), st));

  // 1. masked voxel list (raster order)
  if (mask) {
    int64_t v = 0;
    pt_status s = compact<int64_t>(ctx, mask, ctx->n_grid, nullptr, &v, tmp);
    if (s != PT_OK) return s;
    ctx->v = v;
    if (!ctx->vox_grid.ensure(sizeof(int64_t) * (v > 0 ? v : 1))) {
      set_error(ctx, "pt_prepare: out of device memory");
      return PT_ERR_NOMEM;
    }
    s = compact<int64_t>(ctx, mask, ctx->n_grid, ctx->vox_grid.as<int64_t>(), &v, tmp);
    if (s != PT_OK) return s;
  } else {
    ctx->v = ctx->n_grid;
    if (!ctx->vox_grid.ensure(sizeof(int64_t) * ctx->v)) {
      set_error(ctx, "pt_prepare: out of device memory");
      return PT_ERR_NOMEM;
    }
    iota64_kernel<<<grid_for(ctx->v, 256), 256, 0, st>>>(ctx->vox_grid.as<int64_t>(), ctx->v);
    PT_LAUNCH_CHECK(ctx);
  }
  const int64_t v = ctx->v;
  const int64_t vv = v > 0 ? v : 1;

  // 2. FP64 moments, observed t, validity
  Buf mom;
  struct Guard2 {
    Buf* b;
    ~Guard2() { b->release(); }
  } guard2{&mom};
  if (!mom.ensure(vv * (2 * sizeof(double) + 1) + 64) || !ctx->t_obs64.ensure(sizeof(double) * vv)) {
    set_error(ctx, "pt_prepare: out of device memory");
    return PT_ERR_NOMEM;
  }
  double* mean = mom.as<double>();
  double* inv_norm = mean + vv;
  uint8_t* valid = reinterpret_cast<uint8_t*>(inv_norm + vv);
  if (v > 0) {
    moments_kernel<<<unsigned((v + 127) / 128), 128, 0, st>>>(
        X, ctx->n_grid, ctx->n, ctx->n1, ctx->vox_grid.as<int64_t>(), v, mean, inv_norm,
        ctx->t_obs64.as<double>(), valid, ctx->status.as<uint32_t>());
    PT_LAUNCH_CHECK(ctx);
  }
  uint32_t bits = 0;
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(&bits, ctx->status.p, sizeof(bits), cudaMemcpyDeviceToHost, st));
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  if (bits & kErrBadData) {
    set_error(ctx, "pt_prepare: X holds NaN or Inf in a mask voxel");
    return PT_ERR_INVALID;
  }

  // 3. compact list of voxels with a defined t
  int64_t vval = 0;
  if (v > 0) {
    pt_status s = compact<int32_t>(ctx, valid, v, nullptr, &vval, tmp);
    if (s != PT_OK) return s;
  }
  ctx->v_valid = vval;
  ctx->v_pad = (vval + 255) / 256 * 256;
  if (ctx->v_pad == 0) ctx->v_pad = 256;
  if (!ctx->valid_map.ensure(sizeof(int32_t) * (vval > 0 ? vval : 1))) {
    set_error(ctx, "pt_prepare: out of device memory");
    return PT_ERR_NOMEM;
  }
  if (vval > 0) {
    pt_status s = compact<int32_t>(ctx, valid, v, ctx->valid_map.as<int32_t>(), &vval, tmp);
    if (s != PT_OK) return s;
  }

  // 4. unit-norm centred data, FP32 and BF16 pieces
  const size_t elems = size_t(ctx->v_pad) * ctx->n_pad;
  if (!ctx->Xn32.ensure(sizeof(float) * elems) || !ctx->Xraw.ensure(sizeof(float) * elems) ||
      !ctx->Xnb.ensure(sizeof(__nv_bfloat16) * 3 * elems)) {
    set_error(ctx, "pt_prepare: out of device memory");
    return PT_ERR_NOMEM;
  }
  normalize_kernel<<<grid_for(int64_t(elems), 256), 256, 0, st>>>(
      X, ctx->n_grid, ctx->n, ctx->n_pad, ctx->vox_grid.as<int64_t>(),
      ctx->valid_map.as<int32_t>(), ctx->v_valid, ctx->v_pad, mean, inv_norm,
      ctx->Xn32.as<float>(), ctx->Xnb.as<__nv_bfloat16>(), ctx->Xraw.as<float>());
  PT_LAUNCH_CHECK(ctx);
  for (auto& o : ctx->obs) o.valid = false;
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
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
