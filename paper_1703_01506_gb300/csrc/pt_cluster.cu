// Cluster-level summaries of thresholded statistic maps (the cluster tables of
// Sec. 6, Figs. 8-9), and the largest cluster under each relabelling: the
// cluster-level counterpart of the max-null (Sec. 2).
//
// A voxel is active when its statistic reaches the threshold tau; clusters are
// the connected sets of active mask voxels on the 3D grid under 6-, 18- or
// 26-connectivity. Through the monotone map of each relabelling the test
// t >= tau is u >= u(tau), u = tau / sqrt(k (n-2) + k tau^2), so the rows come
// from the NaivePT contraction writing u (a batch of relabellings at a time)
// and never as t.
//
// Components by union-find over compact voxel indices, one label array per
// relabelling of the batch: a link always points to a smaller index, so a
// root is the smallest voxel of its component, every find walks strictly
// decreasing indices and every unite retries on a strictly smaller index.
// Nothing waits on another thread; links are made with atomicMin and read
// through L2 (__ldcg), where the atomics land.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {

// Rows of u for relabellings (launchers of pt_naive.cu / pt_naive_tc.cu).
__global__ void simt_contract_kernel(const float* L, const float* Xn, int n_pad, int64_t P,
                                     int64_t v, int tiles_per_cta, int mode, int two_sided,
                                     const float* u_obs, const uint8_t* rowflag,
                                     unsigned long long* maxkey, uint32_t* cnt, float* uout);

namespace {

// Forward half of the neighbourhood (lexicographically positive offsets):
// 6-connectivity uses the first 3, 18 the first 9, 26 all 13.
__constant__ int8_t kOffsets[13][3] = {{0, 0, 1}, {0, 1, 0}, {1, 0, 0},              // faces
                                       {0, 1, 1}, {0, 1, -1}, {1, 0, 1}, {1, 0, -1},
                                       {1, 1, 0}, {1, -1, 0},                         // edges
                                       {1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};  // corners

int n_offsets(int connectivity) { return connectivity == 6 ? 3 : connectivity == 18 ? 9 : 13; }

int grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 64) b = 152 * 64;
  return int(b);
}

__global__ void grid_inv_fill_kernel(int32_t* __restrict__ inv, int64_t n_grid) {
  for (int64_t g = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; g < n_grid;
       g += int64_t(gridDim.x) * blockDim.x)
    inv[g] = -1;
}

__global__ void grid_inv_set_kernel(const int64_t* __restrict__ vox_grid,
                                    const int32_t* __restrict__ valid_map, int64_t V,
                                    int32_t* __restrict__ inv) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < V;
       c += int64_t(gridDim.x) * blockDim.x)
    inv[vox_grid[valid_map[c]]] = int32_t(c);
}

// L (in place over the u rows, B x V) = c where u >= u_tau, else -1.
__global__ void cc_init_kernel(float* __restrict__ U, int64_t total, int64_t V, float u_tau) {
  int32_t* L = reinterpret_cast<int32_t*>(U);
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float u = U[e];
    L[e] = u >= u_tau ? int32_t(e % V) : -1;
  }
}

__device__ __forceinline__ int32_t cc_find(const int32_t* L, int32_t x) {
  int32_t y = __ldcg(L + x);
  while (y != x) {  // y < x: strictly decreasing walk to the root
    x = y;
    y = __ldcg(L + x);
  }
  return x;
}

__device__ __forceinline__ void cc_unite(int32_t* L, int32_t a, int32_t b) {
  while (true) {
    a = cc_find(L, a);
    b = cc_find(L, b);
    if (a == b) return;
    if (a > b) {
      const int32_t t = a;
      a = b;
      b = t;
    }
    const int32_t old = atomicMin(L + b, a);  // link the larger root under the smaller
    if (old == b) return;
    b = old;  // b was linked meanwhile (old < b): unite a with where it went
  }
}

__global__ void cc_union_kernel(int32_t* __restrict__ L, int64_t total, int64_t V,
                                const int32_t* __restrict__ valid_map,
                                const int64_t* __restrict__ vox_grid,
                                const int32_t* __restrict__ inv, int64_t d0, int64_t d1,
                                int64_t d2, int noff) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (__ldcg(L + e) < 0) continue;
    const int64_t b = e / V;
    const int32_t c = int32_t(e - b * V);
    int32_t* Lb = L + b * V;
    const int64_t g = vox_grid[valid_map[c]];
    const int64_t i2 = g % d2, i1 = (g / d2) % d1, i0 = g / (d1 * d2);
    for (int k = 0; k < noff; ++k) {
      const int64_t j0 = i0 + kOffsets[k][0], j1 = i1 + kOffsets[k][1], j2 = i2 + kOffsets[k][2];
      if (j0 < 0 || j0 >= d0 || j1 < 0 || j1 >= d1 || j2 < 0 || j2 >= d2) continue;
      const int32_t cn = inv[(j0 * d1 + j1) * d2 + j2];
      if (cn < 0 || __ldcg(Lb + cn) < 0) continue;
      cc_unite(Lb, c, cn);
    }
  }
}

// S[b][root] += 1 for every active voxel (S zeroed).
__global__ void cc_count_kernel(const int32_t* __restrict__ L, int64_t total, int64_t V,
                                int32_t* __restrict__ S) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    if (__ldcg(L + e) < 0) continue;
    const int64_t b = e / V;
    const int32_t r = cc_find(L + b * V, int32_t(e - b * V));
    atomicAdd(S + b * V + r, 1);
  }
}

// out[b] = max_c S[b][c] (0 with no active voxel); one block per row.
__global__ void cc_max_kernel(const int32_t* __restrict__ S, int64_t V, int32_t* __restrict__ out) {
  __shared__ int32_t wm[32];
  const int64_t b = blockIdx.x;
  int32_t m = 0;
  for (int64_t c = threadIdx.x; c < V; c += blockDim.x) m = max(m, S[b * V + c]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? wm[threadIdx.x] : 0;
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) out[b] = m;
  }
}

// Observed map in mask order: label = mask index of the cluster's smallest
// voxel (-1 inactive or without a statistic), size = its cluster's size.
__global__ void cc_observed_out_kernel(const int32_t* __restrict__ L, const int32_t* __restrict__ S,
                                       int64_t V, const int32_t* __restrict__ valid_map,
                                       int32_t* __restrict__ label, int32_t* __restrict__ size) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < V;
       c += int64_t(gridDim.x) * blockDim.x) {
    const int32_t j = valid_map[c];
    if (__ldcg(L + c) < 0) continue;  // label/size keep their -1 / 0 fill
    const int32_t r = cc_find(L, int32_t(c));
    label[j] = valid_map[r];
    size[j] = S[r];
  }
}

__global__ void fill_i32_kernel(int32_t* __restrict__ p, int64_t n, int32_t v) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n;
       e += int64_t(gridDim.x) * blockDim.x)
    p[e] = v;
}

pt_status check_cluster_args(pt_ctx* ctx, double tau, const int32_t* dims, int connectivity) {
  if (ctx->glm_q1) {
    set_error(ctx, "cluster summaries of the plain two-sample t only (context has covariates)");
    return PT_ERR_UNSUPPORTED;
  }
  if (!dims || dims[0] < 1 || dims[1] < 1 || dims[2] < 1 ||
      int64_t(dims[0]) * dims[1] * dims[2] != ctx->n_grid) {
    set_error(ctx, "cluster summaries: need dims with d0 * d1 * d2 = n_grid");
    return PT_ERR_INVALID;
  }
  if (connectivity != 6 && connectivity != 18 && connectivity != 26) {
    set_error(ctx, "cluster summaries: connectivity must be 6, 18 or 26");
    return PT_ERR_INVALID;
  }
  if (!std::isfinite(tau)) {
    set_error(ctx, "cluster summaries: tau must be finite");
    return PT_ERR_INVALID;
  }
  if (ctx->n_grid >= (int64_t(1) << 31)) {
    set_error(ctx, "cluster summaries: grid too large");
    return PT_ERR_UNSUPPORTED;
  }
  // the inverse map of this grid shape
  if (ctx->grid_dims[0] != dims[0] || ctx->grid_dims[1] != dims[1] ||
      ctx->grid_dims[2] != dims[2] || !ctx->grid_inv.p) {
    if (!ctx->grid_inv.ensure(sizeof(int32_t) * size_t(ctx->n_grid))) {
      set_error(ctx, "out of device memory (cluster grid map)");
      return PT_ERR_NOMEM;
    }
    grid_inv_fill_kernel<<<grid_for(ctx->n_grid, 256), 256, 0, ctx->stream>>>(
        ctx->grid_inv.as<int32_t>(), ctx->n_grid);
    PT_LAUNCH_CHECK(ctx);
    if (ctx->v_valid > 0) {
      grid_inv_set_kernel<<<grid_for(ctx->v_valid, 256), 256, 0, ctx->stream>>>(
          ctx->vox_grid.as<int64_t>(), ctx->valid_map.as<int32_t>(), ctx->v_valid,
          ctx->grid_inv.as<int32_t>());
      PT_LAUNCH_CHECK(ctx);
    }
    for (int q = 0; q < 3; ++q) ctx->grid_dims[q] = dims[q];
  }
  return PT_OK;
}

// u threshold of the t threshold tau (strictly increasing map; |u| < 1/sqrt(k)).
float u_of_tau(const pt_ctx* ctx, double tau) {
  return float(tau / std::sqrt(ctx->k * (ctx->n - 2) + ctx->k * tau * tau));
}

// Labels rows (B x V int32, active = c) -> component sizes -> per-row maxima.
pt_status components(pt_ctx* ctx, int32_t* L, int64_t B, int32_t* S, int connectivity) {
  const int64_t V = ctx->v_valid, total = B * V;
  cudaStream_t st = ctx->stream;
  cc_union_kernel<<<grid_for(total, 256), 256, 0, st>>>(
      L, total, V, ctx->valid_map.as<int32_t>(), ctx->vox_grid.as<int64_t>(),
      ctx->grid_inv.as<int32_t>(), ctx->grid_dims[0], ctx->grid_dims[1], ctx->grid_dims[2],
      n_offsets(connectivity));
  PT_LAUNCH_CHECK(ctx);
  PT_CUDA_TRY(ctx, cudaMemsetAsync(S, 0, sizeof(int32_t) * size_t(total), st));
  cc_count_kernel<<<grid_for(total, 256), 256, 0, st>>>(L, total, V, S);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

}  // namespace

pt_status cluster_maxnull_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, double tau,
                               const int32_t* dims, int connectivity, int precision,
                               int32_t* maxsize) {
  pt_status s = check_cluster_args(ctx, tau, dims, connectivity);
  if (s != PT_OK) return s;
  cudaStream_t st = ctx->stream;
  const int64_t V = ctx->v_valid;
  if (V == 0) {
    PT_CUDA_TRY(ctx, cudaMemsetAsync(maxsize, 0, sizeof(int32_t) * size_t(P), st));
    return PT_OK;
  }
  // batch of relabellings: two int32/float arrays of B x V, about 1 GB in all
  int64_t B = std::max<int64_t>(128, (int64_t(1) << 29) / (4 * V) / 128 * 128);
  B = std::min<int64_t>(B, (P + 127) / 128 * 128);
  Buf ub, sb;
  struct G {
    Buf *a, *b;
    ~G() {
      a->release();
      b->release();
    }
  } guard{&ub, &sb};
  if (!ub.ensure(sizeof(float) * size_t(B) * V) || !sb.ensure(sizeof(int32_t) * size_t(B) * V)) {
    set_error(ctx, "out of device memory (cluster rows)");
    return PT_ERR_NOMEM;
  }
  const bool tc = precision != PT_PREC_FP32;
  if (tc) {
    s = tc_supported(ctx);
    if (s == PT_OK) s = ensure_xnb(ctx, precision);
  } else {
    s = ensure_xn32(ctx);
  }
  if (s != PT_OK) return s;
  if (!ctx->cnt.ensure(sizeof(uint32_t) * (V + 1))) {  // the labels kernel counts observed-set rows
    set_error(ctx, "out of device memory (workspace)");
    return PT_ERR_NOMEM;
  }
  const float ut = u_of_tau(ctx, tau);
  for (int64_t i0 = 0; i0 < P; i0 += B) {
    const int64_t nb = std::min(B, P - i0);
    int64_t P_pad = 0;
    s = build_labels(ctx, perms + i0 * ctx->n, nb, prec_label_layout(precision), &P_pad);
    if (s != PT_OK) return s;
    if (tc) {
      s = tc_rows(ctx, ctx->labels.p, nb, precision, 1, ub.as<float>(), 0, 0, nullptr, nullptr,
                  nullptr);
      if (s != PT_OK) return s;
    } else {
      const dim3 grid{unsigned((V + 127) / 128), unsigned((nb + 127) / 128), 1u};
      simt_contract_kernel<<<grid, 256, 0, st>>>(ctx->labels.as<float>(), ctx->Xn32.as<float>(),
                                                 ctx->n_pad, nb, V, 1, 1, 0, nullptr,
                                                 ctx->rowflag.as<uint8_t>(), nullptr, nullptr,
                                                 ub.as<float>());
      PT_LAUNCH_CHECK(ctx);
    }
    cc_init_kernel<<<grid_for(nb * V, 256), 256, 0, st>>>(ub.as<float>(), nb * V, V, ut);
    PT_LAUNCH_CHECK(ctx);
    s = components(ctx, reinterpret_cast<int32_t*>(ub.p), nb, sb.as<int32_t>(), connectivity);
    if (s != PT_OK) return s;
    cc_max_kernel<<<unsigned(nb), 256, 0, st>>>(sb.as<int32_t>(), V, maxsize + i0);
    PT_LAUNCH_CHECK(ctx);
  }
  // the batch buffers are released on return: wait for the kernels that use them
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return PT_OK;
}

pt_status cluster_observed_impl(pt_ctx* ctx, double tau, const int32_t* dims, int connectivity,
                                int32_t* label, int32_t* size) {
  pt_status s = check_cluster_args(ctx, tau, dims, connectivity);
  if (s != PT_OK) return s;
  cudaStream_t st = ctx->stream;
  const int64_t V = ctx->v_valid, v = ctx->v;
  if (v > 0) {
    fill_i32_kernel<<<grid_for(v, 256), 256, 0, st>>>(label, v, -1);
    PT_LAUNCH_CHECK(ctx);
    PT_CUDA_TRY(ctx, cudaMemsetAsync(size, 0, sizeof(int32_t) * size_t(v), st));
  }
  if (V == 0) return PT_OK;
  Buf ub, sb;
  struct G {
    Buf *a, *b;
    ~G() {
      a->release();
      b->release();
    }
  } guard{&ub, &sb};
  if (!ub.ensure(sizeof(float) * size_t(V)) || !sb.ensure(sizeof(int32_t) * size_t(V))) {
    set_error(ctx, "out of device memory (cluster map)");
    return PT_ERR_NOMEM;
  }
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(ub.p, ctx->u_obs.p, sizeof(float) * size_t(V),
                                   cudaMemcpyDeviceToDevice, st));
  cc_init_kernel<<<grid_for(V, 256), 256, 0, st>>>(ub.as<float>(), V, V, u_of_tau(ctx, tau));
  PT_LAUNCH_CHECK(ctx);
  s = components(ctx, reinterpret_cast<int32_t*>(ub.p), 1, sb.as<int32_t>(), connectivity);
  if (s != PT_OK) return s;
  cc_observed_out_kernel<<<grid_for(V, 256), 256, 0, st>>>(
      reinterpret_cast<int32_t*>(ub.p), sb.as<int32_t>(), V, ctx->valid_map.as<int32_t>(), label,
      size);
  PT_LAUNCH_CHECK(ctx);
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return PT_OK;
}

}  // namespace pt

extern "C" {

pt_status pt_cluster_maxnull(pt_ctx* ctx, const int32_t* perms, int64_t P, double tau,
                             const int32_t* dims, int32_t connectivity, int32_t precision,
                             int32_t* maxsize) {
  pt::NvtxRange nvtx_range("pt_cluster_maxnull");
  if (!ctx || !perms || !maxsize || !dims) {
    pt::set_error(ctx, "pt_cluster_maxnull: NULL argument");
    return PT_ERR_INVALID;
  }
  if (P < 1 || P > INT32_MAX || precision < PT_PREC_FP32 || precision > PT_PREC_FP16X2) {
    pt::set_error(ctx, "pt_cluster_maxnull: need 1 <= P <= 2^31-1 and a valid precision");
    return PT_ERR_INVALID;
  }
  try {
    cudaSetDevice(ctx->device);
    return pt::cluster_maxnull_impl(ctx, perms, P, tau, dims, connectivity, precision, maxsize);
  } catch (...) {
    pt::set_error(ctx, "pt_cluster_maxnull: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_cluster_observed(pt_ctx* ctx, double tau, const int32_t* dims, int32_t connectivity,
                              int32_t* label, int32_t* size) {
  pt::NvtxRange nvtx_range("pt_cluster_observed");
  if (!ctx || !dims || !label || !size) {
    pt::set_error(ctx, "pt_cluster_observed: NULL argument");
    return PT_ERR_INVALID;
  }
  try {
    cudaSetDevice(ctx->device);
    return pt::cluster_observed_impl(ctx, tau, dims, connectivity, label, size);
  } catch (...) {
    pt::set_error(ctx, "pt_cluster_observed: internal error");
    return PT_ERR_CUDA;
  }
}

}  // extern "C"
