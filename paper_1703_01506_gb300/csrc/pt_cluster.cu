// Cluster-level summaries of thresholded statistic maps (the cluster tables of
// Sec. 6, Figs. 8-9), and the largest cluster under each relabelling: the
// cluster-level counterpart of the max-null (Sec. 2).
//
// A voxel is active when its statistic reaches the threshold tau; clusters are
// the connected sets of active mask voxels on the 3D grid under 6-, 18- or
// 26-connectivity. Through the monotone map of each relabelling the test
// t >= tau is u >= u(tau), u = tau / sqrt(k (n-2) + k tau^2), so the NaivePT
// contraction writes, per relabelling of a batch, one bit per voxel (u >=
// u(tau)) and nothing else: T stays out of memory.
//
// Components by union-find over the compact indices of the active voxels,
// one label array per relabelling of the batch of which only active entries
// are ever written or read (a neighbour's activity is a bit test): a link
// always points to a smaller index, so a root is the smallest voxel of its
// component, every find walks strictly decreasing indices and every unite
// retries on a strictly smaller index. Nothing waits on another thread; links
// are made with atomicMin and read through L2 (__ldcg), where the atomics land.
// The kernels walk bit words, so their work follows the active voxels.
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

// Bit rows from rows of u (the FP32 path): bit c of row b = U[b][c] >= u_tau.
__global__ void cc_bits_from_rows_kernel(const float* __restrict__ U, int64_t B, int64_t V,
                                         int64_t W, float u_tau, uint32_t* __restrict__ BM) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < B * W;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = e / W, c0 = (e - b * W) * 32;
    uint32_t w = 0u;
    for (int k = 0; k < 32 && c0 + k < V; ++k) w |= uint32_t(U[b * V + c0 + k] >= u_tau) << k;
    BM[e] = w;
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

__device__ __forceinline__ bool bit_at(const uint32_t* __restrict__ row, int32_t c) {
  return (__ldg(row + (c >> 5)) >> (c & 31)) & 1u;
}

// Per bit word e of the batch (row b = e / W): the word's active voxels c.
#define CC_FOR_ACTIVE(...)                                                         \
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < B * W;       \
       e += int64_t(gridDim.x) * blockDim.x) {                                      \
    uint32_t w = BM[e];                                                             \
    if (!w) continue;                                                               \
    const int64_t b = e / W;                                                        \
    const int32_t c0 = int32_t((e - b * W) * 32);                                   \
    while (w) {                                                                     \
      const int32_t c = c0 + __ffs(int(w)) - 1;                                     \
      w &= w - 1u;                                                                  \
      __VA_ARGS__                                                                   \
    }                                                                               \
  }

// L[b][c] = c and S[b][c] = 0 for every active voxel (the only entries used).
__global__ void cc_init_kernel(const uint32_t* __restrict__ BM, int64_t B, int64_t W, int64_t V,
                               int32_t* __restrict__ L, int32_t* __restrict__ S) {
  CC_FOR_ACTIVE({
    L[b * V + c] = c;
    S[b * V + c] = 0;
  })
}

__global__ void cc_union_kernel(const uint32_t* __restrict__ BM, int64_t B, int64_t W, int64_t V,
                                int32_t* __restrict__ L, const int32_t* __restrict__ valid_map,
                                const int64_t* __restrict__ vox_grid,
                                const int32_t* __restrict__ inv, int64_t d0, int64_t d1,
                                int64_t d2, int noff) {
  CC_FOR_ACTIVE({
    int32_t* Lb = L + b * V;
    const uint32_t* row = BM + b * W;
    const int64_t g = vox_grid[valid_map[c]];
    const int64_t i2 = g % d2, i1 = (g / d2) % d1, i0 = g / (d1 * d2);
    for (int k = 0; k < noff; ++k) {
      const int64_t j0 = i0 + kOffsets[k][0], j1 = i1 + kOffsets[k][1], j2 = i2 + kOffsets[k][2];
      if (j0 < 0 || j0 >= d0 || j1 < 0 || j1 >= d1 || j2 < 0 || j2 >= d2) continue;
      const int32_t cn = inv[(j0 * d1 + j1) * d2 + j2];
      if (cn < 0 || !bit_at(row, cn)) continue;
      cc_unite(Lb, c, cn);
    }
  })
}

// S[b][root] += 1 for every active voxel.
__global__ void cc_count_kernel(const uint32_t* __restrict__ BM, int64_t B, int64_t W, int64_t V,
                                const int32_t* __restrict__ L, int32_t* __restrict__ S) {
  CC_FOR_ACTIVE({
    const int32_t r = cc_find(L + b * V, c);
    atomicAdd(S + b * V + r, 1);
  })
}

// out[b] = max over the active voxels c of S[b][c] (0 with none); one block per row.
__global__ void cc_max_kernel(const uint32_t* __restrict__ BM, int64_t W, int64_t V,
                              const int32_t* __restrict__ S, int32_t* __restrict__ out) {
  __shared__ int32_t wm[32];
  const int64_t b = blockIdx.x;
  int32_t m = 0;
  for (int64_t q = threadIdx.x; q < W; q += blockDim.x) {
    uint32_t w = BM[b * W + q];
    while (w) {
      const int32_t c = int32_t(q * 32) + __ffs(int(w)) - 1;
      w &= w - 1u;
      m = max(m, __ldcg(S + b * V + c));
    }
  }
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
__global__ void cc_observed_out_kernel(const uint32_t* __restrict__ BM, const int32_t* __restrict__ L,
                                       const int32_t* __restrict__ S, int64_t V,
                                       const int32_t* __restrict__ valid_map,
                                       int32_t* __restrict__ label, int32_t* __restrict__ size) {
  for (int64_t c = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; c < V;
       c += int64_t(gridDim.x) * blockDim.x) {
    if (!bit_at(BM, int32_t(c))) continue;  // label/size keep their -1 / 0 fill
    const int32_t j = valid_map[c];
    const int32_t r = cc_find(L, int32_t(c));
    label[j] = valid_map[r];
    size[j] = __ldcg(S + r);
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

// Bit rows (B x W words) -> labels of the active voxels -> component sizes at the roots.
pt_status components(pt_ctx* ctx, const uint32_t* BM, int64_t B, int32_t* L, int32_t* S,
                     int connectivity) {
  const int64_t V = ctx->v_valid, W = (V + 31) / 32;
  cudaStream_t st = ctx->stream;
  cc_init_kernel<<<grid_for(B * W, 256), 256, 0, st>>>(BM, B, W, V, L, S);
  PT_LAUNCH_CHECK(ctx);
  cc_union_kernel<<<grid_for(B * W, 256), 256, 0, st>>>(
      BM, B, W, V, L, ctx->valid_map.as<int32_t>(), ctx->vox_grid.as<int64_t>(),
      ctx->grid_inv.as<int32_t>(), ctx->grid_dims[0], ctx->grid_dims[1], ctx->grid_dims[2],
      n_offsets(connectivity));
  PT_LAUNCH_CHECK(ctx);
  cc_count_kernel<<<grid_for(B * W, 256), 256, 0, st>>>(BM, B, W, V, L, S);
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
  // batch of relabellings: label and size arrays of B x V int32 (about 1 GB each,
  // of which only the active voxels' entries are touched) and B x W bit words
  const bool tc = precision != PT_PREC_FP32;
  const int64_t W = (V + 31) / 32;
  int64_t B = std::max<int64_t>(128, (int64_t(1) << 28) / V / 128 * 128);
  B = std::min<int64_t>(B, (P + 127) / 128 * 128);
  Buf lb, sb, bm, ub;
  struct G {
    Buf *a, *b, *c, *d;
    ~G() {
      a->release();
      b->release();
      c->release();
      d->release();
    }
  } guard{&lb, &sb, &bm, &ub};
  if (!lb.ensure(sizeof(int32_t) * size_t(B) * V) || !sb.ensure(sizeof(int32_t) * size_t(B) * V) ||
      !bm.ensure(sizeof(uint32_t) * size_t(B) * W) ||
      (!tc && !ub.ensure(sizeof(float) * size_t(B) * V))) {
    set_error(ctx, "out of device memory (cluster rows)");
    return PT_ERR_NOMEM;
  }
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
      PT_CUDA_TRY(ctx, cudaMemsetAsync(bm.p, 0, sizeof(uint32_t) * size_t(nb) * W, st));
      s = tc_rows(ctx, ctx->labels.p, nb, precision, 3, bm.as<float>(), 0, 0, nullptr, nullptr,
                  nullptr, ut);
      if (s != PT_OK) return s;
    } else {
      const dim3 grid{unsigned((V + 127) / 128), unsigned((nb + 127) / 128), 1u};
      simt_contract_kernel<<<grid, 256, 0, st>>>(ctx->labels.as<float>(), ctx->Xn32.as<float>(),
                                                 ctx->n_pad, nb, V, 1, 1, 0, nullptr,
                                                 ctx->rowflag.as<uint8_t>(), nullptr, nullptr,
                                                 ub.as<float>());
      PT_LAUNCH_CHECK(ctx);
      cc_bits_from_rows_kernel<<<grid_for(nb * W, 256), 256, 0, st>>>(ub.as<float>(), nb, V, W,
                                                                      ut, bm.as<uint32_t>());
      PT_LAUNCH_CHECK(ctx);
    }
    s = components(ctx, bm.as<uint32_t>(), nb, lb.as<int32_t>(), sb.as<int32_t>(), connectivity);
    if (s != PT_OK) return s;
    cc_max_kernel<<<unsigned(nb), 256, 0, st>>>(bm.as<uint32_t>(), W, V, sb.as<int32_t>(),
                                                maxsize + i0);
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
  const int64_t W = (V + 31) / 32;
  Buf lb, sb, bm;
  struct G {
    Buf *a, *b, *c;
    ~G() {
      a->release();
      b->release();
      c->release();
    }
  } guard{&lb, &sb, &bm};
  if (!lb.ensure(sizeof(int32_t) * size_t(V)) || !sb.ensure(sizeof(int32_t) * size_t(V)) ||
      !bm.ensure(sizeof(uint32_t) * size_t(W))) {
    set_error(ctx, "out of device memory (cluster map)");
    return PT_ERR_NOMEM;
  }
  cc_bits_from_rows_kernel<<<grid_for(W, 256), 256, 0, st>>>(ctx->u_obs.as<float>(), 1, V, W,
                                                             u_of_tau(ctx, tau),
                                                             bm.as<uint32_t>());
  PT_LAUNCH_CHECK(ctx);
  s = components(ctx, bm.as<uint32_t>(), 1, lb.as<int32_t>(), sb.as<int32_t>(), connectivity);
  if (s != PT_OK) return s;
  cc_observed_out_kernel<<<grid_for(V, 256), 256, 0, st>>>(
      bm.as<uint32_t>(), lb.as<int32_t>(), sb.as<int32_t>(), V, ctx->valid_map.as<int32_t>(),
      label, size);
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
