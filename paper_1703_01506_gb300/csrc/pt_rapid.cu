// RapidPT (Alg. 2; Sec. 4.1 training, Sec. 4.2 recovery) on the GPU.
//
//   training  T_ex (n_train x v) by the NaivePT contraction writing t rows;
//             U0 = orthonormalised Philox normals; for each pass and training
//             column, in order: m = ceil(eta v) sampled voxels, l1 weight solve
//             (ADMM) against U at those voxels, rank-one geodesic update of U
//             towards the residual; FP64-factorised QR every qr_every steps.
//             W_ex = U^T T_ex, sigma = std of the sampled residuals of the last
//             pass, shift mu (Alg. 2 literal, or mean shift of the maximum).
//   recovery  per later relabelling: t at its m sampled voxels, l1 weight solve
//             with U frozen, then max_j (U w + sigma z)_j + mu, where noise is
//             drawn only at voxels whose (U w)_j + sigma * |z|max can still
//             reach the running maximum (|z| <= sqrt(-2 ln 2^-32) for the
//             Box-Muller draws used), which leaves the maximum unchanged.
//
// The weight solve and the update follow one explicit reading of the cited
// GRASTA/GROUSE steps (the paper gives no formulas):
//   ADMM on min ||s||_1 s.t. A w + s = b:  w <- G^-1 A^T (b - s - y/rho),
//   s <- soft(b - A w - y/rho, 1/rho),  y <- y + rho (A w + s - b),  G = A^T A;
//   r = b - A w, lift(r) summed onto the sampled voxels, g2 = A^T r,
//   Gamma = lift(r) - U g2, theta = step * atan(||r|| / ||w||),
//   U <- U + [(cos theta - 1) U w / ||w|| + sin theta Gamma / ||Gamma||] w^T / ||w||,
//   with ||Gamma||^2 = ||lift||^2 - ||g2||^2 (U orthonormal).
// Random numbers: Philox4x32-10 by counter (pt_draws.h). The reconstruction
// with noise runs on the tensor cores (pt_recon_tc.cu).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pt_internal.h"
#include "pt_draws.h"
#include "pt_kernels.h"

namespace pt {

// Kernels of the NaivePT path reused here (pt_naive.cu).
__global__ void finalize_max_kernel(const unsigned long long* maxkey, int64_t P,
                                    const int32_t* valid_map, const float* Xraw, int n, int n1,
                                    int n_pad, const int32_t* perms, int two_sided,
                                    float* maxnull, int32_t* argmax);
__global__ void scatter_counts_kernel(const uint32_t* cnt, int64_t v_valid,
                                      const int32_t* valid_map, uint32_t* counts,
                                      int accumulate);
__global__ void simt_contract_kernel(const float* L, const float* Xn, int n_pad, int64_t P,
                                     int64_t v, int tiles_per_cta, int mode, int two_sided,
                                     const float* u_obs, const uint8_t* rowflag,
                                     unsigned long long* maxkey, uint32_t* cnt, float* uout);

namespace cg = cooperative_groups;

namespace {

constexpr int kMaxRank = 128;

// One row of the geodesic update of U (Sec. 4.1; GROUSE-style rank-one step):
// U_j <- U_j + coef_j w^T/||w||, coef_j = alpha (U_j . w) + beta (lift_j - U_j . g2).
// Shared by the whole-U update and by the next step's gather, which applies a
// still-running update to the rows it samples: both give the same bits.
// w, wh and g2 are shared-memory vectors (16-byte aligned); they are re-read
// for every row (volatile loads), so a loop over rows holds only the row in
// registers.
__device__ __forceinline__ float4 lds4(const float* p) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "r"(uint32_t(__cvta_generic_to_shared(p))));
  return v;
}

// Bulk copy of `bytes` from global src to this CTA's shared dst, completing
// on the mbarrier bar (dst, src and bytes multiples of 16).
__device__ __forceinline__ void bulk_copy_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                              uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}
// Orders this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) writes.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bulk prefetch of [p, p + bytes) into L2 (p and bytes multiples of 16).
__device__ __forceinline__ void prefetch_l2_bulk(const void* p, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

template <int RP>
__device__ __forceinline__ void geodesic_row(float4 (&x)[RP / 4], float lj, const float* w,
                                             const float* wh, const float* g2, float alpha,
                                             float beta) {
  float p = 0.0f, g = 0.0f;
#pragma unroll
  for (int c4 = 0; c4 < RP / 4; ++c4) {
    const float4 wc = lds4(w + 4 * c4), gc = lds4(g2 + 4 * c4);
    p = fmaf(x[c4].x, wc.x, p);
    p = fmaf(x[c4].y, wc.y, p);
    p = fmaf(x[c4].z, wc.z, p);
    p = fmaf(x[c4].w, wc.w, p);
    g = fmaf(x[c4].x, gc.x, g);
    g = fmaf(x[c4].y, gc.y, g);
    g = fmaf(x[c4].z, gc.z, g);
    g = fmaf(x[c4].w, gc.w, g);
  }
  const float coef = fmaf(alpha, p, beta * (lj - g));
#pragma unroll
  for (int c4 = 0; c4 < RP / 4; ++c4) {
    const float4 hc = lds4(wh + 4 * c4);
    x[c4].x = fmaf(coef, hc.x, x[c4].x);
    x[c4].y = fmaf(coef, hc.y, x[c4].y);
    x[c4].z = fmaf(coef, hc.z, x[c4].z);
    x[c4].w = fmaf(coef, hc.w, x[c4].w);
  }
}

// ---------------------------------------------------------------------------
// Cluster l1 weight solve (Sec. 4.1 / 4.2, the Complete step). The m sampled
// rows are split over the CL CTAs of a thread-block cluster: each CTA keeps
// its rows of A = U_Omega and of b, s, y, x in shared memory, and the R-length
// reductions (Gram matrix, A^T x, A^T r) are summed across the cluster
// through distributed shared memory, in rank order, so every CTA holds
// bit-identical sums and hence the same weights w.
// ---------------------------------------------------------------------------
constexpr int kCluThreads = 512;  // 16 warps per CTA
constexpr int kCluWarps = kCluThreads / 32;

struct CluSmem {
  float* A;      // mloc x clu_rs(RP)
  float* b;      // mloc each: b, s, y, x
  float* s;
  float* y;
  float* x;
  int32_t* idx;  // mloc sampled voxel of each local row
  float* G;      // R x RG (RG = R rounded up to 4): the Gram matrix, inverted in place
  float* Gp;     // R x RG, upper triangle: this CTA's Gram partial, read by the cluster
                 // in float4 steps
  float* xch;    // 2 x CL x kSlot: the partial vectors every rank pushed here, one slot
                 // per rank (parity-alternated)
  float* stage;  // kSlot: this CTA's partial vector before it is pushed
  float* red;    // kCluWarps x RP cross-warp partials; the Gauss-Jordan staging
  float* vec;    // kSlot: a cluster sum
  float* wv;     // RP: weights
  float* misc;   // 8 scalars, then one partial per warp
  float* pinv;   // 16: inverse of the current Gauss-Jordan pivot block
  float* Lrow;   // n_pad labels of the relabelling (recovery)
};
constexpr int kSlot = kMaxRank + 8;

// Row stride of A in shared memory: 16-byte rows whose stride in 16-byte units
// is odd, so a warp reading 32 different rows in float4 steps hits every bank
// group once per four lanes (and column-wise reads stay conflict-free).
__host__ __device__ constexpr int clu_rs(int RP) { return (RP / 4) % 2 == 0 ? RP + 4 : RP; }

__host__ __device__ inline size_t clu_carve(float* base, int mloc, int R, int RP, int n_pad,
                                            int CL, CluSmem* f) {
  const int RS = clu_rs(RP);
  const size_t RG = size_t(R + 3) / 4 * 4;
  size_t o = 0;
  auto take = [&](size_t nfl) {
    float* p = base ? base + o : nullptr;
    o += (nfl + 3) / 4 * 4;  // keep 16-byte alignment
    return p;
  };
  CluSmem t;
  t.A = take(size_t(mloc) * RS);
  t.b = take(mloc);
  t.s = take(mloc);
  t.y = take(mloc);
  t.x = take(mloc);
  t.idx = reinterpret_cast<int32_t*>(take(mloc));
  t.G = take(size_t(R) * RG);
  // The Gram partial is dead once the cluster has summed it (a cluster barrier
  // follows the sum), before s, y and x are first written: it shares their
  // space when it fits there (contiguous: s, y, x are taken in a row).
  const size_t gp = size_t(R) * RG;
  t.Gp = gp <= 3 * ((size_t(mloc) + 3) / 4 * 4) ? t.s : take(gp);
  t.xch = take(2 * size_t(CL) * kSlot);
  t.stage = take(kSlot);
  t.red = take(size_t(kCluWarps) * RP);
  t.vec = take(kSlot);
  t.wv = take(RP);
  t.misc = take(8 + kCluWarps);
  t.pinv = take(16);
  t.Lrow = take(n_pad);
  if (f) *f = t;
  return o * sizeof(float);
}

// Pushes this CTA's partial vector p[0..len) into its slot (par, rank) in every
// CTA of the cluster (remote shared-memory stores; the cluster barrier that
// follows makes them visible).
__device__ __forceinline__ void clu_push(cg::cluster_group& cl, const CluSmem& f, int par,
                                         int rank, const float* p, int len, int CL) {
  float* mine = f.xch + (size_t(par) * CL + rank) * kSlot;
  for (int e = threadIdx.x; e < len * CL; e += blockDim.x) {
    const int r = e / len, c = e - r * len;
    cl.map_shared_rank(mine, r)[c] = p[c];
  }
}

// Sum over the ranks, in rank order, of the pushed slots (par, .)[c].
__device__ __forceinline__ float clu_slot_sum(const CluSmem& f, int par, int c, int CL) {
  const float* s = f.xch + size_t(par) * CL * kSlot + c;
  float sum = 0.0f;
  for (int r = 0; r < CL; ++r) sum += s[size_t(r) * kSlot];
  return sum;
}

// Sum over the cluster's CTAs (rank order) of stage[0..len) into vec.
__device__ __forceinline__ void clu_sum(cg::cluster_group& cl, const CluSmem& f, int& par,
                                        int len, int CL, int rank) {
  __syncthreads();
  clu_push(cl, f, par, rank, f.stage, len, CL);
  cl.sync();
  for (int c = threadIdx.x; c < len; c += blockDim.x) f.vec[c] = clu_slot_sum(f, par, c, CL);
  par ^= 1;
  __syncthreads();
}

// out[c] = sum over local rows q of A[q][c] x[q], c < R.
template <int RP>
__device__ __forceinline__ void clu_AtX(const CluSmem& f, int mloc, int R, const float* x,
                                        float* out) {
  constexpr int RS = clu_rs(RP), KC = (RP + 31) / 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float acc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) acc[k] = 0.0f;
  for (int q = w; q < mloc; q += kCluWarps) {
    const float xq = x[q];
    const float* row = f.A + q * RS;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const int c = lane + 32 * k;
      if (c < RP) acc[k] = fmaf(row[c], xq, acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int c = lane + 32 * k;
    if (c < RP) f.red[w * RP + c] = acc[k];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    float t = 0.0f;
#pragma unroll
    for (int ww = 0; ww < kCluWarps; ++ww) t += f.red[ww * RP + c];
    out[c] = t;
  }
}

// Block sum of one value per thread into *dst (thread 0 writes).
__device__ __forceinline__ void clu_block_sum_to(float v, const CluSmem& f, float* dst) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) f.misc[8 + (threadIdx.x >> 5)] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.0f;
    for (int w = 0; w < kCluWarps; ++w) t += f.misc[8 + w];
    *dst = t;
  }
}

template <int RP>
__device__ __forceinline__ float clu_row_dot(const float* row, const float* v) {
  const float4* r4 = reinterpret_cast<const float4*>(row);
  const float4* v4 = reinterpret_cast<const float4*>(v);  // v: 16-byte aligned
  float4 a[RP / 4];
#pragma unroll
  for (int c4 = 0; c4 < RP / 4; ++c4) a[c4] = r4[c4];
  float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
  for (int c4 = 0; c4 < RP / 4; ++c4) {
    const float4 w = v4[c4];
    t0 = fmaf(a[c4].x, w.x, t0);
    t1 = fmaf(a[c4].y, w.y, t1);
    t0 = fmaf(a[c4].z, w.z, t0);
    t1 = fmaf(a[c4].w, w.w, t1);
  }
  return t0 + t1;
}

// Sum over local rows q = first, first + step, ... of the 4 x 4 outer products
// of A's column blocks ti and tj (four rows per step in flight).
template <int RP>
__device__ __forceinline__ void gram_tile(const float* A, int mloc, int first, int step, int ti,
                                          int tj, float (&acc)[4][4]) {
  constexpr int RS = clu_rs(RP);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = 0.0f;
#pragma unroll 4
  for (int q = first; q < mloc; q += step) {
    const float4 u = *reinterpret_cast<const float4*>(A + q * RS + 4 * ti);
    const float4 v = *reinterpret_cast<const float4*>(A + q * RS + 4 * tj);
    const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) acc[a][b2] = fmaf(uu[a], vv[b2], acc[a][b2]);
  }
}

__device__ __forceinline__ void tile_of(int tile, int RT, int& ti, int& tj) {
  ti = 0;
  int rem = tile;
  while (rem >= RT - ti) {
    rem -= RT - ti;
    ++ti;
  }
  tj = ti + rem;
}

// Gram G = A^T A over the cluster, then G^-1 in place (block Gauss-Jordan
// without pivoting: G is symmetric positive definite), then ADMM; leaves w in
// f.wv (zero-padded to RP). An ADMM iteration: A^T x over the CTA's rows, the
// CTA's share G^-1 (A^T x)_local pushed to every rank, one cluster barrier, the
// rank-ordered sum of the pushed shares, then the s, y, x updates with one
// thread per row.
template <int RP>
__device__ void clu_l1_fit(cg::cluster_group& cl, const CluSmem& f, int mloc, int R, float rho,
                           int iters, int CL, int rank, int& par) {
  constexpr int RS = clu_rs(RP);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int RG = (R + 3) / 4 * 4;
  // --- local Gram partial by 4x4 register tiles of the upper triangle. With
  // fewer tiles than threads, ngr thread groups take every ngr-th row each,
  // all at once, and add their sums into Gp in group order.
  constexpr int RT = RP / 4;
  constexpr int ntile = RT * (RT + 1) / 2;
  constexpr int ngr = ntile >= kCluThreads ? 1 : kCluThreads / ntile;
  auto put_tile = [&](int ti, int tj, const float (&acc)[4][4], bool add) {
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b2 = 0; b2 < 4; ++b2) {
        const int c = 4 * ti + a, d = 4 * tj + b2;
        if (c < R && d < RG) {
          const float val = (c <= d && d < R) ? acc[a][b2] : 0.0f;
          f.Gp[c * RG + d] = add ? f.Gp[c * RG + d] + val : val;
        }
      }
  };
  if constexpr (ngr == 1) {
    for (int t = tid; t < ntile; t += kCluThreads) {
      int ti, tj;
      tile_of(t, RT, ti, tj);
      float acc[4][4];
      gram_tile<RP>(f.A, mloc, 0, 1, ti, tj, acc);
      put_tile(ti, tj, acc, false);
    }
  } else {
    const bool act = tid < ntile * ngr;
    const int grp = tid / ntile;
    int ti = 0, tj = 0;
    tile_of(tid - grp * ntile, RT, ti, tj);
    float acc[4][4];
    gram_tile<RP>(f.A, act ? mloc : 0, grp, ngr, ti, tj, acc);
    for (int g = 0; g < ngr; ++g) {
      if (act && grp == g) put_tile(ti, tj, acc, g > 0);
      __syncthreads();
    }
  }
  __syncthreads();
  cl.sync();  // every CTA's partial is complete
  // --- cluster sum of the upper triangle: rank k sums the float4 units u with
  // u % CL == k over all ranks (rank order) and writes the sum into every
  // rank's G; then each CTA mirrors the upper triangle
  const int rg4 = RG / 4;
  for (int e = rank + CL * tid; e < R * rg4; e += CL * kCluThreads) {
    const int c = e / rg4, d4 = e - c * rg4;
    if (4 * d4 + 3 < c) continue;  // wholly below the diagonal
    float4 sum = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int r0 = 0; r0 < CL; r0 += 4) {  // four ranks' loads in flight, added in rank order
      float4 t[4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + u < CL)
          t[u] = *reinterpret_cast<const float4*>(cl.map_shared_rank(f.Gp, r0 + u) + c * RG +
                                                  4 * d4);
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (r0 + u < CL) {
          sum.x += t[u].x;
          sum.y += t[u].y;
          sum.z += t[u].z;
          sum.w += t[u].w;
        }
    }
    for (int r = 0; r < CL; ++r)
      *reinterpret_cast<float4*>(cl.map_shared_rank(f.G, r) + c * RG + 4 * d4) = sum;
  }
  cl.sync();  // G's upper triangle is complete everywhere; the partials are dead
  for (int e = tid; e < R * R; e += kCluThreads) {
    const int c = e / R, d = e - c * R;
    if (d < c) f.G[c * RG + d] = f.G[d * RG + c];
  }
  // --- G^-1 in place by block Gauss-Jordan with 4 x 4 pivot blocks K. Round:
  // (A) warp 0 inverts P = G[K][K] while the other warps copy the pivot
  // columns G[.][K] (fac) and rows G[K][.] (rowb); (B) z = P^-1 rowb, with
  // P^-1 itself in the columns of K; (C) rows i in K become z, every other
  // row i becomes (G[i] outside K) - G[i][K] z. Three block barriers a round.
  float* fac = f.red;            // R x 4
  float* rowb = f.red + 4 * R;   // 4 x R
  float* zr = f.red + 8 * R;     // 4 x RG (16-byte aligned: 8 R floats are 32 R bytes)
  constexpr int kRowsPerWarp = (RP + kCluWarps - 1) / kCluWarps;
  constexpr int CW = RP <= 64 ? 2 : 4;  // columns per lane
  using VecT = typename std::conditional<CW == 2, float2, float4>::type;
  static_assert(CW * 32 >= RP, "one pass over the columns");
  for (int k = 0; k < R; k += 4) {
    const int bk = R - k < 4 ? R - k : 4;
    const int kb = k + bk;
    __syncthreads();
    if (warp == 0) {
      float pa[4][4], pi[4][4];  // Gauss-Jordan on the bk x bk block, padded with I
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          pa[r][c] = (r < bk && c < bk) ? f.G[(k + r) * RG + k + c] : (r == c ? 1.0f : 0.0f);
          pi[r][c] = r == c ? 1.0f : 0.0f;
        }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float inv = __frcp_rn(pa[q][q]);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          pa[q][c] *= inv;
          pi[q][c] *= inv;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          if (r == q) continue;
          const float fr = pa[r][q];
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            pa[r][c] = fmaf(-fr, pa[q][c], pa[r][c]);
            pi[r][c] = fmaf(-fr, pi[q][c], pi[r][c]);
          }
        }
      }
      if (lane == 0)
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) f.pinv[4 * r + c] = pi[r][c];
    } else {
      for (int e = tid - 32; e < 8 * R; e += kCluThreads - 32) {
        if (e < 4 * R) {
          const int i = e >> 2, c = e & 3;
          fac[e] = c < bk ? f.G[i * RG + k + c] : 0.0f;
        } else {
          const int r = (e - 4 * R) / R, j = e - 4 * R - r * R;
          rowb[r * R + j] = r < bk ? f.G[(k + r) * RG + j] : 0.0f;
        }
      }
    }
    __syncthreads();
    for (int e = tid; e < 4 * RG; e += kCluThreads) {
      const int r = e / RG, j = e - r * RG;
      float t = 0.0f;
      if (r < bk && j < R) {
        if (j >= k && j < kb) {
          t = f.pinv[4 * r + (j - k)];
        } else {
#pragma unroll
          for (int c = 0; c < 4; ++c)
            if (c < bk) t = fmaf(f.pinv[4 * r + c], rowb[c * R + j], t);
        }
      }
      zr[e] = t;
    }
    __syncthreads();
    // a thread's entries: rows warp + 16 t, the CW adjacent columns CW lane ..
    // CW lane + CW - 1 (vector accesses; columns R .. RG - 1 are padding that
    // is computed but never read)
    if (CW * lane < RG) {
      const int j0 = CW * lane;
      VecT zc[4];
#pragma unroll
      for (int c = 0; c < 4; ++c) zc[c] = *reinterpret_cast<const VecT*>(zr + c * RG + j0);
#pragma unroll
      for (int t = 0; t < kRowsPerWarp; ++t) {
        const int i = warp + kCluWarps * t;
        if (i >= R) continue;
        VecT* gp = reinterpret_cast<VecT*>(f.G + i * RG + j0);
        if (i >= k && i < kb) {
          const int r = i - k;  // selected without indexing a register array
          *gp = r == 0 ? zc[0] : r == 1 ? zc[1] : r == 2 ? zc[2] : zc[3];
        } else {
          const float4 fi = *reinterpret_cast<const float4*>(fac + 4 * i);
          VecT g = *gp;
          float* gg = reinterpret_cast<float*>(&g);
#pragma unroll
          for (int u = 0; u < CW; ++u) {
            const int j = j0 + u;
            float v = (j >= k && j < kb) ? 0.0f : gg[u];
            v = fmaf(-fi.x, reinterpret_cast<const float*>(&zc[0])[u], v);
            v = fmaf(-fi.y, reinterpret_cast<const float*>(&zc[1])[u], v);
            v = fmaf(-fi.z, reinterpret_cast<const float*>(&zc[2])[u], v);
            v = fmaf(-fi.w, reinterpret_cast<const float*>(&zc[3])[u], v);
            gg[u] = v;
          }
          *gp = g;
        }
      }
    }
  }
  __syncthreads();  // G holds G^-1; fac, rowb and zr (in red) are read until here
  // --- ADMM on min ||s||_1 s.t. A w + s = b (s = y = 0 at the start, so x = b).
  // Rows belong to warps in groups of 32: thread t handles rows t, t + 512, ...,
  // so a warp's rows form whole groups. Per group the warp first updates each
  // row with the current w (thread = row: A_q . w in float4 steps, then s, y, x)
  // and then adds the group's rows into A^T x (lane = column, x_q read back
  // from shared memory four rows at a time), so no block barrier separates
  // the two.
  // Then: the warps' partial sums (one barrier), this CTA's sum (one barrier),
  // its share of the next w, G^-1 (this CTA's A^T x), pushed to every rank (one
  // cluster barrier), the rank-ordered sum of the shares (one barrier). G^-1 is
  // the same in every CTA and the rank-ordered sum is too, so every CTA holds
  // the same w.
  const float irho = 1.0f / rho;
  // A^T x pass: lane l takes the VW adjacent columns VW l .. VW l + VW - 1
  // (one 8- or 16-byte load per row), four rows per step.
  constexpr int VW = RP <= 64 ? 2 : 4;
  constexpr int NLANE = RP / VW;
  static_assert(RP % 4 == 0 && NLANE <= 32, "columns per lane");
  const bool lane_on = lane < NLANE;
  float acc[VW] = {};
  auto add_row = [&](int row, float xj) {
    const float* src = f.A + row * RS + VW * lane;
    if constexpr (VW == 2) {
      const float2 a2 = *reinterpret_cast<const float2*>(src);
      acc[0] = fmaf(a2.x, xj, acc[0]);
      acc[1] = fmaf(a2.y, xj, acc[1]);
    } else {
      const float4 a4 = *reinterpret_cast<const float4*>(src);
      acc[0] = fmaf(a4.x, xj, acc[0]);
      acc[1] = fmaf(a4.y, xj, acc[1]);
      acc[2] = fmaf(a4.z, xj, acc[2]);
      acc[3] = fmaf(a4.w, xj, acc[3]);
    }
  };
  auto rows_pass = [&](bool update) {
#pragma unroll
    for (int k = 0; k < VW; ++k) acc[k] = 0.0f;
    for (int base = warp * 32; base < mloc; base += kCluThreads) {
      const int q = base + lane;
      float xq = 0.0f;
      if (q < mloc) {
        const float bq = f.b[q];
        if (update) {
          const float aw = clu_row_dot<RP>(f.A + q * RS, f.wv);
          const float yq = f.y[q];
          const float e = bq - aw - yq * irho;
          const float sq = copysignf(fmaxf(fabsf(e) - irho, 0.0f), e);
          const float yn = yq + rho * (aw + sq - bq);
          f.s[q] = sq;
          f.y[q] = yn;
          xq = bq - sq - yn * irho;
        } else {
          f.s[q] = 0.0f;
          f.y[q] = 0.0f;
          xq = bq;
        }
        f.x[q] = xq;
      }
      const int rows_here = mloc - base < 32 ? mloc - base : 32;
      __syncwarp();  // the group's x, written above by each row's thread
      int jq = 0;
      for (; jq + 4 <= rows_here; jq += 4) {
        const float4 x4 = *reinterpret_cast<const float4*>(f.x + base + jq);  // broadcast
        if (lane_on) {
          add_row(base + jq, x4.x);
          add_row(base + jq + 1, x4.y);
          add_row(base + jq + 2, x4.z);
          add_row(base + jq + 3, x4.w);
        }
      }
      for (; jq < rows_here; ++jq)
        if (lane_on) add_row(base + jq, f.x[base + jq]);
    }
  };
  rows_pass(false);  // A^T b
  // this CTA's share of w: GS adjacent lanes share a column c, each summing
  // a CH-long run of the terms of G^-1 (A^T x)_local, then a shuffle tree
  constexpr int GS = kCluThreads / RP >= 8 ? 8 : (kCluThreads / RP >= 4 ? 4 : 2);
  constexpr int CH = ((RP + GS - 1) / GS + 3) / 4 * 4;
  const int gsub = tid % GS;
  for (int c = R + tid; c < RG; c += kCluThreads) f.vec[c] = 0.0f;  // padding of A^T x
  for (int it = 0; it < iters; ++it) {
    if (lane_on) {
#pragma unroll
      for (int k = 0; k < VW; ++k) f.red[warp * RP + VW * lane + k] = acc[k];
    }
    __syncthreads();
    for (int c = tid; c < R; c += kCluThreads) {
      float t = 0.0f;
#pragma unroll
      for (int ww = 0; ww < kCluWarps; ++ww) t += f.red[ww * RP + c];
      f.vec[c] = t;  // this CTA's A^T x
    }
    __syncthreads();
    float* mine = f.xch + (size_t(par) * CL + rank) * kSlot;
    for (int c0 = 0; c0 < R; c0 += kCluThreads / GS) {
      const int c = c0 + tid / GS;
      float t0 = 0.0f, t1 = 0.0f;
      if (c < R) {
#pragma unroll
        for (int q4 = 0; q4 < CH / 4; ++q4) {
          const int d = gsub * CH + 4 * q4;
          if (d < RG) {  // row c of G^-1 (symmetric) against vec; both zero past R
            const float4 g = *reinterpret_cast<const float4*>(f.G + c * RG + d);
            const float4 v = *reinterpret_cast<const float4*>(f.vec + d);
            t0 = fmaf(g.x, v.x, t0);
            t1 = fmaf(g.y, v.y, t1);
            t0 = fmaf(g.z, v.z, t0);
            t1 = fmaf(g.w, v.w, t1);
          }
        }
      }
      float t = t0 + t1;
#pragma unroll
      for (int o = GS / 2; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
      if (c < R)  // every lane of the column's group holds t: lane g pushes to ranks g, g + GS, ...
        for (int r = gsub; r < CL; r += GS) cl.map_shared_rank(mine, r)[c] = t;
    }
    cl.sync();
    for (int c = tid; c < RP; c += kCluThreads) f.wv[c] = c < R ? clu_slot_sum(f, par, c, CL) : 0.0f;
    par ^= 1;
    __syncthreads();
    rows_pass(true);
  }
  __syncthreads();
  // f.wv holds the last iteration's w (entries c >= R are zero)
}

// Rows [q0, q0 + mloc) of the m sampled rows belong to cluster rank `rank`.
__device__ __forceinline__ void clu_rows(int m, int CL, int rank, int& q0, int& mloc) {
  const int per = (m + CL - 1) / CL;
  q0 = rank * per;
  mloc = m - q0 < per ? m - q0 : per;
  if (mloc < 0) mloc = 0;
}

// One training step (Sec. 4.1): sampled rows of the training column, l1
// weights, residual lifted onto the sampled voxels, and the geodesic step's
// coefficients (written to upd). The same launch applies the previous step's
// geodesic update to all of U on its other clusters: the step's fit (cluster
// 0, 16 SMs) and the update (bandwidth-bound, the rest of the GPU) overlap.
struct CluStepArgs {
  const float* U;     // V x RP: U of the previous step when pend_upd is set, else this step's
  const float* pend_upd;   // nullable: coefficients of the previous step's update (not yet
  const float* pend_lift;  // applied to U); the sampled rows are updated here on the fly
  const float* Trow;  // t of this training column (V values)
  const float* samp;  // nullable: t at the step's draws (recovery rows), else Trow[draw]
  uint32_t tag;       // draw tag of the step's samples (training or recovery)
  uint32_t V;
  int R, m, CL;
  uint32_t k0, k1;
  int pass, col;
  float rho, step;
  int iters;
  float* lift;    // V: zero except at the draws of step (clear_pass, clear_col)
  float* upd;     // 3 RP + 4: w, w/||w||, g2, alpha, beta
  float* w_hist;  // nullable
  int fit;        // 1: cluster 0 runs this step's fit; 0: every CTA runs the update
  int clear_pass, clear_col;  // lift entries zeroed before the fit adds to it (-1: none)
  const float* gu_src;        // nullable: U of the previous step ...
  float* gu_dst;              // ... updated into this buffer (all V rows)
  const float* gu_lift;       // that step's lift and coefficients
  const float* gu_coef;
  int gu_chunk;               // rows of U per shared-memory buffer of the update
  uint32_t* status;           // device status word (an update copy that never completes)
};

// Bulk copy of `bytes` from this CTA's shared src to global dst (a bulk group
// of the issuing thread; src, dst and bytes multiples of 16).
__device__ __forceinline__ void bulk_copy_s2g(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src),
               "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
// Waits until this thread's bulk groups have read their shared-memory source
// (kReadOnly) or have completed.
template <bool kReadOnly>
__device__ __forceinline__ void bulk_wait_all() {
  if constexpr (kReadOnly)
    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
  else
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// U_next = U + coef w^T/||w|| over all V rows (geodesic_row), by CTAs
// first_cta.. of the grid. Chunks of gu_chunk rows of U come into shared
// memory by bulk copies (one per row, two buffers: the CTA's next chunk is in
// flight while it updates this one), thread q updates row q of the chunk in
// place, and the row goes back out by a bulk copy. Lane-per-row global loads
// of rows 4 RP bytes apart ran at ~12 GB/s per SM.
template <int RP>
__device__ __forceinline__ void geodesic_rows(const CluStepArgs& a, int first_cta, float* smc,
                                              uint64_t* gbar, int* abort_flag) {
  constexpr int RS = clu_rs(RP);
  constexpr uint32_t kRowBytes = RP * sizeof(float);
  const int tid = threadIdx.x;
  const int CH = a.gu_chunk;
  float* su = smc;  // w, w/||w||, g2, alpha, beta
  float* const buf0 = smc + (3 * RP + 2 + 3) / 4 * 4;  // buffer b at buf0 + b CH RS
  const uint32_t bar0 = smem_addr(&gbar[0]);           // barrier b at bar0 + 8 b
  for (int e = tid; e < 3 * RP + 2; e += kCluThreads) su[e] = a.gu_coef[e];
  if (tid == 0) {
    mbar_init(bar0, 1);
    mbar_init(bar0 + 8u, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  const float alpha = su[3 * RP], beta = su[3 * RP + 1];
  const int64_t V = a.V, nchunks = (V + CH - 1) / CH;
  const int64_t nctas = int64_t(gridDim.x) - first_cta, c0 = int64_t(blockIdx.x) - first_cta;
  auto load = [&](int64_t c, int b) {  // thread 0 arms the barrier; row q's thread copies it
    const int64_t r0 = c * CH;
    const int rows = int(V - r0 < CH ? V - r0 : CH);
    const uint32_t bar = bar0 + 8u * uint32_t(b);
    if (tid == 0) mbar_arrive_expect_tx(bar, uint32_t(rows) * kRowBytes);
    if (tid < rows)
      bulk_copy_g2s(smem_addr(buf0 + (size_t(b) * CH + tid) * RS), a.gu_src + (r0 + tid) * RP,
                    kRowBytes, bar);
  };
  if (c0 < nchunks) load(c0, 0);
  if (c0 + nctas < nchunks) load(c0 + nctas, 1);
  uint32_t phases = 0u;  // bit b: parity of buffer b's next phase
  uint32_t inflight = (c0 < nchunks ? 1u : 0u) | (c0 + nctas < nchunks ? 2u : 0u);  // bit b: buffer b loading
  bool stuck = false;  // a wait expired: no further loads, the rest is skipped
  int k = 0;
  for (int64_t c = c0; c < nchunks && !stuck; c += nctas, ++k) {
    const int b = k & 1;
    const int64_t r0 = c * CH;
    const int rows = int(V - r0 < CH ? V - r0 : CH);
    stuck = __syncthreads_or(!mbar_wait(bar0 + 8u * uint32_t(b), (phases >> b) & 1u, a.status,
                                        abort_flag)) != 0;
    if (stuck) break;
    phases ^= 1u << b;
    inflight &= ~(1u << b);
    if (tid < rows) {
      float4* row = reinterpret_cast<float4*>(buf0 + (size_t(b) * CH + tid) * RS);
      float4 x[RP / 4];
#pragma unroll
      for (int c4 = 0; c4 < RP / 4; ++c4) x[c4] = row[c4];
      geodesic_row<RP>(x, __ldcs(a.gu_lift + r0 + tid), su, su + RP, su + 2 * RP, alpha, beta);
#pragma unroll
      for (int c4 = 0; c4 < RP / 4; ++c4) row[c4] = x[c4];
      fence_proxy_async_smem();  // the row's writes precede its bulk copy out
      bulk_copy_s2g(a.gu_dst + (r0 + tid) * RP, smem_addr(row), kRowBytes);
    }
    if (c + 2 * nctas < nchunks) {  // refill this buffer once every row copy has read it
      bulk_wait_all<true>();
      fence_proxy_async_smem();
      __syncthreads();
      load(c + 2 * nctas, b);
      inflight |= 1u << b;
    }
  }
  // loads still in flight after an expired wait: one more bounded wait each
  // before the CTA (and its shared memory) goes away
  for (int b = 0; b < 2; ++b)
    if (stuck && (inflight >> b & 1u))
      mbar_wait(bar0 + 8u * uint32_t(b), (phases >> b) & 1u, a.status, abort_flag, kWaitLimitNs,
                false);
  bulk_wait_all<false>();
}

template <int RP>
__global__ void __launch_bounds__(kCluThreads, 1) train_step_cluster_kernel(CluStepArgs a) {
  extern __shared__ __align__(16) float smc[];
  __shared__ __align__(8) uint64_t gbar[2];
  __shared__ int gabort;
  const int first = a.fit ? a.CL : 0;  // CTAs [0, CL) form cluster 0
  if (int(blockIdx.x) >= first) {
    if (a.gu_src) geodesic_rows<RP>(a, first, smc, gbar, &gabort);
    return;
  }
  cg::cluster_group cl = cg::this_cluster();
  const int rank = int(cl.block_rank());
  constexpr int RS = clu_rs(RP);
  int q0, mloc;
  clu_rows(a.m, a.CL, rank, q0, mloc);
  CluSmem f;
  clu_carve(smc, (a.m + a.CL - 1) / a.CL, a.R, RP, 0, a.CL, &f);
  const int tid = threadIdx.x;
  if (a.clear_pass >= 0)  // ordered before this step's lift adds by the fit's cluster barriers
    for (int q = tid; q < mloc; q += blockDim.x)
      a.lift[draw_index(a.k0, a.k1, a.tag, uint32_t(q0 + q), uint32_t(a.clear_col),
                        uint32_t(a.clear_pass), a.V)] = 0.0f;
  if (a.pend_upd) {  // the previous update's coefficients, staged in red (free here)
    for (int e = tid; e < 3 * RP + 2; e += blockDim.x) f.red[e] = a.pend_upd[e];
    __syncthreads();
  }
  for (int q = tid; q < mloc; q += blockDim.x) {
    const uint32_t j = draw_index(a.k0, a.k1, a.tag, uint32_t(q0 + q), uint32_t(a.col),
                                  uint32_t(a.pass), a.V);
    f.idx[q] = int32_t(j);
    f.b[q] = a.samp ? a.samp[q0 + q] : a.Trow[j];
    const float4* src = reinterpret_cast<const float4*>(a.U + int64_t(j) * RP);
    float4 x[RP / 4];
#pragma unroll
    for (int c4 = 0; c4 < RP / 4; ++c4) x[c4] = src[c4];
    if (a.pend_upd)
      geodesic_row<RP>(x, a.pend_lift[j], f.red, f.red + RP, f.red + 2 * RP, f.red[3 * RP],
                       f.red[3 * RP + 1]);
    float4* dst = reinterpret_cast<float4*>(f.A + q * RS);
#pragma unroll
    for (int c4 = 0; c4 < RP / 4; ++c4) dst[c4] = x[c4];
  }
  __syncthreads();
  int par = 0;
  clu_l1_fit<RP>(cl, f, mloc, a.R, a.rho, a.iters, a.CL, rank, par);
  // residual r (into x), lifted onto the sampled voxels; A^T r and ||r||^2
  float rr = 0.0f;
  for (int q = tid; q < mloc; q += blockDim.x) {
    const float r = f.b[q] - clu_row_dot<RP>(f.A + q * RS, f.wv);
    f.x[q] = r;
    atomicAdd(&a.lift[f.idx[q]], r);
    rr = fmaf(r, r, rr);
  }
  __syncthreads();
  clu_AtX<RP>(f, mloc, a.R, f.x, f.stage);
  clu_block_sum_to(rr, f, f.stage + a.R);
  clu_sum(cl, f, par, a.R + 1, a.CL, rank);  // the barrier also publishes the lift atomics
  float* g2 = f.misc;                   // keep g2 and ||r||^2 before vec is reused
  if (tid == 0) f.misc[0] = f.vec[a.R];
  float* g2v = f.red;  // R values (red is free now)
  for (int c = tid; c < a.R; c += blockDim.x) g2v[c] = f.vec[c];
  // ||lift||^2 = sum_q lift[idx_q] r_q (a voxel sampled twice holds both r)
  float ll = 0.0f;
  for (int q = tid; q < mloc; q += blockDim.x) ll = fmaf(__ldcg(&a.lift[f.idx[q]]), f.x[q], ll);
  __syncthreads();
  clu_block_sum_to(ll, f, f.stage);
  clu_sum(cl, f, par, 1, a.CL, rank);
  cl.sync();  // no CTA leaves while another may still read its shared memory
  if (rank != 0) return;
  if (tid == 0) {
    const float nr2 = g2[0], nl2 = f.vec[0];
    float nw2 = 0.0f, ng2 = 0.0f;
    for (int c = 0; c < a.R; ++c) {
      nw2 = fmaf(f.wv[c], f.wv[c], nw2);
      ng2 = fmaf(g2v[c], g2v[c], ng2);
    }
    const float nw = sqrtf(nw2);
    const float nG = sqrtf(fmaxf(nl2 - ng2, 0.0f));
    float alpha = 0.0f, beta = 0.0f;
    if (nw > 0.0f && nG > 0.0f) {
      const float theta = a.step * atanf(sqrtf(nr2) / nw);
      alpha = (cosf(theta) - 1.0f) / nw;
      beta = sinf(theta) / nG;
    }
    f.misc[1] = alpha;
    f.misc[2] = beta;
    f.misc[3] = nw;
  }
  __syncthreads();
  const float nw = f.misc[3];
  for (int c = tid; c < RP; c += blockDim.x) {
    const float wc = c < a.R ? f.wv[c] : 0.0f;
    a.upd[c] = wc;
    a.upd[RP + c] = nw > 0.0f ? wc / nw : 0.0f;
    a.upd[2 * RP + c] = c < a.R ? g2v[c] : 0.0f;
    if (a.w_hist && c < a.R) a.w_hist[c] = wc;
  }
  if (tid == 0) {
    a.upd[3 * RP] = f.misc[1];
    a.upd[3 * RP + 1] = f.misc[2];
  }
}

// Sampled t (Alg. 2 recovery): Tt[i - row0][q] = t of relabelling i at its
// q-th drawn voxel. A CTA takes one relabelling (labels in shared memory) and
// 64 draws; a warp computes S dot products at once, lanes over the n_pad
// subjects in float4 steps (T per lane), so many row loads are in flight.
template <int T>
__global__ void __launch_bounds__(256) sampled_t_kernel(const int32_t* __restrict__ perms, int n,
                                                        int n1, int n_pad,
                                                        const float* __restrict__ Xn32,
                                                        uint32_t V, int m, uint32_t k0,
                                                        uint32_t k1, float kf, float ctf,
                                                        int64_t row0, float* __restrict__ Tt) {
  constexpr int S = T <= 2 ? 4 : (T == 4 ? 2 : 1);
  __shared__ __align__(16) float L[32 * 4 * T];
  const int64_t i = row0 + blockIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int s = threadIdx.x; s < 32 * 4 * T; s += blockDim.x) L[s] = 0.0f;
  __syncthreads();
  for (int q = threadIdx.x; q < n1; q += blockDim.x) {
    const int32_t e = perms[i * n + q];
    if (e >= 0 && e < n) L[e] = 1.0f;  // bad rows are reported by validate_perms_kernel
  }
  __syncthreads();
  const int nf4 = n_pad / 4;
  const float4* L4 = reinterpret_cast<const float4*>(L);
  const int qb = blockIdx.y * 64 + warp * 8;
  for (int g = 0; g < 8; g += S) {
    float4 x[S][T];
#pragma unroll
    for (int u = 0; u < S; ++u) {
      const int q = qb + g + u;
      const uint32_t j = q < m ? draw_index(k0, k1, TAG_REC, uint32_t(q), uint32_t(i), 0u, V) : 0u;
      const float4* xr = reinterpret_cast<const float4*>(Xn32 + int64_t(j) * n_pad);
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const int f4 = lane + 32 * t;
        x[u][t] = (q < m && f4 < nf4) ? xr[f4] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
#pragma unroll
    for (int u = 0; u < S; ++u) {
      float p = 0.0f;
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const float4 l = L4[lane + 32 * t];
        p = fmaf(x[u][t].x, l.x, fmaf(x[u][t].y, l.y, fmaf(x[u][t].z, l.z, fmaf(x[u][t].w, l.w, p))));
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) p += __shfl_xor_sync(0xffffffffu, p, o);
      const int q = qb + g + u;
      if (lane == 0 && q < m) {
        const float den = 1.0f - kf * p * p;
        Tt[(i - row0) * m + q] = den > 0.0f ? ctf * p * rsqrtf(den) : (p > 0.0f ? 3.0e38f : -3.0e38f);
      }
    }
  }
}

// Recovery fits (Sec. 4.2), one cluster per relabelling at a time.
struct CluRecArgs {
  const float* Tt;    // (row - row_first) x m: t at the sampled voxels
  uint32_t V;
  int R, m, CL;
  const float* U;     // V x RP
  uint32_t k0, k1;
  float rho;
  int iters;
  int64_t row_first, row_end;
  float* W;           // (row - row_first) x RP
  uint32_t* status;   // device status word (a load that never completes: kErrTimeout)
};

template <int RP>
__global__ void __launch_bounds__(kCluThreads, 1) recover_fit_cluster_kernel(CluRecArgs a) {
  extern __shared__ __align__(16) float smc[];
  __shared__ __align__(8) unsigned long long load_bar;
  __shared__ int abort_flag;
  cg::cluster_group cl = cg::this_cluster();
  const int rank = int(cl.block_rank());
  const int64_t cid = blockIdx.x / a.CL, ncl = gridDim.x / a.CL;
  constexpr int RS = clu_rs(RP);
  constexpr uint32_t kRowBytes = RP * sizeof(float);
  int q0, mloc;
  clu_rows(a.m, a.CL, rank, q0, mloc);
  CluSmem f;
  clu_carve(smc, (a.m + a.CL - 1) / a.CL, a.R, RP, 0, a.CL, &f);
  const int tid = threadIdx.x;
  const uint32_t bar = smem_addr(&load_bar);
  if (tid == 0) {
    mbar_init(bar, 1);
    abort_flag = 0;
    fence_mbar_init();
  }
  __syncthreads();
  int par = 0;
  uint32_t phase = 0;
  bool have_idx = false;  // f.idx holds this relabelling's draws (from the previous prefetch)
  bool stuck = false;     // a load whose wait expired may still be in flight (phase `phase`)
  for (int64_t i = a.row_first + cid; i < a.row_end; i += ncl) {
    // this relabelling's rows of U, one bulk copy per row (each thread copies
    // the rows whose draws it holds), completing on load_bar; after an expired
    // wait no further copies are issued (the fits then run on stale rows and
    // the status word reports the timeout)
    if (!have_idx)
      for (int q = tid; q < mloc; q += kCluThreads)
        f.idx[q] = int32_t(draw_index(a.k0, a.k1, TAG_REC, uint32_t(q0 + q), uint32_t(i), 0u, a.V));
    if (!stuck) {
      if (tid == 0) mbar_arrive_expect_tx(bar, uint32_t(mloc) * kRowBytes);
      fence_proxy_async_smem();  // the last relabelling's reads of A precede the copies
      __syncthreads();
      for (int q = tid; q < mloc; q += kCluThreads)
        bulk_copy_g2s(smem_addr(f.A + q * RS), a.U + int64_t(f.idx[q]) * RP, kRowBytes, bar);
    }
    const float* trow = a.Tt + (i - a.row_first) * a.m + q0;
    for (int q = tid; q < mloc; q += kCluThreads) f.b[q] = trow[q];
    if (!stuck) {  // a wait that expired in any thread stops the loads for the whole CTA
      stuck = __syncthreads_or(!mbar_wait(bar, phase, a.status, &abort_flag)) != 0;
      if (!stuck) phase ^= 1u;
    } else {
      __syncthreads();
    }
    // the next relabelling's rows of U go into L2 while this one is fitted
    // (each thread keeps the draws of the rows it will copy)
    have_idx = i + ncl < a.row_end;
    if (have_idx)
      for (int q = tid; q < mloc; q += kCluThreads) {
        const uint32_t jn = draw_index(a.k0, a.k1, TAG_REC, uint32_t(q0 + q), uint32_t(i + ncl), 0u, a.V);
        f.idx[q] = int32_t(jn);
        prefetch_l2_bulk(a.U + int64_t(jn) * RP, kRowBytes);
      }
    clu_l1_fit<RP>(cl, f, mloc, a.R, a.rho, a.iters, a.CL, rank, par);
    if (rank == 0)
      for (int c = tid; c < RP; c += kCluThreads)
        a.W[(i - a.row_first) * RP + c] = c < a.R ? f.wv[c] : 0.0f;
    __syncthreads();
  }
  // copies of a load whose wait expired: one more bounded wait before the CTA
  // (and its shared memory) goes away
  if (stuck) mbar_wait(bar, phase, a.status, &abort_flag, kWaitLimitNs, false);
  cl.sync();  // no CTA leaves while another may still read its shared memory
}

__device__ __forceinline__ float row_dot_rt(const float* __restrict__ row,
                                            const float* __restrict__ v, int RP) {
  float t = 0.0f;
  for (int c = 0; c < RP; ++c) t = fmaf(row[c], v[c], t);
  return t;
}

// ---------------------------------------------------------------------------
// U0 and QR
// ---------------------------------------------------------------------------
__global__ void u0_kernel(float* __restrict__ U, int64_t V, int R, int RP, uint32_t k0,
                          uint32_t k1) {
  const int64_t total = V * RP;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = e / RP;
    const int c = int(e - j * RP);
    U[e] = c < R ? draw_normal(k0, k1, TAG_U0, uint32_t(j), uint32_t(c)) : 0.0f;
  }
}

// Partial Gram matrices U^T U over row ranges, for the QR of U: 4 x 4 tiles of
// the upper triangle per thread, products exact as float pairs (FMA residual)
// and sums in float-float (~44 bits; the FP32 pipes are many times the FP64
// rate here); each (block, row group) writes its tile sums as FP64 partials
// indexed like the pairs (c <= d) of the factorisation.
constexpr int kGramThreads = 256;
__global__ void __launch_bounds__(kGramThreads) gram_ff_kernel(const float* __restrict__ U,
                                                               int64_t V, int R, int RP,
                                                               int ngroups,
                                                               double* __restrict__ partials) {
  const int RT = RP / 4, ntile = RT * (RT + 1) / 2;
  const int npairs = R * (R + 1) / 2;
  const int64_t per = (V + gridDim.x - 1) / gridDim.x;
  const int64_t j0 = blockIdx.x * per, j1 = min(V, j0 + per);
  for (int t = threadIdx.x; t < ntile * ngroups; t += blockDim.x) {
    const int tile = t % ntile, g = t / ntile;
    int ti = 0, rem = tile;
    while (rem >= RT - ti) {
      rem -= RT - ti;
      ++ti;
    }
    const int tj = ti + rem;
    float h[4][4], l[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) h[a][b] = l[a][b] = 0.0f;
    for (int64_t j = j0 + g; j < j1; j += ngroups) {
      const float4 u = *reinterpret_cast<const float4*>(U + j * RP + 4 * ti);
      const float4 v = *reinterpret_cast<const float4*>(U + j * RP + 4 * tj);
      const float uu[4] = {u.x, u.y, u.z, u.w}, vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const float p = uu[a] * vv[b];
          ff_acc(h[a][b], l[a][b], p, fmaf(uu[a], vv[b], -p));
        }
    }
    double* out = partials + (int64_t(blockIdx.x) * ngroups + g) * npairs;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int c = 4 * ti + a, d = 4 * tj + b;
        if (c <= d && d < R) out[c * R - c * (c - 1) / 2 + (d - c)] = ff_d(h[a][b], l[a][b]);
      }
  }
}

// One block: sum the partial Grams (FP64, block order), Cholesky G = R^T R,
// R^-1 (upper), stored as FP32 RP x RP (zero padded).
__global__ void __launch_bounds__(1024) qr_factor_kernel(const double* __restrict__ partials,
                                                         int nparts, int R, int RP,
                                                         float* __restrict__ Rinv_out) {
  extern __shared__ double dsm[];
  double* G = dsm;        // R x R: upper factor R above/on the diagonal, R^-1 (off-diagonal,
                          // transposed) below it
  double* dg = G + R * R;  // diagonal of R^-1
  const int npairs = R * (R + 1) / 2;
  for (int pi = threadIdx.x; pi < npairs; pi += blockDim.x) {
    double t = 0.0;
    for (int b = 0; b < nparts; ++b) t += partials[int64_t(b) * npairs + pi];
    int c = 0, rem = pi;
    while (rem >= R - c) {
      rem -= R - c;
      ++c;
    }
    const int d = c + rem;
    G[c * R + d] = t;
    G[d * R + c] = t;
  }
  __syncthreads();
  // Cholesky, upper factor: G = R^T R, R[k][k] > 0 (stored in the upper triangle of G)
  for (int k = 0; k < R; ++k) {
    if (threadIdx.x == 0) G[k * R + k] = sqrt(fmax(G[k * R + k], 1e-300));
    __syncthreads();
    const double dk = G[k * R + k];
    for (int j = k + 1 + threadIdx.x; j < R; j += blockDim.x) G[k * R + j] /= dk;
    __syncthreads();
    const int nt = R - k - 1;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
      const int i = k + 1 + e / nt, j = k + 1 + e % nt;
      if (j >= i) G[i * R + j] -= G[k * R + i] * G[k * R + j];
    }
    __syncthreads();
  }
  // R^-1 (upper) by columns: back substitution of R x = e_c. Entry (i, c), i < c,
  // is kept at G[c][i]; the diagonal 1/R[c][c] in dg[c].
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    dg[c] = 1.0 / G[c * R + c];
    for (int i = c - 1; i >= 0; --i) {
      double t = 0.0;
      for (int k = i + 1; k <= c; ++k) t -= G[i * R + k] * (k == c ? dg[c] : G[c * R + k]);
      G[c * R + i] = t / G[i * R + i];
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) {
    const int i = e / RP, j = e % RP;
    float x = 0.0f;
    if (i < R && j < R && i <= j) x = float(i == j ? dg[j] : G[j * R + i]);
    Rinv_out[e] = x;
  }
}

// U[j] <- U[j] R^-1 (row times upper-triangular matrix).
__global__ void qr_apply_kernel(float* __restrict__ U, int64_t V, int R, int RP,
                                const float* __restrict__ Rinv) {
  extern __shared__ float ri[];
  for (int e = threadIdx.x; e < RP * RP; e += blockDim.x) ri[e] = Rinv[e];
  __syncthreads();
  float row[kMaxRank];
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < V;
       j += int64_t(gridDim.x) * blockDim.x) {
    float* u = U + j * RP;
    for (int c = 0; c < R; ++c) row[c] = u[c];
    for (int c = 0; c < R; ++c) {
      float t = 0.0f;
      for (int k = 0; k <= c; ++k) t = fmaf(row[k], ri[k * RP + c], t);
      u[c] = t;
    }
  }
}

// ---------------------------------------------------------------------------
// W_ex = U^T T_ex^T (split over voxels, FP64 reduction of the splits)
// ---------------------------------------------------------------------------
// part[split][i][c] = sum over the split's voxels j of T_ex[i][j] U[j][c] for one
// 64 x 64 tile of (training column i, basis column c) per CTA: 32-voxel slabs of
// T_ex (read along voxels, stored voxel-major) and of U in shared memory, a 4 x 4
// register tile per thread (16 FMAs per two 16-byte shared loads).
constexpr int kWexTile = 64;
__global__ void __launch_bounds__(256) wex_partial_kernel(const float* __restrict__ U,
                                                          const float* __restrict__ Tex,
                                                          int64_t V, int ell, int RP,
                                                          int64_t per_split,
                                                          float* __restrict__ part) {
  __shared__ __align__(16) float Ts[32][kWexTile + 4];  // [voxel][training column]
  __shared__ __align__(16) float Us[32][kWexTile + 4];  // [voxel][basis column]
  const int i0 = blockIdx.x * kWexTile, c0 = blockIdx.z * kWexTile;
  const int64_t j0 = blockIdx.y * per_split, j1 = min(V, j0 + per_split);
  const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
  float acc[4][4];
#pragma unroll
  for (int q = 0; q < 4; ++q)
#pragma unroll
    for (int p = 0; p < 4; ++p) acc[q][p] = 0.0f;
  for (int64_t jb = j0; jb < j1; jb += 32) {
    for (int e = tid; e < kWexTile * 32; e += 256) {
      const int r = e >> 5, jj = e & 31;
      const int64_t j = jb + jj;
      Ts[jj][r] = (i0 + r < ell && j < j1) ? __ldcs(&Tex[int64_t(i0 + r) * V + j]) : 0.0f;
    }
    for (int e = tid; e < 32 * kWexTile; e += 256) {
      const int jj = e >> 6, c = e & (kWexTile - 1);
      const int64_t j = jb + jj;
      Us[jj][c] = (c0 + c < RP && j < j1) ? U[j * RP + c0 + c] : 0.0f;
    }
    __syncthreads();
#pragma unroll 8
    for (int jj = 0; jj < 32; ++jj) {
      const float4 t = *reinterpret_cast<const float4*>(&Ts[jj][4 * tr]);
      const float4 u = *reinterpret_cast<const float4*>(&Us[jj][4 * tc]);
      const float tv[4] = {t.x, t.y, t.z, t.w}, uv[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int p = 0; p < 4; ++p) acc[q][p] = fmaf(tv[q], uv[p], acc[q][p]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + 4 * tr + q;
    if (i >= ell) continue;
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int c = c0 + 4 * tc + p;
      if (c < RP) part[(int64_t(blockIdx.y) * ell + i) * RP + c] = acc[q][p];
    }
  }
}

// W[i][c] = sum over splits (FP64); W is ell x RP (row i = weights of column i).
__global__ void wex_reduce_kernel(const float* __restrict__ part, int nsplit, int ell, int RP,
                                  float* __restrict__ W) {
  const int64_t total = int64_t(ell) * RP;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    double t = 0.0;
    for (int s = 0; s < nsplit; ++s) t += double(part[int64_t(s) * total + e]);
    W[e] = float(t);
  }
}

// Sampled residuals of the last pass: sum and sum of squares per block (FP64).
__global__ void __launch_bounds__(256) sigma_partial_kernel(
    const float* __restrict__ U, const float* __restrict__ Tex, const float* __restrict__ W,
    uint32_t V, int ell, int m, int RP, uint32_t k0, uint32_t k1, int pass,
    double* __restrict__ part) {
  __shared__ double red[2][8];
  double s1 = 0.0, s2 = 0.0;
  const int64_t total = int64_t(ell) * m;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(e / m), q = int(e - int64_t(i) * m);
    const uint32_t j = draw_index(k0, k1, TAG_TRAIN, uint32_t(q), uint32_t(i), uint32_t(pass), V);
    const float r = Tex[int64_t(i) * V + j] - row_dot_rt(U + int64_t(j) * RP, W + int64_t(i) * RP, RP);
    s1 += r;
    s2 += double(r) * r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    s2 += __shfl_xor_sync(0xffffffffu, s2, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s1;
    red[1][threadIdx.x >> 5] = s2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < 8; ++w) {
      a += red[0][w];
      c += red[1][w];
    }
    part[2 * blockIdx.x] = a;
    part[2 * blockIdx.x + 1] = c;
  }
}

// ---------------------------------------------------------------------------
// Residual max (Alg. 2, the literal training shift): rows = training columns
// (weights W_ex), columns = voxels; max_j (T_ex[i][j] - (U w_i)_j). Each CTA
// walks a range of voxel tiles for one 128-row tile and keeps per-row maxima.
// ---------------------------------------------------------------------------
struct ResidArgs {
  const float* W;  // rows x RP
  int64_t rows;
  const float* U;  // V x RP
  int64_t V;
  int RP;
  const float* Tex;  // rows x V
  int64_t tiles_per_cta;
  unsigned long long* maxkey;  // rows, zero on entry
};

__global__ void __launch_bounds__(256) residual_max_kernel(ResidArgs a) {
  __shared__ __align__(16) float Ws[16][128];
  __shared__ __align__(16) float Us[16][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = int64_t(blockIdx.y) * 128;
  const int64_t vt0 = int64_t(blockIdx.x) * a.tiles_per_cta;
  const int64_t vtiles = (a.V + 127) / 128;
  const int64_t vt1 = min(vtiles, vt0 + a.tiles_per_cta);
  float best[8];
  uint32_t bj[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    best[q] = -INFINITY;
    bj[q] = 0xffffffffu;
  }
  for (int64_t vt = vt0; vt < vt1; ++vt) {
    const int64_t c0 = vt * 128;
    float acc[8][8];
#pragma unroll
    for (int p = 0; p < 8; ++p)
#pragma unroll
      for (int q = 0; q < 8; ++q) acc[p][q] = 0.0f;
    for (int k0 = 0; k0 < a.RP; k0 += 16) {
      __syncthreads();
      for (int e = tid; e < 16 * 128; e += 256) {
        const int rr = e >> 4, kk = e & 15;
        const int64_t row = r0 + rr, col = c0 + rr;
        Ws[kk][rr] = (row < a.rows && k0 + kk < a.RP) ? a.W[row * a.RP + k0 + kk] : 0.0f;
        Us[kk][rr] = (col < a.V && k0 + kk < a.RP) ? a.U[col * a.RP + k0 + kk] : 0.0f;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) {
        const float4 w0 = *reinterpret_cast<const float4*>(&Ws[kk][ty * 4]);
        const float4 w1 = *reinterpret_cast<const float4*>(&Ws[kk][64 + ty * 4]);
        const float4 u0 = *reinterpret_cast<const float4*>(&Us[kk][tx * 4]);
        const float4 u1 = *reinterpret_cast<const float4*>(&Us[kk][64 + tx * 4]);
        const float wv[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
        const float uv[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
#pragma unroll
        for (int p = 0; p < 8; ++p)
#pragma unroll
          for (int q = 0; q < 8; ++q) acc[p][q] = fmaf(wv[p], uv[q], acc[p][q]);
      }
    }
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int64_t row = r0 + ((p < 4) ? (ty * 4 + p) : (64 + ty * 4 + p - 4));
      if (row >= a.rows) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t cc = c0 + ((q < 4) ? (tx * 4 + q) : (64 + tx * 4 + q - 4));
        if (cc >= a.V) continue;
        const float val = a.Tex[row * a.V + cc] - acc[p][q];
        if (val > best[p] || (val == best[p] && uint32_t(cc) < bj[p])) {
          best[p] = val;
          bj[p] = uint32_t(cc);
        }
      }
    }
  }
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    float bv = best[p];
    uint32_t bi = bj[p];
#pragma unroll
    for (int o = 1; o < 16; o <<= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, bv, o);
      const uint32_t oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > bv || (ob == bv && oi < bi)) {
        bv = ob;
        bi = oi;
      }
    }
    const int64_t row = r0 + ((p < 4) ? (ty * 4 + p) : (64 + ty * 4 + p - 4));
    if (tx == 0 && row < a.rows && bi != 0xffffffffu) {
      const unsigned long long key = pack_key(bv, bi);
      if (key > __ldcg(&a.maxkey[row])) atomicMax(&a.maxkey[row], key);
    }
  }
}

// One warp per relabelling row: entries in range and distinct.
__global__ void validate_perms_kernel(const int32_t* __restrict__ perms, int64_t row0, int64_t P,
                                      int n, uint32_t* __restrict__ status) {
  __shared__ uint32_t seen_all[8][32];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint32_t* seen = seen_all[wib];
  for (int64_t i = row0 + int64_t(blockIdx.x) * 8 + wib; i < P; i += int64_t(gridDim.x) * 8) {
    seen[lane] = 0u;
    __syncwarp();
    bool bad = false;
    for (int q = lane; q < n; q += 32) {
      const int32_t e = perms[i * n + q];
      if (e < 0 || e >= n) {
        bad = true;
        continue;
      }
      const uint32_t bit = 1u << (e & 31);
      if (atomicOr(&seen[e >> 5], bit) & bit) bad = true;
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(status, kErrBadPerm);
    __syncwarp();
  }
}

__global__ void keys_to_values_kernel(const unsigned long long* __restrict__ keys, int64_t rows,
                                      float shift, float* __restrict__ out) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < rows;
       i += int64_t(gridDim.x) * blockDim.x) {
    const unsigned long long k = keys[i];
    out[i] = k ? unpack_key_value(k) + shift : -INFINITY;
  }
}

__global__ void u_to_t_kernel(float* __restrict__ T, int64_t total, float kf, float ctf) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const float u = T[e];
    const float den = 1.0f - kf * u * u;
    T[e] = den > 0.0f ? ctf * u * rsqrtf(den) : (u > 0.0f ? INFINITY : -INFINITY);
  }
}

// Rows of t in compact (valid-voxel) order -> rows in mask order; voxels
// without a statistic keep the NaN the destination was filled with.
__global__ void scatter_rows_kernel(const float* __restrict__ src, int64_t P, int64_t V,
                                    const int32_t* __restrict__ valid_map, int64_t v,
                                    float* __restrict__ dst) {
  const int64_t total = P * V;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / V, c = e - i * V;
    dst[i * v + valid_map[c]] = src[e];
  }
}

__global__ void pack_u_kernel(const float* __restrict__ Uin, int64_t V, int R, int RP,
                              float* __restrict__ Uout, int to_padded) {
  const int64_t total = V * RP;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t j = e / RP;
    const int c = int(e - j * RP);
    if (to_padded) Uout[e] = c < R ? Uin[j * R + c] : 0.0f;
    else if (c < R) Uout[j * R + c] = Uin[e];
  }
}

// Padded rank RP: the rank rounded up to 4 (to 8 above 64), so rows of U stay
// 16-byte aligned without wasting HBM traffic on padding columns (U is
// streamed by every geodesic update).
constexpr int padded_rank(int rank) { return rank <= 64 ? (rank + 3) / 4 * 4 : (rank + 7) / 8 * 8; }

template <int RP, class F>
bool with_rp_tail(int rp, F&& f) {
  if constexpr (RP > kMaxRank) {
    return false;
  } else {
    if (rp == RP) {
      f(std::integral_constant<int, RP>{});
      return true;
    }
    return with_rp_tail<(RP < 64 ? RP + 4 : RP + 8)>(rp, f);
  }
}

// Calls f(std::integral_constant<int, RP>) for the padded rank RP (4..128).
template <class F>
bool with_rp(int rp, F&& f) {
  return with_rp_tail<4>(rp, f);
}

int grid_n(int64_t work, int threads, int cap = 152 * 16) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return int(b);
}

constexpr size_t kCluSmemLimit = 227 * 1024 - 64;  // the kernels add a few static bytes

// Sequential fits (training steps, recovery with U updates) take 16-CTA
// clusters: one fit at a time is latency-bound, and fewer rows per CTA win over
// the dearer exchange (at r = 50, m = 1750 an ADMM iteration took ~5.6k cycles
// on 16 CTAs, ~3.7k of them the exchange, and about twice that on 4 CTAs).
constexpr int kTrainMinCluster = 16;

// Smallest cluster size (from `first`, doubling up to 16) whose per-CTA share
// of the sampled rows fits in shared memory; 0 if none does.
int choose_cluster(int m, int R, int RP, int n_pad, int first, size_t* smem) {
  for (int CL = first; CL <= 16; CL *= 2) {
    const size_t b = clu_carve(nullptr, (m + CL - 1) / CL, R, RP, n_pad, CL, nullptr);
    if (b <= kCluSmemLimit) {
      *smem = b;
      return CL;
    }
  }
  return 0;
}

// Shared memory of the training step's whole-U update (geodesic_rows): the
// coefficients and two buffers of *chunk rows (256, fewer when that does not
// fit).
size_t update_smem(int RP, int* chunk) {
  const size_t coef = size_t(3 * RP + 2 + 3) / 4 * 4 * sizeof(float);
  const size_t row = size_t(clu_rs(RP)) * sizeof(float);
  int ch = 256;
  while (ch > 32 && coef + 2 * size_t(ch) * row > kCluSmemLimit - 4096) ch -= 32;
  *chunk = ch;
  return coef + 2 * size_t(ch) * row;
}

// Launch configuration of `kernel` as clusters of CL CTAs of kCluThreads threads.
template <class Arg>
cudaError_t cluster_config(void (*kernel)(Arg), int CL, size_t smem, cudaStream_t st,
                           cudaLaunchConfig_t* cfg, cudaLaunchAttribute* at) {
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(smem));
  if (e == cudaSuccess && CL > 8)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = unsigned(CL);
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  *cfg = cudaLaunchConfig_t{};
  cfg->blockDim = dim3(kCluThreads, 1, 1);
  cfg->dynamicSmemBytes = smem;
  cfg->stream = st;
  cfg->attrs = at;
  cfg->numAttrs = 1;
  cfg->gridDim = dim3(unsigned(CL) * 152u, 1, 1);
  return cudaSuccess;
}

// How many clusters of `kernel` can be resident at once (>= 1 on success).
template <class Arg>
cudaError_t max_active_clusters(void (*kernel)(Arg), int CL, size_t smem, int* maxc) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  cudaError_t e = cluster_config(kernel, CL, smem, nullptr, &cfg, at);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(maxc, kernel, &cfg);
  if (e == cudaSuccess && *maxc < 1) e = cudaErrorInvalidConfiguration;
  return e;
}

// Launches `kernel` as nclusters clusters of CL CTAs of kCluThreads threads;
// nclusters <= 0 asks for as many clusters as can be resident at once (at most
// -nclusters when that is positive).
template <class Arg>
cudaError_t launch_cluster(void (*kernel)(Arg), int nclusters, int CL, size_t smem,
                           cudaStream_t st, const Arg& arg, int* used = nullptr) {
  cudaLaunchConfig_t cfg;
  cudaLaunchAttribute at[1];
  cudaError_t e = cluster_config(kernel, CL, smem, st, &cfg, at);
  if (e != cudaSuccess) return e;
  if (nclusters <= 0) {
    int maxc = 0;
    e = cudaOccupancyMaxActiveClusters(&maxc, kernel, &cfg);
    if (e != cudaSuccess) return e;
    if (maxc < 1) return cudaErrorInvalidConfiguration;
    nclusters = -nclusters > 0 && -nclusters < maxc ? -nclusters : maxc;
  }
  cfg.gridDim = dim3(unsigned(CL) * unsigned(nclusters), 1, 1);
  if (used) *used = nclusters;
  return cudaLaunchKernelEx(&cfg, kernel, arg);
}

pt_status nomem_r(pt_ctx* ctx, const char* what) {
  set_error(ctx, std::string("out of device memory (") + what + ")");
  return PT_ERR_NOMEM;
}

struct RapidPlan {
  int R, RP;
  int64_t V;
  int m;
  uint32_t k0, k1;
};

pt_status check_rapid_args(pt_ctx* ctx, int32_t rank, double sample_rate, const pt_rapid_opts& o,
                           RapidPlan& pl) {
  if (ctx->glm_q1) {
    set_error(ctx, "RapidPT runs the plain two-sample t (context prepared with covariates)");
    return PT_ERR_UNSUPPORTED;
  }
  if (rank < 1 || rank > kMaxRank || rank > ctx->n) {
    set_error(ctx, "RapidPT: need 1 <= rank <= min(n, 128)");
    return PT_ERR_INVALID;
  }
  if (!(sample_rate > 0.0) || sample_rate > 1.0) {
    set_error(ctx, "RapidPT: need 0 < sample_rate <= 1");
    return PT_ERR_INVALID;
  }
  if (o.train_passes < 1 || o.qr_every < 1 || o.admm_iters < 1 || !(o.admm_rho > 0.0f) ||
      !(o.step > 0.0f) || o.shift_mode < 0 || o.shift_mode > 1 || o.precision < 0 ||
      o.precision > PT_PREC_FP16X2 || !(o.rec_step >= 0.0f) || !(o.rec_step < 1e30f)) {
    set_error(ctx, "RapidPT: bad options");
    return PT_ERR_INVALID;
  }
  if (ctx->v_valid < 1 || ctx->v_valid >= (int64_t(1) << 31)) {
    set_error(ctx, "RapidPT: context has no voxel with a defined t");
    return PT_ERR_INVALID;
  }
  pl.R = rank;
  pl.RP = padded_rank(rank);
  pl.V = ctx->v_valid;
  pl.m = int(std::ceil(sample_rate * double(pl.V)));
  if (pl.m < rank) {
    set_error(ctx, "RapidPT: ceil(sample_rate * v) must be at least the rank");
    return PT_ERR_INVALID;
  }
  size_t fit_smem = 0;
  if (choose_cluster(pl.m, pl.R, pl.RP, 0, 16, &fit_smem) == 0) {
    set_error(ctx, "RapidPT: the m sampled rows of a relabelling do not fit the shared memory "
                   "of a 16-CTA cluster (lower sample_rate or rank)");
    return PT_ERR_UNSUPPORTED;
  }
  pl.k0 = uint32_t(o.seed & 0xffffffffull);
  pl.k1 = uint32_t(o.seed >> 32);
  return PT_OK;
}

// Orthonormalise U (V x RP) in place: FP64 Gram and factorisation, FP32 apply.
pt_status qr_inplace(pt_ctx* ctx, float* U, const RapidPlan& pl, Buf& part, Buf& rinv) {
  const int nblocks = 152 * 2;
  const int ntile = (pl.RP / 4) * (pl.RP / 4 + 1) / 2;
  const int ngroups = std::max(1, kGramThreads / ntile);
  const int nparts = nblocks * ngroups;
  const int npairs = pl.R * (pl.R + 1) / 2;
  if (!part.ensure(sizeof(double) * size_t(nparts) * npairs) ||
      !rinv.ensure(sizeof(float) * pl.RP * pl.RP))
    return nomem_r(ctx, "QR");
  gram_ff_kernel<<<nblocks, kGramThreads, 0, ctx->stream>>>(U, pl.V, pl.R, pl.RP, ngroups,
                                                            part.as<double>());
  PT_LAUNCH_CHECK(ctx);
  const int fsm = (pl.R * pl.R + pl.R) * int(sizeof(double));
  if (fsm > 48 * 1024)
    PT_CUDA_TRY(ctx, cudaFuncSetAttribute(qr_factor_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, fsm));
  qr_factor_kernel<<<1, 1024, fsm, ctx->stream>>>(part.as<double>(), nparts, pl.R, pl.RP,
                                                  rinv.as<float>());
  PT_LAUNCH_CHECK(ctx);
  {
    // R^-1 in shared memory: 64 KB at RP = 128, above the 48 KB default
    const size_t asm_bytes = sizeof(float) * size_t(pl.RP) * pl.RP;
    PT_CUDA_TRY(ctx, cudaFuncSetAttribute(qr_apply_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          int(asm_bytes)));
    qr_apply_kernel<<<grid_n(pl.V, 256), 256, asm_bytes, ctx->stream>>>(U, pl.V, pl.R, pl.RP,
                                                                      rinv.as<float>());
    PT_LAUNCH_CHECK(ctx);
  }
  return PT_OK;
}

// Row maxima of (U w + sigma z) (mode 0) or of T_ex - U w (mode 1) for `rows`
// rows of W; keys zeroed here.
// Per-row maxima (packed keys) of the reconstructed rows: mode 0 adds the
// noise sigma z(tag, voxel, label0 + row) on the tensor cores; mode 1 is the
// residual T_ex - U W_ex.
pt_status reconstruct(pt_ctx* ctx, const float* W, int64_t rows, int64_t label0, const float* U,
                      const RapidPlan& pl, float sigma, uint32_t tag, int mode, const float* Tex,
                      unsigned long long* keys) {
  PT_CUDA_TRY(ctx, cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * rows, ctx->stream));
  if (mode == 0)
    return recon_tc(ctx, W, rows, label0, U, pl.V, pl.RP, sigma, tag, pl.k0, pl.k1, keys);
  const int64_t rtiles = (rows + 127) / 128;
  const int64_t vtiles = (pl.V + 127) / 128;
  int64_t per = vtiles;
  const int64_t want = 152 * 8;
  if (rtiles < want) {
    int64_t split = (want + rtiles - 1) / rtiles;
    if (split > vtiles) split = vtiles;
    per = (vtiles + split - 1) / split;
  }
  ResidArgs a;
  a.W = W;
  a.rows = rows;
  a.U = U;
  a.V = pl.V;
  a.RP = pl.RP;
  a.Tex = Tex;
  a.tiles_per_cta = per;
  a.maxkey = keys;
  const dim3 grid{unsigned((vtiles + per - 1) / per), unsigned(rtiles), 1u};
  residual_max_kernel<<<grid, 256, 0, ctx->stream>>>(a);
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// Training
// ---------------------------------------------------------------------------
pt_status rapid_train_impl(pt_ctx* ctx, const int32_t* perms, int32_t n_train, int32_t rank,
                           double sample_rate, const pt_rapid_opts& o, float* U_out,
                           float* train_max, uint32_t* counts, float* w_hist,
                           pt_rapid_info* info) {
  RapidPlan pl;
  pt_status s = check_rapid_args(ctx, rank, sample_rate, o, pl);
  if (s != PT_OK) return s;
  if (n_train < 1) {
    set_error(ctx, "RapidPT: need n_train >= 1");
    return PT_ERR_INVALID;
  }
  cudaStream_t st = ctx->stream;
  const int64_t V = pl.V;
  const int ell = n_train;
  Buf Ub, Ub2, Tex, lift, upd, part, rinv, Wex, keys, sig, tmax;
  struct G {
    std::vector<Buf*> v;
    ~G() {
      for (Buf* b : v) b->release();
    }
  } guard{{&Ub, &Ub2, &Tex, &lift, &upd, &part, &rinv, &Wex, &keys, &sig, &tmax}};
  const int updw = 3 * pl.RP + 4;  // floats per step's update coefficients
  if (!Ub.ensure(sizeof(float) * size_t(V) * pl.RP) ||
      !Ub2.ensure(sizeof(float) * size_t(V) * pl.RP) || !Tex.ensure(sizeof(float) * size_t(ell) * V) ||
      !lift.ensure(sizeof(float) * 2 * V) ||
      !upd.ensure(sizeof(float) * 2 * updw) || !Wex.ensure(sizeof(float) * size_t(ell) * pl.RP) ||
      !keys.ensure(sizeof(unsigned long long) * ell) || !tmax.ensure(sizeof(float) * ell))
    return nomem_r(ctx, "RapidPT training");

  // 1. training rows: maxima (exact winner) and counts through the NaivePT
  //    path, and the t rows T_ex.
  {
    if (!ctx->maxkey.ensure(sizeof(unsigned long long) * ell) ||
        !ctx->cnt.ensure(sizeof(uint32_t) * (V + 1)))
      return nomem_r(ctx, "workspace");
    PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->maxkey.p, 0, sizeof(unsigned long long) * ell, st));
    PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cnt.p, 0, sizeof(uint32_t) * (V + 1), st));
    if (counts) PT_CUDA_TRY(ctx, cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ctx->v, st));
    int64_t P_pad = 0;
    const bool tc = o.precision != PT_PREC_FP32;
    if (tc) {
      s = tc_supported(ctx);
      if (s == PT_OK) s = ensure_xnb(ctx, o.precision);
      if (s == PT_OK) s = build_labels(ctx, perms, ell, prec_label_layout(o.precision), &P_pad);
      if (s == PT_OK)
        s = tc_rows(ctx, ctx->labels.p, ell, o.precision, 2, Tex.as<float>(), 1, 0,
                    ctx->u_obs.as<float>(), ctx->maxkey.as<unsigned long long>(),
                    ctx->cnt.as<uint32_t>());
    } else {
      s = ensure_xn32(ctx);
      if (s == PT_OK) s = build_labels(ctx, perms, ell, 0, &P_pad);
      if (s == PT_OK) {
        const int64_t vt = (V + 127) / 128, pt = (ell + 127) / 128;
        const dim3 grid{unsigned(vt), unsigned(pt), 1u};
        simt_contract_kernel<<<grid, 256, 0, st>>>(ctx->labels.as<float>(), ctx->Xn32.as<float>(),
                                                   ctx->n_pad, ell, V, 1, 0, 0,
                                                   ctx->u_obs.as<float>(), ctx->rowflag.as<uint8_t>(),
                                                   ctx->maxkey.as<unsigned long long>(),
                                                   ctx->cnt.as<uint32_t>(), nullptr);
        PT_LAUNCH_CHECK(ctx);
        simt_contract_kernel<<<grid, 256, 0, st>>>(ctx->labels.as<float>(), ctx->Xn32.as<float>(),
                                                   ctx->n_pad, ell, V, 1, 1, 0, nullptr,
                                                   ctx->rowflag.as<uint8_t>(), nullptr, nullptr,
                                                   Tex.as<float>());
        PT_LAUNCH_CHECK(ctx);
        u_to_t_kernel<<<grid_n(int64_t(ell) * V, 256), 256, 0, st>>>(
            Tex.as<float>(), int64_t(ell) * V, float(ctx->k), float(ctx->c_t));
        PT_LAUNCH_CHECK(ctx);
      }
    }
    if (s != PT_OK) return s;
    const int fin_blocks = grid_n((ell + kFinRowsPerBlock - 1) / kFinRowsPerBlock, 1);
    finalize_max_kernel<<<fin_blocks, 256, 0, st>>>(
        ctx->maxkey.as<unsigned long long>(), ell, ctx->valid_map.as<int32_t>(),
        ctx->Xraw.as<float>(), ctx->n, ctx->n1, ctx->n_pad, perms, 0, tmax.as<float>(),
        reinterpret_cast<int32_t*>(keys.p));
    PT_LAUNCH_CHECK(ctx);
    if (counts) {
      scatter_counts_kernel<<<grid_n(V, 256), 256, 0, st>>>(
          ctx->cnt.as<uint32_t>(), V, ctx->valid_map.as<int32_t>(), counts, 0);
      PT_LAUNCH_CHECK(ctx);
    }
    if (train_max)
      PT_CUDA_TRY(ctx, cudaMemcpyAsync(train_max, tmax.p, sizeof(float) * ell,
                                       cudaMemcpyDeviceToDevice, st));
  }

  // 2. U0 and its QR
  float* U = Ub.as<float>();
  u0_kernel<<<grid_n(V * pl.RP, 256), 256, 0, st>>>(U, V, pl.R, pl.RP, pl.k0, pl.k1);
  PT_LAUNCH_CHECK(ctx);
  s = qr_inplace(ctx, U, pl, part, rinv);
  if (s != PT_OK) return s;

  // 3. sequential subspace tracking over passes x columns, one launch per
  //    step: cluster 0 fits step t on U_{t-1} with step t-1's update applied
  //    to its sampled rows (geodesic_row, the same bits as the whole-U
  //    update), while the other clusters write U_t = update_{t-1}(U_{t-1})
  //    into the other buffer. lift and the coefficients alternate by step
  //    parity; a step clears the lift entries of the step two before it.
  size_t csm = 0;
  const int CL = choose_cluster(pl.m, pl.R, pl.RP, 0, kTrainMinCluster, &csm);
  if (CL == 0) {
    set_error(ctx, "RapidPT: the sampled rows do not fit a 16-CTA cluster");
    return PT_ERR_UNSUPPORTED;
  }
  int gu_chunk = 0;
  csm = std::max(csm, update_smem(pl.RP, &gu_chunk));
  float* ua = U;               // latest complete U (U_{t-1} while an update is pending)
  float* ub = Ub2.as<float>();
  float* liftb[2] = {lift.as<float>(), lift.as<float>() + V};
  float* updb[2] = {upd.as<float>(), upd.as<float>() + updw};
  PT_CUDA_TRY(ctx, cudaMemsetAsync(lift.p, 0, sizeof(float) * 2 * V, st));
  CluStepArgs sa;
  sa.gu_chunk = gu_chunk;
  sa.status = ctx->status.as<uint32_t>();
  sa.samp = nullptr;
  sa.tag = TAG_TRAIN;
  sa.V = uint32_t(V);
  sa.R = pl.R;
  sa.m = pl.m;
  sa.CL = CL;
  sa.k0 = pl.k0;
  sa.k1 = pl.k1;
  sa.rho = o.admm_rho;
  sa.iters = o.admm_iters;
  sa.step = o.step;
  int64_t steps = 0;
  int pend = -1;                          // parity of the step whose update is pending
  int last_pc[2][2] = {{-1, -1}, {-1, -1}};  // (pass, col) of the last step per parity
  int nclu = 0;                           // clusters of a launch that updates U (resident)
  cudaError_t lerr = cudaSuccess;
  with_rp(pl.RP, [&](auto rpc) {
    constexpr int RPc = decltype(rpc)::value;
    auto launch = [&](bool fit) {
      sa.fit = fit ? 1 : 0;
      if (pend >= 0) {
        sa.gu_src = ua;
        sa.gu_dst = ub;
        sa.gu_lift = liftb[pend];
        sa.gu_coef = updb[pend];
      } else {
        sa.gu_src = nullptr;
      }
      lerr = launch_cluster(train_step_cluster_kernel<RPc>, pend >= 0 ? nclu : 1, CL, csm, st,
                            sa);
      count_launch();
      if (pend >= 0) std::swap(ua, ub);
    };
    // the fused launch needs a second cluster for the update
    lerr = max_active_clusters(train_step_cluster_kernel<RPc>, CL, csm, &nclu);
    if (lerr == cudaSuccess && nclu < 2) lerr = cudaErrorInvalidConfiguration;
    for (int p = 0; p < o.train_passes && lerr == cudaSuccess && s == PT_OK; ++p) {
      for (int i = 0; i < ell; ++i) {
        const int cur = int(steps & 1);
        sa.U = ua;
        sa.pend_upd = pend >= 0 ? updb[pend] : nullptr;
        sa.pend_lift = pend >= 0 ? liftb[pend] : nullptr;
        sa.clear_pass = last_pc[cur][0];
        sa.clear_col = last_pc[cur][1];
        sa.lift = liftb[cur];
        sa.upd = updb[cur];
        sa.pass = p;
        sa.col = i;
        sa.Trow = Tex.as<float>() + int64_t(i) * V;
        sa.w_hist = w_hist ? w_hist + steps * pl.R : nullptr;
        launch(true);
        if (lerr != cudaSuccess) break;
        last_pc[cur][0] = p;
        last_pc[cur][1] = i;
        pend = cur;
        ++steps;
        if (steps % o.qr_every == 0) {  // QR needs the whole U of this step
          launch(false);
          if (lerr != cudaSuccess) break;
          pend = -1;
          s = qr_inplace(ctx, ua, pl, part, rinv);
          if (s != PT_OK) break;
        }
      }
    }
    if (lerr == cudaSuccess && s == PT_OK && pend >= 0) {
      launch(false);
      pend = -1;
    }
  });
  U = ua;
  if (lerr != cudaSuccess) {
    set_error(ctx, std::string("RapidPT training launch: ") + cudaGetErrorString(lerr));
    return PT_ERR_CUDA;
  }
  if (s != PT_OK) return s;
  s = qr_inplace(ctx, U, pl, part, rinv);
  if (s != PT_OK) return s;

  // 4. W_ex = U^T T_ex (rows of Wex = weights of training columns)
  {
    const int itiles = (ell + kWexTile - 1) / kWexTile;
    const int ctiles = (pl.RP + kWexTile - 1) / kWexTile;
    int nsplit = std::max(1, 152 * 3 / (itiles * ctiles));  // about three CTAs per SM
    nsplit = int(std::min<int64_t>(nsplit, (V + 1023) / 1024));
    const int64_t per = (V + nsplit - 1) / nsplit;
    if (!part.ensure(std::max(part.bytes, sizeof(float) * size_t(nsplit) * ell * pl.RP)))
      return nomem_r(ctx, "W_ex");
    const dim3 grid{unsigned(itiles), unsigned(nsplit), unsigned(ctiles)};
    wex_partial_kernel<<<grid, 256, 0, st>>>(U, Tex.as<float>(), V, ell, pl.RP, per,
                                            part.as<float>());
    PT_LAUNCH_CHECK(ctx);
    wex_reduce_kernel<<<grid_n(int64_t(ell) * pl.RP, 256), 256, 0, st>>>(
        part.as<float>(), nsplit, ell, pl.RP, Wex.as<float>());
    PT_LAUNCH_CHECK(ctx);
  }
  // 5. sigma over the sampled residuals of the last pass
  const int sblocks = 152 * 4;
  if (!sig.ensure(sizeof(double) * 2 * sblocks)) return nomem_r(ctx, "sigma");
  sigma_partial_kernel<<<sblocks, 256, 0, st>>>(U, Tex.as<float>(), Wex.as<float>(), uint32_t(V),
                                                ell, pl.m, pl.RP, pl.k0, pl.k1,
                                                o.train_passes - 1, sig.as<double>());
  PT_LAUNCH_CHECK(ctx);
  std::vector<double> hs(2 * sblocks);
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(hs.data(), sig.p, sizeof(double) * 2 * sblocks,
                                   cudaMemcpyDeviceToHost, st));
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  double s1 = 0.0, s2 = 0.0;
  for (int b = 0; b < sblocks; ++b) {
    s1 += hs[2 * b];
    s2 += hs[2 * b + 1];
  }
  const double cnt = double(ell) * pl.m;
  const double mean = s1 / cnt;
  const double sigma = std::sqrt(std::max(0.0, s2 / cnt - mean * mean));
  // 6. shift mu
  double mu = 0.0;
  {
    s = reconstruct(ctx, Wex.as<float>(), ell, 0, U, pl, float(sigma),
                    o.shift_mode == 0 ? 0u : TAG_SHIFT, o.shift_mode == 0 ? 1 : 0,
                    Tex.as<float>(), keys.as<unsigned long long>());
    if (s != PT_OK) return s;
    std::vector<unsigned long long> hk(ell);
    std::vector<float> ht(ell);
    PT_CUDA_TRY(ctx, cudaMemcpyAsync(hk.data(), keys.p, sizeof(unsigned long long) * ell,
                                     cudaMemcpyDeviceToHost, st));
    PT_CUDA_TRY(ctx, cudaMemcpyAsync(ht.data(), tmax.p, sizeof(float) * ell,
                                     cudaMemcpyDeviceToHost, st));
    PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
    auto val = [](unsigned long long k) {
      const uint32_t o32 = uint32_t(k >> 32);
      const uint32_t u = (o32 & 0x80000000u) ? (o32 & 0x7fffffffu) : ~o32;
      float f;
      memcpy(&f, &u, 4);
      return double(f);
    };
    if (o.shift_mode == 0) {
      mu = -INFINITY;
      for (int i = 0; i < ell; ++i) mu = std::max(mu, val(hk[i]));
    } else {
      for (int i = 0; i < ell; ++i) mu += double(ht[i]) - val(hk[i]);
      mu /= ell;
    }
  }
  if (U_out) {
    pack_u_kernel<<<grid_n(V * pl.RP, 256), 256, 0, st>>>(U, V, pl.R, pl.RP, U_out, 0);
    PT_LAUNCH_CHECK(ctx);
  }
  if (info) {
    info->sigma = sigma;
    info->mu = mu;
    info->m_per_perm = pl.m;
    info->train_steps = steps;
  }
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return PT_OK;
}

// ---------------------------------------------------------------------------
// Recovery
// ---------------------------------------------------------------------------
// Recovery with U updates (pt_rapid_opts.rec_step > 0): the relabellings in
// row order, each one a training-type step on its own samples (the step kernel
// with the recovery draws and the sampled t values of Tt) followed by the
// reconstruction of that relabelling with the U it was fitted to, which the
// step launch has just materialised in full. QR every qr_every steps.
pt_status recover_with_updates(pt_ctx* ctx, const RapidPlan& pl, const pt_rapid_opts& o,
                               int64_t first_row, int64_t rows, float* U, const float* Tt,
                               float sigma, float* Wrows, unsigned long long* keys) {
  cudaStream_t st = ctx->stream;
  const int64_t V = pl.V;
  Buf Ub2, lift, upd, part, rinv;
  struct G {
    std::vector<Buf*> v;
    ~G() {
      for (Buf* b : v) b->release();
    }
  } guard{{&Ub2, &lift, &upd, &part, &rinv}};
  const int updw = 3 * pl.RP + 4;
  if (!Ub2.ensure(sizeof(float) * size_t(V) * pl.RP) || !lift.ensure(sizeof(float) * 2 * V) ||
      !upd.ensure(sizeof(float) * 2 * updw))
    return nomem_r(ctx, "RapidPT recovery updates");
  size_t csm = 0;
  const int CL = choose_cluster(pl.m, pl.R, pl.RP, 0, kTrainMinCluster, &csm);
  if (CL == 0) {
    set_error(ctx, "RapidPT: the sampled rows do not fit a 16-CTA cluster");
    return PT_ERR_UNSUPPORTED;
  }
  int gu_chunk = 0;
  csm = std::max(csm, update_smem(pl.RP, &gu_chunk));
  PT_CUDA_TRY(ctx, cudaMemsetAsync(lift.p, 0, sizeof(float) * 2 * V, st));
  PT_CUDA_TRY(ctx, cudaMemsetAsync(Wrows, 0, sizeof(float) * size_t(rows) * pl.RP, st));
  PT_CUDA_TRY(ctx, cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * rows, st));
  float* ua = U;
  float* ub = Ub2.as<float>();
  float* liftb[2] = {lift.as<float>(), lift.as<float>() + V};
  float* updb[2] = {upd.as<float>(), upd.as<float>() + updw};
  CluStepArgs sa;
  sa.gu_chunk = gu_chunk;
  sa.status = ctx->status.as<uint32_t>();
  sa.Trow = nullptr;
  sa.tag = TAG_REC;
  sa.V = uint32_t(V);
  sa.R = pl.R;
  sa.m = pl.m;
  sa.CL = CL;
  sa.k0 = pl.k0;
  sa.k1 = pl.k1;
  sa.rho = o.admm_rho;
  sa.iters = o.admm_iters;
  sa.step = o.rec_step;
  sa.pass = 0;
  int pend = -1;
  int64_t last_row[2] = {-1, -1};
  int nclu = 0;
  int64_t steps = 0;
  pt_status s = PT_OK;
  cudaError_t lerr = cudaSuccess;
  with_rp(pl.RP, [&](auto rpc) {
    constexpr int RPc = decltype(rpc)::value;
    auto launch = [&](bool fit) {
      sa.fit = fit ? 1 : 0;
      if (pend >= 0) {
        sa.gu_src = ua;
        sa.gu_dst = ub;
        sa.gu_lift = liftb[pend];
        sa.gu_coef = updb[pend];
      } else {
        sa.gu_src = nullptr;
      }
      lerr = launch_cluster(train_step_cluster_kernel<RPc>, pend >= 0 ? nclu : 1, CL, csm, st,
                            sa);
      count_launch();
      if (pend >= 0) std::swap(ua, ub);
    };
    lerr = max_active_clusters(train_step_cluster_kernel<RPc>, CL, csm, &nclu);
    if (lerr == cudaSuccess && nclu < 2) lerr = cudaErrorInvalidConfiguration;
    for (int64_t k = 0; k < rows && lerr == cudaSuccess && s == PT_OK; ++k) {
      const int64_t i = first_row + k;
      const int cur = int(steps & 1);
      sa.U = ua;
      sa.pend_upd = pend >= 0 ? updb[pend] : nullptr;
      sa.pend_lift = pend >= 0 ? liftb[pend] : nullptr;
      sa.clear_pass = last_row[cur] >= 0 ? 0 : -1;
      sa.clear_col = int(last_row[cur]);
      sa.lift = liftb[cur];
      sa.upd = updb[cur];
      sa.col = int(i);
      sa.samp = Tt + k * pl.m;
      sa.w_hist = Wrows + k * pl.RP;
      launch(true);
      if (lerr != cudaSuccess) break;
      // ua is now the U this relabelling was fitted to, in full
      s = recon_tc(ctx, Wrows + k * pl.RP, 1, i, ua, V, pl.RP, sigma, TAG_NOISE, pl.k0, pl.k1,
                   keys + k);
      if (s != PT_OK) break;
      last_row[cur] = i;
      pend = cur;
      ++steps;
      if (steps % o.qr_every == 0) {
        launch(false);
        if (lerr != cudaSuccess) break;
        pend = -1;
        s = qr_inplace(ctx, ua, pl, part, rinv);
      }
    }
  });
  if (lerr != cudaSuccess) {
    set_error(ctx, std::string("RapidPT recovery update launch: ") + cudaGetErrorString(lerr));
    return PT_ERR_CUDA;
  }
  return s;
}

pt_status rapid_recover_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, int64_t first_row,
                             const float* U_in, int32_t rank, double sample_rate, double sigma,
                             double mu, const pt_rapid_opts& o, float* maxnull, float* W_out) {
  RapidPlan pl;
  pt_status s = check_rapid_args(ctx, rank, sample_rate, o, pl);
  if (s != PT_OK) return s;
  if (first_row < 0 || first_row >= P) {
    set_error(ctx, "RapidPT: need 0 <= first_row < P");
    return PT_ERR_INVALID;
  }
  cudaStream_t st = ctx->stream;
  const int64_t rows = P - first_row;
  s = ensure_xn32(ctx);
  if (s != PT_OK) return s;
  Buf Ub, Wb, keys, Tt;
  struct G {
    std::vector<Buf*> v;
    ~G() {
      for (Buf* b : v) b->release();
    }
  } guard{{&Ub, &Wb, &keys, &Tt}};
  size_t csm = 0;
  const int CL = choose_cluster(pl.m, pl.R, pl.RP, 0, 2, &csm);
  if (CL == 0) {
    set_error(ctx, "RapidPT: the sampled rows do not fit a 16-CTA cluster");
    return PT_ERR_UNSUPPORTED;
  }
  if (!Ub.ensure(sizeof(float) * size_t(pl.V) * pl.RP) ||
      !Wb.ensure(sizeof(float) * size_t(rows) * pl.RP) ||
      !keys.ensure(sizeof(unsigned long long) * rows) ||
      !Tt.ensure(sizeof(float) * size_t(rows) * size_t(pl.m)))
    return nomem_r(ctx, "RapidPT recovery");
  validate_perms_kernel<<<grid_n((rows + 7) / 8, 1), 256, 0, st>>>(perms, first_row, P, ctx->n,
                                                                   ctx->status.as<uint32_t>());
  PT_LAUNCH_CHECK(ctx);
  pack_u_kernel<<<grid_n(pl.V * pl.RP, 256), 256, 0, st>>>(U_in, pl.V, pl.R, pl.RP,
                                                          Ub.as<float>(), 1);
  PT_LAUNCH_CHECK(ctx);
  // t at every recovery relabelling's sampled voxels, all at once
  {
    const int T = ctx->n_pad <= 128 ? 1 : ctx->n_pad <= 256 ? 2 : ctx->n_pad <= 512 ? 4 : 8;
    const dim3 grid{unsigned(rows), unsigned((pl.m + 63) / 64), 1u};
    const float kf = float(ctx->k), ctf = float(ctx->c_t);
#define PT_SAMPLED_T(TT)                                                                    \
  sampled_t_kernel<TT><<<grid, 256, 0, st>>>(perms, ctx->n, ctx->n1, ctx->n_pad,            \
                                             ctx->Xn32.as<float>(), uint32_t(pl.V), pl.m,   \
                                             pl.k0, pl.k1, kf, ctf, first_row, Tt.as<float>())
    if (T == 1) PT_SAMPLED_T(1);
    else if (T == 2) PT_SAMPLED_T(2);
    else if (T == 4) PT_SAMPLED_T(4);
    else PT_SAMPLED_T(8);
#undef PT_SAMPLED_T
    PT_LAUNCH_CHECK(ctx);
  }
  if (o.rec_step > 0.0f) {
    s = recover_with_updates(ctx, pl, o, first_row, rows, Ub.as<float>(), Tt.as<float>(),
                             float(sigma), Wb.as<float>(), keys.as<unsigned long long>());
    if (s != PT_OK) return s;
  } else {
  CluRecArgs a;
  a.Tt = Tt.as<float>();
  a.V = uint32_t(pl.V);
  a.R = pl.R;
  a.m = pl.m;
  a.CL = CL;
  a.U = Ub.as<float>();
  a.k0 = pl.k0;
  a.k1 = pl.k1;
  a.rho = o.admm_rho;
  a.iters = o.admm_iters;
  a.row_first = first_row;
  a.row_end = P;
  a.W = Wb.as<float>();
  a.status = ctx->status.as<uint32_t>();
  cudaError_t lerr = cudaSuccess;
  with_rp(pl.RP, [&](auto rpc) {
    constexpr int RPc = decltype(rpc)::value;
    const int want = int(std::min<int64_t>(rows, 152));
    lerr = launch_cluster(recover_fit_cluster_kernel<RPc>, -want, CL, csm, st, a);
  });
  if (lerr != cudaSuccess) {
    set_error(ctx, std::string("RapidPT recovery launch: ") + cudaGetErrorString(lerr));
    return PT_ERR_CUDA;
  }
  count_launch();
  s = reconstruct(ctx, Wb.as<float>(), rows, first_row, Ub.as<float>(), pl, float(sigma),
                  TAG_NOISE, 0, nullptr, keys.as<unsigned long long>());
  if (s != PT_OK) return s;
  }
  keys_to_values_kernel<<<grid_n(rows, 256), 256, 0, st>>>(keys.as<unsigned long long>(), rows,
                                                          float(mu), maxnull);
  PT_LAUNCH_CHECK(ctx);
  if (W_out) {
    pack_u_kernel<<<grid_n(rows * pl.RP, 256), 256, 0, st>>>(Wb.as<float>(), rows, pl.R, pl.RP,
                                                            W_out, 0);
    PT_LAUNCH_CHECK(ctx);
  }
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(st));
  return PT_OK;
}

// Rows of T (Sec. 2.1): t of every mask voxel under each of P relabellings,
// from the contraction RapidPT uses for its training rows T_ex: the tensor-core
// kernel writing t from its accumulator (BF16 pieces), or the FP32 CUDA-core
// kernel writing u followed by the same u -> t map.
pt_status t_rows_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, int precision, float* T) {
  if (ctx->glm_q1) {
    set_error(ctx, "pt_t_rows: rows of the plain two-sample t only (context has covariates)");
    return PT_ERR_UNSUPPORTED;
  }
  cudaStream_t st = ctx->stream;
  const int64_t V = ctx->v_valid, v = ctx->v;
  PT_CUDA_TRY(ctx, cudaMemsetAsync(T, 0xFF, sizeof(float) * size_t(P) * v, st));  // NaN
  if (V == 0) return PT_OK;
  Buf comp;
  struct G {
    Buf* b;
    ~G() { b->release(); }
  } guard{&comp};
  float* out = T;
  if (V != v) {
    if (!comp.ensure(sizeof(float) * size_t(P) * V)) {
      set_error(ctx, "pt_t_rows: out of device memory");
      return PT_ERR_NOMEM;
    }
    out = comp.as<float>();
  }
  if (!ctx->cnt.ensure(sizeof(uint32_t) * (V + 1))) {  // the labels kernel counts observed-set rows
    set_error(ctx, "pt_t_rows: out of device memory");
    return PT_ERR_NOMEM;
  }
  int64_t P_pad = 0;
  pt_status s;
  if (precision != PT_PREC_FP32) {
    s = tc_supported(ctx);
    if (s == PT_OK) s = ensure_xnb(ctx, precision);
    if (s == PT_OK) s = build_labels(ctx, perms, P, prec_label_layout(precision), &P_pad);
    if (s == PT_OK)
      s = tc_rows(ctx, ctx->labels.p, P, precision, 2, out, 0, 0, nullptr, nullptr, nullptr);
  } else {
    s = ensure_xn32(ctx);
    if (s == PT_OK) s = build_labels(ctx, perms, P, 0, &P_pad);
    if (s == PT_OK) {
      const dim3 grid{unsigned((V + 127) / 128), unsigned((P + 127) / 128), 1u};
      simt_contract_kernel<<<grid, 256, 0, st>>>(ctx->labels.as<float>(), ctx->Xn32.as<float>(),
                                                 ctx->n_pad, P, V, 1, 1, 0, nullptr,
                                                 ctx->rowflag.as<uint8_t>(), nullptr, nullptr, out);
      PT_LAUNCH_CHECK(ctx);
      u_to_t_kernel<<<grid_n(P * V, 256), 256, 0, st>>>(out, P * V, float(ctx->k),
                                                         float(ctx->c_t));
      PT_LAUNCH_CHECK(ctx);
    }
  }
  if (s != PT_OK) return s;
  if (V != v) {
    scatter_rows_kernel<<<grid_n(P * V, 256), 256, 0, st>>>(out, P, V, ctx->valid_map.as<int32_t>(),
                                                            v, T);
    PT_LAUNCH_CHECK(ctx);
  }
  return PT_OK;
}

}  // namespace pt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void pt_rapid_opts_default(pt_rapid_opts* o) {
  if (!o) return;
  o->precision = PT_PREC_BF16X3;
  o->train_passes = 1;
  o->qr_every = 100;
  o->admm_iters = 30;
  o->admm_rho = 2.0f;
  o->step = 1.0f;
  o->shift_mode = 1;
  o->seed = 1;
  o->rec_step = 0.0f;
}

pt_status pt_t_rows(pt_ctx* ctx, const int32_t* perms, int64_t P, int32_t precision, float* T) {
  pt::NvtxRange nvtx_range("pt_t_rows");
  if (!ctx || !perms || !T) {
    pt::set_error(ctx, "pt_t_rows: NULL argument");
    return PT_ERR_INVALID;
  }
  if (P < 1 || P > INT32_MAX || precision < PT_PREC_FP32 || precision > PT_PREC_FP16X2) {
    pt::set_error(ctx, "pt_t_rows: need 1 <= P <= 2^31-1 and a valid precision");
    return PT_ERR_INVALID;
  }
  try {
    cudaSetDevice(ctx->device);
    return pt::t_rows_impl(ctx, perms, P, precision, T);
  } catch (...) {
    pt::set_error(ctx, "pt_t_rows: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_rapid_train(pt_ctx* ctx, const int32_t* perms, int32_t n_train, int32_t rank,
                         double sample_rate, const pt_rapid_opts* opts, float* U_out,
                         float* train_max, uint32_t* counts, float* w_hist,
                         pt_rapid_info* info) {
  pt::NvtxRange nvtx_range("pt_rapid_train");
  if (!ctx || !perms) {
    pt::set_error(ctx, "pt_rapid_train: NULL argument");
    return PT_ERR_INVALID;
  }
  try {
    pt_rapid_opts o;
    pt_rapid_opts_default(&o);
    if (opts) o = *opts;
    cudaSetDevice(ctx->device);
    return pt::rapid_train_impl(ctx, perms, n_train, rank, sample_rate, o, U_out, train_max,
                                counts, w_hist, info);
  } catch (...) {
    pt::set_error(ctx, "pt_rapid_train: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_rapid_recover(pt_ctx* ctx, const int32_t* perms, int64_t P, int64_t first_row,
                           const float* U, int32_t rank, double sample_rate, double sigma,
                           double mu, const pt_rapid_opts* opts, float* maxnull, float* W_out) {
  pt::NvtxRange nvtx_range("pt_rapid_recover");
  if (!ctx || !perms || !U || !maxnull) {
    pt::set_error(ctx, "pt_rapid_recover: NULL argument");
    return PT_ERR_INVALID;
  }
  try {
    pt_rapid_opts o;
    pt_rapid_opts_default(&o);
    if (opts) o = *opts;
    cudaSetDevice(ctx->device);
    return pt::rapid_recover_impl(ctx, perms, P, first_row, U, rank, sample_rate, sigma, mu, o,
                                  maxnull, W_out);
  } catch (...) {
    pt::set_error(ctx, "pt_rapid_recover: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_maxnull_rapid(pt_ctx* ctx, const int32_t* perms, int64_t P, int32_t rank,
                           double sample_rate, int32_t n_train, const pt_rapid_opts* opts,
                           float* maxnull, uint32_t* counts, pt_rapid_info* info) {
  pt::NvtxRange nvtx_range("pt_maxnull_rapid");
  if (!ctx || !perms || !maxnull) {
    pt::set_error(ctx, "pt_maxnull_rapid: NULL argument");
    return PT_ERR_INVALID;
  }
  if (n_train < 1 || n_train >= P) {
    pt::set_error(ctx, "pt_maxnull_rapid: need 1 <= n_train < P");
    return PT_ERR_INVALID;
  }
  try {
    pt_rapid_opts o;
    pt_rapid_opts_default(&o);
    if (opts) o = *opts;
    cudaSetDevice(ctx->device);
    pt::Buf U;
    if (!U.ensure(sizeof(float) * size_t(ctx->v_valid > 0 ? ctx->v_valid : 1) * rank)) {
      pt::set_error(ctx, "out of device memory (U)");
      return PT_ERR_NOMEM;
    }
    pt_rapid_info inf{};
    pt_status s = pt::rapid_train_impl(ctx, perms, n_train, rank, sample_rate, o, U.as<float>(),
                                       maxnull, counts, nullptr, &inf);
    if (s == PT_OK)
      s = pt::rapid_recover_impl(ctx, perms, P, n_train, U.as<float>(), rank, sample_rate,
                                 inf.sigma, inf.mu, o, maxnull + n_train, nullptr);
    U.release();
    if (info) *info = inf;
    return s;
  } catch (...) {
    pt::set_error(ctx, "pt_maxnull_rapid: internal error");
    return PT_ERR_CUDA;
  }
}

}  // extern "C"
