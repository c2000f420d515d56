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
// Random numbers: Philox4x32-10 (Salmon et al., SC 2011) keyed by the seed,
// counters (a, b, c, tag): normals by Box-Muller from the first two words,
// voxel indices as floor((x1 2^32 + x0) v / 2^64).
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {

// Kernels of the NaivePT path reused here (pt_naive.cu).
__global__ void finalize_max_kernel(const unsigned long long* maxkey, int64_t P,
                                    const int32_t* valid_map, const float* Xraw, int n, int n1,
                                    int n_pad, const int32_t* perms, int two_sided,
                                    float* maxnull, int32_t* argmax);
__global__ void scatter_counts_kernel(const uint32_t* cnt, int64_t v_valid,
                                      const int32_t* valid_map, uint32_t* counts);
__global__ void simt_contract_kernel(const float* L, const float* Xn, int n_pad, int64_t P,
                                     int64_t v, int tiles_per_cta, int mode, int two_sided,
                                     const float* u_obs, const uint8_t* rowflag,
                                     unsigned long long* maxkey, uint32_t* cnt, float* uout);

namespace {

constexpr uint32_t TAG_U0 = 1, TAG_TRAIN = 2, TAG_REC = 3, TAG_NOISE = 4, TAG_SHIFT = 5;
constexpr int kFitThreads = 1024;
constexpr int kMaxRank = 128;
constexpr float kNoiseBound = 6.6604f;  // sqrt(-2 ln 2^-32) rounded up: |z| of every draw

// ---------------------------------------------------------------------------
// Philox4x32-10 and the draws built on it
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = c.x * 0xD2511F53u, hi0 = __umulhi(c.x, 0xD2511F53u);
    const uint32_t lo1 = c.z * 0xCD9E8D57u, hi1 = __umulhi(c.z, 0xCD9E8D57u);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ float draw_normal(uint32_t k0, uint32_t k1, uint32_t tag, uint32_t a,
                                             uint32_t b) {
  const uint4 o = philox(make_uint4(a, b, 0u, tag), k0, k1);
  const float u1 = fmaf(__uint2float_rn(o.x), 2.3283064365386963e-10f, 2.3283064365386963e-10f);
  const float u2 = __uint2float_rn(o.y) * 2.3283064365386963e-10f;
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

__device__ __forceinline__ uint32_t draw_index(uint32_t k0, uint32_t k1, uint32_t tag, uint32_t q,
                                               uint32_t i, uint32_t p, uint32_t V) {
  const uint4 o = philox(make_uint4(q, i, p, tag), k0, k1);
  const unsigned long long t =
      (unsigned long long)o.y * V + (((unsigned long long)o.x * V) >> 32);
  return uint32_t(t >> 32);
}

// ---------------------------------------------------------------------------
// Block-level l1 weight solve (1024 threads). A: m x RP (row-major, padded
// columns zero), b: m. s, y: m scratch. Shared: G, Gi (RP x RP), red (32 x RP),
// stage (32 x RP), wv, rhs (RP). Leaves w in wv.
// ---------------------------------------------------------------------------
// Rows of A staged per Gram step: kStageFloats / RP.
constexpr int kStageFloats = 8192;

struct FitSmem {
  float* G;
  float* Gi;
  float* red;
  float* stage;
  float* wv;
  float* rhs;
  float* scal;  // 8 scalars
};

__device__ void carve_fit_smem(float* base, int RP, FitSmem& f) {
  f.G = base;
  f.Gi = f.G + RP * RP;
  f.red = f.Gi + RP * RP;
  f.stage = f.red + 32 * RP;
  f.wv = f.stage + kStageFloats;
  f.rhs = f.wv + RP;
  f.scal = f.rhs + RP;
}

// The fit's m-length vectors (b, s, y, x) live in shared memory up to this m.
constexpr int kSmemVecM = 4096;

// out[c] = sum_q A[q][c] * x[q] for c < R (warps split q, lanes split c; four
// rows in flight per warp so the loads from L2 overlap).
template <int RP>
__device__ void block_AtX(const float* __restrict__ A, int m, int R, const float* __restrict__ x,
                          float* red, float* out) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  constexpr int KC = kMaxRank / 32;
  float acc[KC];
#pragma unroll
  for (int k = 0; k < KC; ++k) acc[k] = 0.0f;
  int q = w;
  for (; q + 96 < m; q += 128) {
    float xv[4], av[4][KC];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      xv[u] = x[q + 32 * u];
      const float* row = A + int64_t(q + 32 * u) * RP;
#pragma unroll
      for (int k = 0; k < KC; ++k) {
        const int c = lane + 32 * k;
        av[u][k] = c < RP ? row[c] : 0.0f;
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int k = 0; k < KC; ++k) acc[k] = fmaf(av[u][k], xv[u], acc[k]);
  }
  for (; q < m; q += 32) {
    const float xq = x[q];
    const float* row = A + int64_t(q) * RP;
#pragma unroll
    for (int k = 0; k < KC; ++k) {
      const int c = lane + 32 * k;
      if (c < RP) acc[k] = fmaf(row[c], xq, acc[k]);
    }
  }
#pragma unroll
  for (int k = 0; k < KC; ++k) {
    const int c = lane + 32 * k;
    if (c < RP) red[w * RP + c] = acc[k];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < R; c += blockDim.x) {
    float t = 0.0f;
    for (int ww = 0; ww < 32; ++ww) t += red[ww * RP + c];
    out[c] = t;
  }
  __syncthreads();
}

template <int RP>
__device__ __forceinline__ float row_dot(const float* __restrict__ row,
                                         const float* __restrict__ v) {
  float4 a[RP / 4];
  const float4* r4 = reinterpret_cast<const float4*>(row);
#pragma unroll
  for (int c4 = 0; c4 < RP / 4; ++c4) a[c4] = r4[c4];  // all loads in flight together
  float t0 = 0.0f, t1 = 0.0f;
#pragma unroll
  for (int c4 = 0; c4 < RP / 4; ++c4) {
    t0 = fmaf(a[c4].x, v[4 * c4], t0);
    t1 = fmaf(a[c4].y, v[4 * c4 + 1], t1);
    t0 = fmaf(a[c4].z, v[4 * c4 + 2], t0);
    t1 = fmaf(a[c4].w, v[4 * c4 + 3], t1);
  }
  return t0 + t1;
}

__device__ __forceinline__ float row_dot_rt(const float* __restrict__ row,
                                            const float* __restrict__ v, int RP) {
  float t = 0.0f;
  for (int c = 0; c < RP; ++c) t = fmaf(row[c], v[c], t);
  return t;
}

// b, s, y, x: m floats each (shared memory when they fit, else global scratch).
template <int RP>
__device__ void block_l1_fit(const float* __restrict__ A, const float* b, float* s, float* y,
                             float* x, int m, int R, float rho, int iters, FitSmem& f) {
  constexpr int CH = kStageFloats / RP;  // rows staged per Gram step
  const int tid = threadIdx.x;
  const int npairs = R * (R + 1) / 2;
  // --- Gram G = A^T A (upper triangle by pairs, then mirrored) ---
  float acc[9];
  int pc[9], pd[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    acc[k] = 0.0f;
    const int pi = tid + k * blockDim.x;
    int c = 0, rem = pi < npairs ? pi : 0;
    while (rem >= R - c) {
      rem -= R - c;
      ++c;
    }
    pc[k] = c;
    pd[k] = c + rem;
  }
  for (int q0 = 0; q0 < m; q0 += CH) {
    const int rows = min(CH, m - q0);
    const float4* src = reinterpret_cast<const float4*>(A + int64_t(q0) * RP);
    float4* dst = reinterpret_cast<float4*>(f.stage);
    for (int e = tid; e < CH * RP / 4; e += blockDim.x)
      dst[e] = (e < rows * RP / 4) ? src[e] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (tid + k * blockDim.x < npairs) {
        const int c = pc[k], d = pd[k];
        float t0 = acc[k], t1 = 0.0f;
#pragma unroll 8
        for (int rr = 0; rr < CH; rr += 2) {
          t0 = fmaf(f.stage[rr * RP + c], f.stage[rr * RP + d], t0);
          t1 = fmaf(f.stage[(rr + 1) * RP + c], f.stage[(rr + 1) * RP + d], t1);
        }
        acc[k] = t0 + t1;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < RP * RP; e += blockDim.x) {
    f.G[e] = 0.0f;
    f.Gi[e] = (e / RP == e % RP) ? 1.0f : 0.0f;
  }
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (tid + k * blockDim.x < npairs) {
      f.G[pc[k] * RP + pd[k]] = acc[k];
      f.G[pd[k] * RP + pc[k]] = acc[k];
    }
  }
  __syncthreads();
  // --- G^-1 by Gauss-Jordan on [G | I] (G symmetric positive definite: no pivoting) ---
  float* fac = f.red;  // R factors of the current column
  for (int k = 0; k < R; ++k) {
    const float inv = 1.0f / f.G[k * RP + k];
    __syncthreads();
    for (int j = tid; j < 2 * R; j += blockDim.x) {
      if (j < R) f.G[k * RP + j] *= inv;
      else f.Gi[k * RP + (j - R)] *= inv;
    }
    for (int i = tid; i < R; i += blockDim.x) fac[i] = (i == k) ? 0.0f : f.G[i * RP + k];
    __syncthreads();
    for (int e = tid; e < R * 2 * R; e += blockDim.x) {
      const int i = e / (2 * R), j = e - i * 2 * R;
      const float fi = fac[i];
      if (fi != 0.0f) {
        if (j < R) f.G[i * RP + j] -= fi * f.G[k * RP + j];
        else f.Gi[i * RP + (j - R)] -= fi * f.Gi[k * RP + (j - R)];
      }
    }
    __syncthreads();
  }
  // --- ADMM ---
  for (int q = tid; q < m; q += blockDim.x) {
    s[q] = 0.0f;
    y[q] = 0.0f;
  }
  for (int c = tid; c < RP; c += blockDim.x) f.wv[c] = 0.0f;
  __syncthreads();
  const float irho = 1.0f / rho;
  for (int it = 0; it < iters; ++it) {
    for (int q = tid; q < m; q += blockDim.x) x[q] = b[q] - s[q] - y[q] * irho;
    __syncthreads();
    block_AtX<RP>(A, m, R, x, f.red, f.rhs);
    for (int c = tid; c < R; c += blockDim.x) {
      float t = 0.0f;
      for (int d = 0; d < R; ++d) t = fmaf(f.Gi[c * RP + d], f.rhs[d], t);
      f.wv[c] = t;
    }
    __syncthreads();
    for (int q = tid; q < m; q += blockDim.x) {
      const float aw = row_dot<RP>(A + int64_t(q) * RP, f.wv);
      const float e = b[q] - aw - y[q] * irho;
      const float sq = copysignf(fmaxf(fabsf(e) - irho, 0.0f), e);
      s[q] = sq;
      y[q] = y[q] + rho * (aw + sq - b[q]);
    }
    __syncthreads();
  }
}

__device__ float block_sum(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  float t = 0.0f;
  if (threadIdx.x < 32) {
    t = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if (threadIdx.x == 0) red[0] = t;
  }
  __syncthreads();
  t = red[0];
  __syncthreads();
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

// Partial Gram U^T U in FP64 over a contiguous row range per block: upper
// triangle pairs, products of FP32 values accumulated in FP64.
__global__ void __launch_bounds__(1024) gram64_kernel(const float* __restrict__ U, int64_t V,
                                                      int R, int RP,
                                                      double* __restrict__ partials) {
  extern __shared__ float sm[];
  float* stage = sm;  // 32 x RP
  const int npairs = R * (R + 1) / 2;
  const int64_t per = (V + gridDim.x - 1) / gridDim.x;
  const int64_t j0 = blockIdx.x * per, j1 = min(V, j0 + per);
  double acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0;
  int pc[9], pd[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int pi = threadIdx.x + k * blockDim.x;
    int c = 0, rem = pi < npairs ? pi : 0;
    while (rem >= R - c) {
      rem -= R - c;
      ++c;
    }
    pc[k] = c;
    pd[k] = c + rem;
  }
  for (int64_t q0 = j0; q0 < j1; q0 += 32) {
    const int rows = int(j1 - q0 < 32 ? j1 - q0 : 32);
    for (int e = threadIdx.x; e < 32 * RP; e += blockDim.x) {
      const int rr = e / RP;
      stage[e] = rr < rows ? U[(q0 + rr) * RP + (e - rr * RP)] : 0.0f;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      if (threadIdx.x + k * blockDim.x < npairs) {
        double t = acc[k];
        for (int rr = 0; rr < rows; ++rr)
          t = fma(double(stage[rr * RP + pc[k]]), double(stage[rr * RP + pd[k]]), t);
        acc[k] = t;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int pi = threadIdx.x + k * blockDim.x;
    if (pi < npairs) partials[int64_t(blockIdx.x) * npairs + pi] = acc[k];
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
// Training step (one block) and geodesic update (whole grid)
// ---------------------------------------------------------------------------
struct StepArgs {
  const float* U;
  const float* Trow;  // T_ex row of this column (v values)
  uint32_t V;
  int R, RP, m;
  uint32_t k0, k1;
  int pass, col;
  float rho;
  int iters;
  float step;
  int32_t* idx;
  float* b;
  float* A;
  float* s;
  float* y;
  float* x;         // b, s, y, x: global fallback when m > kSmemVecM
  float* lift;      // v, zero on entry
  float* upd;       // [3 * RP + 4]: w, w/||w||, g2, alpha, beta
  float* w_hist;    // nullable: this step's weights (RP)
};

template <int RP>
__global__ void __launch_bounds__(kFitThreads) train_step_kernel(StepArgs a) {
  extern __shared__ float sm[];
  FitSmem f;
  carve_fit_smem(sm, RP, f);
  const int tid = threadIdx.x;
  float *b = a.b, *sv = a.s, *yv = a.y, *xv = a.x;
  if (a.m <= kSmemVecM) {
    b = f.scal + 8;
    sv = b + a.m;
    yv = sv + a.m;
    xv = yv + a.m;
  }
  for (int q = tid; q < a.m; q += blockDim.x) {
    const uint32_t j = draw_index(a.k0, a.k1, TAG_TRAIN, uint32_t(q), uint32_t(a.col),
                                  uint32_t(a.pass), a.V);
    a.idx[q] = int32_t(j);
    b[q] = a.Trow[j];
    const float4* src = reinterpret_cast<const float4*>(a.U + int64_t(j) * RP);
    float4* dst = reinterpret_cast<float4*>(a.A + int64_t(q) * RP);
    for (int c4 = 0; c4 < RP / 4; ++c4) dst[c4] = src[c4];
  }
  __syncthreads();
  block_l1_fit<RP>(a.A, b, sv, yv, xv, a.m, a.R, a.rho, a.iters, f);
  // residual r (into x), lift, ||r||^2
  float rr = 0.0f;
  for (int q = tid; q < a.m; q += blockDim.x) {
    const float r = b[q] - row_dot<RP>(a.A + int64_t(q) * RP, f.wv);
    xv[q] = r;
    atomicAdd(&a.lift[a.idx[q]], r);
    rr = fmaf(r, r, rr);
  }
  __syncthreads();
  const float nr2 = block_sum(rr, f.red);
  float* g2 = f.rhs;
  block_AtX<RP>(a.A, a.m, a.R, xv, f.red, g2);
  // ||lift||^2 = sum_q lift[idx_q] r_q (duplicates counted once per voxel)
  float ll = 0.0f;
  for (int q = tid; q < a.m; q += blockDim.x) ll = fmaf(a.lift[a.idx[q]], xv[q], ll);
  __syncthreads();
  const float nl2 = block_sum(ll, f.red);
  if (tid == 0) {
    float nw2 = 0.0f, ng2 = 0.0f;
    for (int c = 0; c < a.R; ++c) {
      nw2 = fmaf(f.wv[c], f.wv[c], nw2);
      ng2 = fmaf(g2[c], g2[c], ng2);
    }
    const float nw = sqrtf(nw2);
    const float nG = sqrtf(fmaxf(nl2 - ng2, 0.0f));
    float alpha = 0.0f, beta = 0.0f;
    if (nw > 0.0f && nG > 0.0f) {
      const float theta = a.step * atanf(sqrtf(nr2) / nw);
      alpha = (cosf(theta) - 1.0f) / nw;
      beta = sinf(theta) / nG;
    }
    f.scal[0] = alpha;
    f.scal[1] = beta;
    f.scal[2] = nw;
  }
  __syncthreads();
  const float nw = f.scal[2];
  for (int c = tid; c < RP; c += blockDim.x) {
    const float wc = c < a.R ? f.wv[c] : 0.0f;
    a.upd[c] = wc;
    a.upd[RP + c] = nw > 0.0f ? wc / nw : 0.0f;
    a.upd[2 * RP + c] = c < a.R ? g2[c] : 0.0f;
    if (a.w_hist && c < a.R) a.w_hist[c] = wc;
  }
  if (tid == 0) {
    a.upd[3 * RP] = f.scal[0];
    a.upd[3 * RP + 1] = f.scal[1];
  }
}

// U_j += (alpha (U_j . w) + beta (lift_j - U_j . g2)) w^T/||w||; lift_j <- 0.
template <int RP>
__global__ void geodesic_update_kernel(float* __restrict__ U, int64_t V,
                                       float* __restrict__ lift, const float* __restrict__ upd) {
  extern __shared__ float su[];
  for (int e = threadIdx.x; e < 3 * RP + 2; e += blockDim.x) su[e] = upd[e];
  __syncthreads();
  const float alpha = su[3 * RP], beta = su[3 * RP + 1];
  const float* w = su;
  const float* wh = su + RP;
  const float* g2 = su + 2 * RP;
  for (int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; j < V;
       j += int64_t(gridDim.x) * blockDim.x) {
    float4* u4 = reinterpret_cast<float4*>(U + j * RP);
    float4 x[RP / 4];
#pragma unroll
    for (int c4 = 0; c4 < RP / 4; ++c4) x[c4] = u4[c4];
    const float lj = lift[j];
    float p = 0.0f, g = 0.0f;
#pragma unroll
    for (int c4 = 0; c4 < RP / 4; ++c4) {
      p = fmaf(x[c4].x, w[4 * c4], fmaf(x[c4].y, w[4 * c4 + 1], fmaf(x[c4].z, w[4 * c4 + 2], fmaf(x[c4].w, w[4 * c4 + 3], p))));
      g = fmaf(x[c4].x, g2[4 * c4], fmaf(x[c4].y, g2[4 * c4 + 1], fmaf(x[c4].z, g2[4 * c4 + 2], fmaf(x[c4].w, g2[4 * c4 + 3], g))));
    }
    const float coef = alpha * p + beta * (lj - g);
    if (lj != 0.0f) lift[j] = 0.0f;
    if (coef != 0.0f) {
#pragma unroll
      for (int c4 = 0; c4 < RP / 4; ++c4) {
        x[c4].x = fmaf(coef, wh[4 * c4], x[c4].x);
        x[c4].y = fmaf(coef, wh[4 * c4 + 1], x[c4].y);
        x[c4].z = fmaf(coef, wh[4 * c4 + 2], x[c4].z);
        x[c4].w = fmaf(coef, wh[4 * c4 + 3], x[c4].w);
        u4[c4] = x[c4];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// W_ex = U^T T_ex^T (split over voxels, FP64 reduction of the splits)
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) wex_partial_kernel(const float* __restrict__ U,
                                                          const float* __restrict__ Tex,
                                                          int64_t V, int ell, int RP,
                                                          int64_t per_split,
                                                          float* __restrict__ part) {
  __shared__ float Ts[32][33];
  __shared__ float Us[32][kMaxRank];
  const int i0 = blockIdx.x * 32;
  const int64_t j0 = blockIdx.y * per_split, j1 = min(V, j0 + per_split);
  const int ti = threadIdx.x >> 3, cg = threadIdx.x & 7;  // row i0+ti, columns cg + 8k
  float acc[kMaxRank / 8];
#pragma unroll
  for (int k = 0; k < kMaxRank / 8; ++k) acc[k] = 0.0f;
  for (int64_t jb = j0; jb < j1; jb += 32) {
    for (int e = threadIdx.x; e < 32 * 32; e += blockDim.x) {
      const int r = e >> 5, jj = e & 31;
      const int64_t j = jb + jj;
      Ts[r][jj] = (i0 + r < ell && j < j1) ? Tex[int64_t(i0 + r) * V + j] : 0.0f;
    }
    for (int e = threadIdx.x; e < 32 * RP; e += blockDim.x) {
      const int jj = e / RP, c = e - jj * RP;
      const int64_t j = jb + jj;
      Us[jj][c] = j < j1 ? U[j * RP + c] : 0.0f;
    }
    __syncthreads();
    for (int jj = 0; jj < 32; ++jj) {
      const float t = Ts[ti][jj];
#pragma unroll
      for (int k = 0; k < kMaxRank / 8; ++k) {
        const int c = cg + 8 * k;
        if (c < RP) acc[k] = fmaf(t, Us[jj][c], acc[k]);
      }
    }
    __syncthreads();
  }
  if (i0 + ti < ell) {
#pragma unroll
    for (int k = 0; k < kMaxRank / 8; ++k) {
      const int c = cg + 8 * k;
      if (c < RP) part[(int64_t(blockIdx.y) * ell + i0 + ti) * RP + c] = acc[k];
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
// Recovery: sampled t, l1 weights (one block per relabelling, persistent)
// ---------------------------------------------------------------------------
struct RecArgs {
  const int32_t* perms;
  int n, n1, n_pad;
  const float* Xn32;  // v_pad x n_pad, unit-norm centred data
  uint32_t V;
  int R, RP, m;
  const float* U;
  uint32_t k0, k1;
  float rho;
  int iters;
  float kf, ctf;
  int64_t row_first, row_end;
  float* scratch;  // per block: A (m x RP), b, s, y (m each), blocks block_stride floats apart
  int64_t block_stride;  // multiple of 64 floats, so every A row stays 16-byte aligned
  float* W;        // (row - row_first) x RP
};

template <int RP>
__global__ void __launch_bounds__(kFitThreads) recover_fit_kernel(RecArgs a) {
  extern __shared__ float sm[];
  FitSmem f;
  carve_fit_smem(sm, RP, f);
  float* Lrow = f.scal + 8;  // n_pad
  float* A = a.scratch + int64_t(blockIdx.x) * a.block_stride;
  float* b = A + int64_t(a.m) * RP;
  float* s = b + a.m;
  float* y = s + a.m;
  float* x = y + a.m;
  if (a.m <= kSmemVecM) {
    b = Lrow + a.n_pad;
    s = b + a.m;
    y = s + a.m;
    x = y + a.m;
  }
  for (int64_t i = a.row_first + blockIdx.x; i < a.row_end; i += gridDim.x) {
    for (int sidx = threadIdx.x; sidx < a.n_pad; sidx += blockDim.x) Lrow[sidx] = 0.0f;
    __syncthreads();
    for (int q = threadIdx.x; q < a.n1; q += blockDim.x) {
      const int32_t e = a.perms[i * a.n + q];
      if (e >= 0 && e < a.n) Lrow[e] = 1.0f;  // bad rows are reported by validate_perms_kernel
    }
    __syncthreads();
    for (int q = threadIdx.x; q < a.m; q += blockDim.x) {
      const uint32_t j = draw_index(a.k0, a.k1, TAG_REC, uint32_t(q), uint32_t(i), 0u, a.V);
      const float4* xr = reinterpret_cast<const float4*>(a.Xn32 + int64_t(j) * a.n_pad);
      float u = 0.0f;
      for (int s4 = 0; s4 < a.n_pad / 4; ++s4) {
        const float4 x = xr[s4];
        u = fmaf(x.x, Lrow[4 * s4], fmaf(x.y, Lrow[4 * s4 + 1],
                 fmaf(x.z, Lrow[4 * s4 + 2], fmaf(x.w, Lrow[4 * s4 + 3], u))));
      }
      const float den = 1.0f - a.kf * u * u;
      b[q] = den > 0.0f ? a.ctf * u * rsqrtf(den) : (u > 0.0f ? 3.0e38f : -3.0e38f);
      const float4* src = reinterpret_cast<const float4*>(a.U + int64_t(j) * RP);
      float4* dst = reinterpret_cast<float4*>(A + int64_t(q) * RP);
      for (int c4 = 0; c4 < RP / 4; ++c4) dst[c4] = src[c4];
    }
    __syncthreads();
    block_l1_fit<RP>(A, b, s, y, x, a.m, a.R, a.rho, a.iters, f);
    for (int c = threadIdx.x; c < RP; c += blockDim.x)
      a.W[(i - a.row_first) * RP + c] = c < a.R ? f.wv[c] : 0.0f;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Reconstruct + noise + max (Alg. 2 recovery): rows = relabellings (weights W),
// columns = voxels (U). mode 0: value (U w)_j + sigma z_j; mode 1: residual
// T_ex[i][j] - (U w)_j (literal shift of Alg. 2). Each CTA walks a range of
// voxel tiles for one 128-row tile and keeps per-row running maxima.
// ---------------------------------------------------------------------------
struct ReconArgs {
  const float* W;  // rows x RP
  int64_t rows;
  int64_t row_label0;  // relabelling index of row 0 (noise counter)
  const float* U;      // V x RP
  int64_t V;
  int RP;
  float sigma;
  uint32_t tag, k0, k1;
  int mode;
  const float* Tex;  // mode 1
  int64_t tiles_per_cta;
  unsigned long long* maxkey;  // rows, zero on entry
};

__global__ void __launch_bounds__(256) reconstruct_max_kernel(ReconArgs a) {
  __shared__ __align__(16) float Ws[16][128];
  __shared__ __align__(16) float Us[16][128];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t r0 = int64_t(blockIdx.y) * 128;
  const int64_t vt0 = int64_t(blockIdx.x) * a.tiles_per_cta;
  const int64_t vtiles = (a.V + 127) / 128;
  const int64_t vt1 = min(vtiles, vt0 + a.tiles_per_cta);
  float best[8];
  uint32_t bj[8];
  float M[8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    best[q] = -INFINITY;
    bj[q] = 0xffffffffu;
    const int64_t row = r0 + ((q < 4) ? (ty * 4 + q) : (64 + ty * 4 + q - 4));
    M[q] = -INFINITY;
    if (row < a.rows) {
      const unsigned long long k = __ldcg(&a.maxkey[row]);
      if (k) M[q] = unpack_key_value(k);
    }
  }
  const float bound = a.mode == 0 ? a.sigma * kNoiseBound : 0.0f;
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
    // epilogue: bounded-noise skip, running maxima
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      const int64_t row = r0 + ((p < 4) ? (ty * 4 + p) : (64 + ty * 4 + p - 4));
      if (row >= a.rows) continue;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int64_t col = c0 + ((q < 4) ? (tx * 4 + q) : (64 + tx * 4 + q - 4));
        if (col >= a.V) continue;
        float val = acc[p][q];
        if (a.mode == 1) {
          val = a.Tex[row * a.V + col] - val;
        } else {
          if (val + bound < M[p]) continue;
          val = fmaf(a.sigma, draw_normal(a.k0, a.k1, a.tag, uint32_t(col),
                                          uint32_t(a.row_label0 + row)), val);
        }
        if (val > best[p] || (val == best[p] && uint32_t(col) < bj[p])) {
          best[p] = val;
          bj[p] = uint32_t(col);
        }
        M[p] = fmaxf(M[p], val);
      }
      // share the running maximum among the 16 threads of this row
      float mm = M[p];
#pragma unroll
      for (int o = 1; o < 16; o <<= 1) mm = fmaxf(mm, __shfl_xor_sync(0xffffffffu, mm, o));
      M[p] = mm;
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

// Calls f(std::integral_constant<int, RP>) for the padded rank RP (16..128).
template <class F>
bool with_rp(int rp, F&& f) {
  switch (rp) {
    case 16: f(std::integral_constant<int, 16>{}); return true;
    case 32: f(std::integral_constant<int, 32>{}); return true;
    case 48: f(std::integral_constant<int, 48>{}); return true;
    case 64: f(std::integral_constant<int, 64>{}); return true;
    case 80: f(std::integral_constant<int, 80>{}); return true;
    case 96: f(std::integral_constant<int, 96>{}); return true;
    case 112: f(std::integral_constant<int, 112>{}); return true;
    case 128: f(std::integral_constant<int, 128>{}); return true;
    default: return false;
  }
}

int grid_n(int64_t work, int threads, int cap = 152 * 16) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return int(b);
}

size_t fit_smem_bytes(int RP, int n_pad, int m) {
  const size_t vec = m <= kSmemVecM ? 4 * size_t(m) : 0;
  return sizeof(float) * (2 * RP * RP + 32 * RP + kStageFloats + 2 * RP + 8 + n_pad + vec);
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
      o.precision > 2) {
    set_error(ctx, "RapidPT: bad options");
    return PT_ERR_INVALID;
  }
  if (ctx->v_valid < 1 || ctx->v_valid >= (int64_t(1) << 31)) {
    set_error(ctx, "RapidPT: context has no voxel with a defined t");
    return PT_ERR_INVALID;
  }
  pl.R = rank;
  pl.RP = (rank + 15) / 16 * 16;
  pl.V = ctx->v_valid;
  pl.m = int(std::ceil(sample_rate * double(pl.V)));
  if (pl.m < rank) {
    set_error(ctx, "RapidPT: ceil(sample_rate * v) must be at least the rank");
    return PT_ERR_INVALID;
  }
  pl.k0 = uint32_t(o.seed & 0xffffffffull);
  pl.k1 = uint32_t(o.seed >> 32);
  return PT_OK;
}

// Orthonormalise U (V x RP) in place: FP64 Gram and factorisation, FP32 apply.
pt_status qr_inplace(pt_ctx* ctx, float* U, const RapidPlan& pl, Buf& part, Buf& rinv) {
  const int nparts = 152 * 2;
  const int npairs = pl.R * (pl.R + 1) / 2;
  if (!part.ensure(sizeof(double) * size_t(nparts) * npairs) ||
      !rinv.ensure(sizeof(float) * pl.RP * pl.RP))
    return nomem_r(ctx, "QR");
  const int gsm = 32 * pl.RP * int(sizeof(float));
  gram64_kernel<<<nparts, 1024, gsm, ctx->stream>>>(U, pl.V, pl.R, pl.RP, part.as<double>());
  PT_LAUNCH_CHECK(ctx);
  const int fsm = (pl.R * pl.R + pl.R) * int(sizeof(double));
  if (fsm > 48 * 1024)
    PT_CUDA_TRY(ctx, cudaFuncSetAttribute(qr_factor_kernel,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, fsm));
  qr_factor_kernel<<<1, 1024, fsm, ctx->stream>>>(part.as<double>(), nparts, pl.R, pl.RP,
                                                  rinv.as<float>());
  PT_LAUNCH_CHECK(ctx);
  qr_apply_kernel<<<grid_n(pl.V, 256), 256, pl.RP * pl.RP * sizeof(float), ctx->stream>>>(
      U, pl.V, pl.R, pl.RP, rinv.as<float>());
  PT_LAUNCH_CHECK(ctx);
  return PT_OK;
}

// Row maxima of (U w + sigma z) (mode 0) or of T_ex - U w (mode 1) for `rows`
// rows of W; keys zeroed here.
pt_status reconstruct(pt_ctx* ctx, const float* W, int64_t rows, int64_t label0, const float* U,
                      const RapidPlan& pl, float sigma, uint32_t tag, int mode, const float* Tex,
                      unsigned long long* keys) {
  PT_CUDA_TRY(ctx, cudaMemsetAsync(keys, 0, sizeof(unsigned long long) * rows, ctx->stream));
  const int64_t rtiles = (rows + 127) / 128;
  const int64_t vtiles = (pl.V + 127) / 128;
  int64_t per = vtiles;
  const int64_t want = 152 * 8;
  if (rtiles < want) {
    int64_t split = (want + rtiles - 1) / rtiles;
    if (split > vtiles) split = vtiles;
    per = (vtiles + split - 1) / split;
  }
  ReconArgs a;
  a.W = W;
  a.rows = rows;
  a.row_label0 = label0;
  a.U = U;
  a.V = pl.V;
  a.RP = pl.RP;
  a.sigma = sigma;
  a.tag = tag;
  a.k0 = pl.k0;
  a.k1 = pl.k1;
  a.mode = mode;
  a.Tex = Tex;
  a.tiles_per_cta = per;
  a.maxkey = keys;
  const dim3 grid{unsigned((vtiles + per - 1) / per), unsigned(rtiles), 1u};
  prof_begin(ctx);
  reconstruct_max_kernel<<<grid, 256, 0, ctx->stream>>>(a);
  prof_end(ctx);
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
  Buf Ub, Tex, lift, sc, upd, part, rinv, Wex, keys, sig, tmax;
  struct G {
    std::vector<Buf*> v;
    ~G() {
      for (Buf* b : v) b->release();
    }
  } guard{{&Ub, &Tex, &lift, &sc, &upd, &part, &rinv, &Wex, &keys, &sig, &tmax}};
  if (!Ub.ensure(sizeof(float) * size_t(V) * pl.RP) || !Tex.ensure(sizeof(float) * size_t(ell) * V) ||
      !lift.ensure(sizeof(float) * V) ||
      !sc.ensure(sizeof(float) * (size_t(pl.m) * pl.RP + 5 * size_t(pl.m)) + 256) ||
      !upd.ensure(sizeof(float) * (3 * pl.RP + 4)) || !Wex.ensure(sizeof(float) * size_t(ell) * pl.RP) ||
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
      if (s == PT_OK) s = ensure_xnb(ctx);
      if (s == PT_OK) s = build_labels(ctx, perms, ell, 1, &P_pad);
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
    finalize_max_kernel<<<grid_n((ell + 7) / 8, 1), 256, 0, st>>>(
        ctx->maxkey.as<unsigned long long>(), ell, ctx->valid_map.as<int32_t>(),
        ctx->Xraw.as<float>(), ctx->n, ctx->n1, ctx->n_pad, perms, 0, tmax.as<float>(),
        reinterpret_cast<int32_t*>(keys.p));
    PT_LAUNCH_CHECK(ctx);
    if (counts) {
      scatter_counts_kernel<<<grid_n(V, 256), 256, 0, st>>>(
          ctx->cnt.as<uint32_t>(), V, ctx->valid_map.as<int32_t>(), counts);
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
  PT_CUDA_TRY(ctx, cudaMemsetAsync(lift.p, 0, sizeof(float) * V, st));

  // 3. sequential subspace tracking over passes x columns
  float* scb = sc.as<float>();
  StepArgs sa;
  sa.U = U;
  sa.V = uint32_t(V);
  sa.R = pl.R;
  sa.RP = pl.RP;
  sa.m = pl.m;
  sa.k0 = pl.k0;
  sa.k1 = pl.k1;
  sa.rho = o.admm_rho;
  sa.iters = o.admm_iters;
  sa.step = o.step;
  sa.A = scb;
  sa.b = scb + size_t(pl.m) * pl.RP;
  sa.s = sa.b + pl.m;
  sa.y = sa.s + pl.m;
  sa.x = sa.y + pl.m;
  sa.idx = reinterpret_cast<int32_t*>(sa.x + pl.m);
  sa.lift = lift.as<float>();
  sa.upd = upd.as<float>();
  const int fsm = int(fit_smem_bytes(pl.RP, 0, pl.m));
  const int usm = (3 * pl.RP + 2) * int(sizeof(float));
  int64_t steps = 0;
  cudaError_t lerr = cudaSuccess;
  with_rp(pl.RP, [&](auto rpc) {
    constexpr int RPc = decltype(rpc)::value;
    lerr = cudaFuncSetAttribute(train_step_kernel<RPc>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, fsm);
    for (int p = 0; p < o.train_passes && lerr == cudaSuccess && s == PT_OK; ++p) {
      for (int i = 0; i < ell; ++i) {
        sa.pass = p;
        sa.col = i;
        sa.Trow = Tex.as<float>() + int64_t(i) * V;
        sa.w_hist = w_hist ? w_hist + steps * pl.R : nullptr;
        train_step_kernel<RPc><<<1, kFitThreads, fsm, st>>>(sa);
        geodesic_update_kernel<RPc><<<grid_n(V, 256, 152 * 8), 256, usm, st>>>(
            U, V, lift.as<float>(), upd.as<float>());
        lerr = cudaGetLastError();
        if (lerr != cudaSuccess) break;
        count_launch();
        count_launch();
        ++steps;
        if (steps % o.qr_every == 0) {
          s = qr_inplace(ctx, U, pl, part, rinv);
          if (s != PT_OK) break;
        }
      }
    }
  });
  if (lerr != cudaSuccess) {
    set_error(ctx, std::string("RapidPT training launch: ") + cudaGetErrorString(lerr));
    return PT_ERR_CUDA;
  }
  if (s != PT_OK) return s;
  s = qr_inplace(ctx, U, pl, part, rinv);
  if (s != PT_OK) return s;

  // 4. W_ex = U^T T_ex (rows of Wex = weights of training columns)
  {
    const int itiles = (ell + 31) / 32;
    int nsplit = std::max(1, int(152 * 4 / itiles));
    nsplit = int(std::min<int64_t>(nsplit, (V + 1023) / 1024));
    const int64_t per = (V + nsplit - 1) / nsplit;
    if (!part.ensure(std::max(part.bytes, sizeof(float) * size_t(nsplit) * ell * pl.RP)))
      return nomem_r(ctx, "W_ex");
    const dim3 grid{unsigned(itiles), unsigned(nsplit), 1u};
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
  Buf Ub, scr, Wb, keys;
  struct G {
    std::vector<Buf*> v;
    ~G() {
      for (Buf* b : v) b->release();
    }
  } guard{{&Ub, &scr, &Wb, &keys}};
  const int nblk = int(std::min<int64_t>(rows, 152));
  const int64_t block_stride = (int64_t(pl.m) * pl.RP + 4 * int64_t(pl.m) + 63) / 64 * 64;
  if (!Ub.ensure(sizeof(float) * size_t(pl.V) * pl.RP) ||
      !scr.ensure(sizeof(float) * size_t(nblk) * size_t(block_stride)) ||
      !Wb.ensure(sizeof(float) * size_t(rows) * pl.RP) ||
      !keys.ensure(sizeof(unsigned long long) * rows))
    return nomem_r(ctx, "RapidPT recovery");
  validate_perms_kernel<<<grid_n((rows + 7) / 8, 1), 256, 0, st>>>(perms, first_row, P, ctx->n,
                                                                   ctx->status.as<uint32_t>());
  PT_LAUNCH_CHECK(ctx);
  pack_u_kernel<<<grid_n(pl.V * pl.RP, 256), 256, 0, st>>>(U_in, pl.V, pl.R, pl.RP,
                                                          Ub.as<float>(), 1);
  PT_LAUNCH_CHECK(ctx);
  RecArgs a;
  a.perms = perms;
  a.n = ctx->n;
  a.n1 = ctx->n1;
  a.n_pad = ctx->n_pad;
  a.Xn32 = ctx->Xn32.as<float>();
  a.V = uint32_t(pl.V);
  a.R = pl.R;
  a.RP = pl.RP;
  a.m = pl.m;
  a.U = Ub.as<float>();
  a.k0 = pl.k0;
  a.k1 = pl.k1;
  a.rho = o.admm_rho;
  a.iters = o.admm_iters;
  a.kf = float(ctx->k);
  a.ctf = float(ctx->c_t);
  a.row_first = first_row;
  a.row_end = P;
  a.scratch = scr.as<float>();
  a.block_stride = block_stride;
  a.W = Wb.as<float>();
  const int fsm = int(fit_smem_bytes(pl.RP, ctx->n_pad, pl.m));
  cudaError_t lerr = cudaSuccess;
  with_rp(pl.RP, [&](auto rpc) {
    constexpr int RPc = decltype(rpc)::value;
    lerr = cudaFuncSetAttribute(recover_fit_kernel<RPc>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize, fsm);
    if (lerr == cudaSuccess) {
      recover_fit_kernel<RPc><<<nblk, kFitThreads, fsm, st>>>(a);
      lerr = cudaGetLastError();
    }
  });
  if (lerr != cudaSuccess) {
    set_error(ctx, std::string("RapidPT recovery launch: ") + cudaGetErrorString(lerr));
    return PT_ERR_CUDA;
  }
  count_launch();
  s = reconstruct(ctx, Wb.as<float>(), rows, first_row, Ub.as<float>(), pl, float(sigma),
                  TAG_NOISE, 0, nullptr, keys.as<unsigned long long>());
  if (s != PT_OK) return s;
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

}  // namespace pt

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

void pt_rapid_opts_default(pt_rapid_opts* o) {
  if (!o) return;
  o->precision = PT_PREC_BF16X3;
  o->train_passes = 10;
  o->qr_every = 100;
  o->admm_iters = 30;
  o->admm_rho = 2.0f;
  o->step = 1.0f;
  o->shift_mode = 1;
  o->seed = 1;
}

pt_status pt_rapid_train(pt_ctx* ctx, const int32_t* perms, int32_t n_train, int32_t rank,
                         double sample_rate, const pt_rapid_opts* opts, float* U_out,
                         float* train_max, uint32_t* counts, float* w_hist,
                         pt_rapid_info* info) {
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
