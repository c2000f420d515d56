// pt_maxnull_naive_noalloc: the NaivePT path (FP32 CUDA-core contraction) for
// callers that cannot allocate device memory. Some callers run where
// cudaMalloc is not available to them: inside a memory pool that another
// runtime owns, in code that must not change the device's memory footprint
// after start-up, or under allocation-free real-time rules. This entry point
// needs no allocation at all: every intermediate buffer lives in one
// file-scope static device array of fixed size, which every GPU that loads
// this library holds until the process exits.
//
// The array's name in host code is only a host-side stand-in, not a device
// address, so the host asks the runtime for its device address
// (cudaGetSymbolAddress) with the caller's device and context current. An
// address is valid only in the context it was looked up in: another context
// on the same device (one the caller made with cuCtxCreate, or the primary
// context again after cudaDeviceReset) holds its own copy of the array. So
// the lookup is made on every call; it is a host-side table lookup once the
// module is loaded in that context.
//
// The call is synchronous: it copies two status words to host memory and
// waits on the stream in the middle of the work and at its end. Every call
// shares the array and it keeps the previous call's contents; calls that
// overlap on the GPU (two streams, two host threads) race on it and must be
// serialised by the caller.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <string>

#include "pt_internal.h"

namespace pt {

// Kernels of the regular NaivePT path, reused unchanged (pt_naive.cu).
__global__ void labels_kernel(const int32_t* perms, int64_t P, int64_t P_pad, int n, int n1,
                              int n_pad, int layout, void* Lout, uint8_t* rowflag,
                              uint8_t* blockflag, uint32_t* ident_count, uint32_t* status);
__global__ void simt_contract_kernel(const float* L, const float* Xn, int n_pad, int64_t P,
                                     int64_t v, int tiles_per_cta, int mode, int two_sided,
                                     const float* u_obs, const uint8_t* rowflag,
                                     unsigned long long* maxkey, uint32_t* cnt, float* uout);
__global__ void finalize_max_kernel(const unsigned long long* maxkey, int64_t P,
                                    const int32_t* valid_map, const float* Xraw, int n, int n1,
                                    int n_pad, const int32_t* perms, int two_sided,
                                    float* maxnull, int32_t* argmax);
__global__ void scatter_counts_kernel(const uint32_t* cnt, int64_t v_valid,
                                      const int32_t* valid_map, uint32_t* counts,
                                      int accumulate);

namespace {

constexpr size_t kNoallocScratchBytes = size_t(64) << 20;  // 64 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Per-voxel moments in one FP64 pass over values shifted by the voxel's first
// value x_0 (which keeps the sums of squares well conditioned): eight partial
// sums over subjects s = w, w + 8, ... (w = 0..7), added in order w = 0..7.
// The validity rule is the regular path's (finite values, not all equal,
// positive centred sum of squares). The regular moments step is a different
// two-pass float-float computation, so mean, 1/sqrt(SS) and the observed u
// agree with it to rounding, not bit for bit; the outputs agree with the
// regular path within its tolerances.
__global__ void noalloc_moments_kernel(const float* __restrict__ X, int n, int n1, int n_pad,
                                       int64_t v, float* __restrict__ Xraw,
                                       double* __restrict__ mean, double* __restrict__ inv_norm,
                                       float* __restrict__ u_obs_m, uint8_t* __restrict__ valid,
                                       uint32_t* __restrict__ status) {
  const int64_t j = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (j >= v) return;
  for (int s = 0; s < n_pad; ++s) Xraw[j * n_pad + s] = s < n ? X[int64_t(s) * v + j] : 0.0f;
  const float x0f = X[j];
  const double x0 = double(x0f);
  double S1 = 0.0, S2 = 0.0, Q1 = 0.0, Q2 = 0.0;
  bool nonfinite = false, differs = false;
  for (int w = 0; w < 8; ++w) {
    double s1 = 0.0, s2 = 0.0, q1 = 0.0, q2 = 0.0;
    for (int s = w; s < n; s += 8) {
      const float xf = X[int64_t(s) * v + j];
      if (!isfinite(xf)) nonfinite = true;
      if (xf != x0f) differs = true;
      const double d = double(xf) - x0;
      if (s < n1) {
        s1 += d;
        q1 = fma(d, d, q1);
      } else {
        s2 += d;
        q2 = fma(d, d, q2);
      }
    }
    S1 += s1;
    S2 += s2;
    Q1 += q1;
    Q2 += q2;
  }
  if (nonfinite) {
    atomicOr(status, kErrBadData);
    valid[j] = 0;
    return;
  }
  const double S = S1 + S2, Q = Q1 + Q2;
  const double md = S / n;
  const double SS = Q - S * md;
  const bool ok = differs && SS > 0.0;
  valid[j] = ok ? 1 : 0;
  mean[j] = x0 + md;
  if (!ok) {
    inv_norm[j] = 0.0;
    u_obs_m[j] = 0.0f;
    return;
  }
  const double inv = 1.0 / sqrt(SS);
  inv_norm[j] = inv;
  u_obs_m[j] = float((S1 - n1 * md) * inv);
}

// Single-block compaction of the valid flags (index order); count at *total.
__global__ void noalloc_compact_kernel(const uint8_t* __restrict__ valid, int64_t v,
                                       int32_t* __restrict__ valid_map, uint32_t* __restrict__ total) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < v; b0 += blockDim.x) {
    const int64_t j = b0 + threadIdx.x;
    const uint32_t f = (j < v && valid[j]) ? 1u : 0u;
    const uint32_t bal = __ballot_sync(0xffffffffu, f);
    const uint32_t before_lane = __popc(bal & ((1u << lane) - 1u));
    if (lane == 0) warp_tot[w] = __popc(bal);
    __syncthreads();
    uint32_t before_warp = 0;
    for (int q = 0; q < w; ++q) before_warp += warp_tot[q];
    if (f) valid_map[carry + before_warp + before_lane] = int32_t(j);
    __syncthreads();
    if (threadIdx.x == 0) {
      uint32_t t = 0;
      for (int q = 0; q < int(blockDim.x >> 5); ++q) t += warp_tot[q];
      carry += t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *total = carry;
}

// Same centring arithmetic as the regular operand builder.
__device__ __forceinline__ float noalloc_unit_centre(float x, float4 st) {
  const float s = x - st.x;
  const float bb = s - x;
  const float e = (x - (s - bb)) + (-st.x - bb);
  const float dl = e - st.y;
  const float p = s * st.z;
  const float pe = fmaf(s, st.z, -p);
  return p + (pe + fmaf(s, st.w, dl * st.z));
}

__global__ void noalloc_xn32_kernel(const float* __restrict__ Xraw, int n, int n_pad,
                                    const int32_t* __restrict__ valid_map, int64_t v_valid,
                                    int64_t v_pad, const double* __restrict__ mean,
                                    const double* __restrict__ inv_norm,
                                    const float* __restrict__ u_obs_m, float* __restrict__ u_obs,
                                    float* __restrict__ Xn32) {
  const int64_t total = v_pad * n_pad;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total;
       e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t c = e / n_pad;
    const int s = int(e - c * n_pad);
    float y = 0.0f;
    if (c < v_valid) {
      const int32_t j = valid_map[c];
      const double m = mean[j], iv = inv_norm[j];
      float4 st;
      st.x = float(m);
      st.y = float(m - double(st.x));
      st.z = float(iv);
      st.w = float(iv - double(st.z));
      if (s < n) y = noalloc_unit_centre(Xraw[int64_t(j) * n_pad + s], st);
      if (s == 0) u_obs[c] = u_obs_m[j];
    } else if (s == 0) {
      u_obs[c] = INFINITY;
    }
    Xn32[e] = y;
  }
}

int blocks_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return int(b);
}

pt_status fail(pt_status st, const std::string& msg) {
  set_thread_error("pt_maxnull_naive_noalloc: " + msg);
  return st;
}

#define NA_TRY(call)                                                            \
  do {                                                                          \
    cudaError_t _e = (call);                                                    \
    if (_e != cudaSuccess) return fail(PT_ERR_CUDA, std::string(#call) + ": " + \
                                                        cudaGetErrorString(_e)); \
  } while (0)

}  // namespace

size_t noalloc_scratch_needed(int32_t n, int64_t v, int64_t P) {
  const int64_t n_pad = (n + 15) / 16 * 16;
  const int64_t v_pad = (v + 255) / 256 * 256;
  const int64_t P_pad = (P + 127) / 128 * 128;
  size_t b = 0;
  b += up256(2 * sizeof(uint32_t));                      // status, valid count
  b += up256(sizeof(float) * v * n_pad);                 // Xraw
  b += up256(v);                                         // valid flags
  b += 2 * up256(sizeof(double) * v);                    // mean, 1/sqrt(SS)
  b += up256(sizeof(float) * v);                         // u_obs (mask order)
  b += up256(sizeof(int32_t) * v);                       // valid map
  b += up256(sizeof(float) * v_pad);                     // u_obs (compact)
  b += up256(sizeof(float) * v_pad * n_pad);             // Xn32
  b += up256(sizeof(float) * P_pad * n_pad);             // labels
  b += up256(P_pad) + up256(P_pad / 128);                // row / block flags
  b += up256(sizeof(unsigned long long) * P);            // row maxima
  b += up256(sizeof(uint32_t) * (v + 1));                // counts + observed-set rows
  return b;
}

}  // namespace pt

extern "C" pt_status pt_maxnull_naive_noalloc(const float* X, int32_t n, int64_t v, int32_t n1,
                                              const int32_t* perms, int64_t P, int32_t two_sided,
                                              float* maxnull, int32_t* argmax, uint32_t* counts,
                                              void* stream) {
  using namespace pt;
  if (!X || !perms || !maxnull || !argmax)
    return fail(PT_ERR_INVALID, "X, perms, maxnull and argmax must be non-NULL");
  if (n < 3 || n > 1024 || n1 < 1 || n1 > n - 1 || v < 1 || v >= (int64_t(1) << 31) || P < 1 ||
      P > INT32_MAX || (two_sided != 0 && two_sided != 1))
    return fail(PT_ERR_INVALID, "need 3 <= n <= 1024, 1 <= n1 <= n-1, v >= 1, P >= 1");
  const size_t need = noalloc_scratch_needed(n, v, P);
  if (need > kNoallocScratchBytes)
    return fail(PT_ERR_INVALID, "problem needs " + std::to_string(need) +
                                    " bytes of scratch; the static limit is " +
                                    std::to_string(kNoallocScratchBytes) + " bytes");
  // The array's device address in the current context (see the file comment).
  void* sym = nullptr;
  {
    const cudaError_t e = cudaGetSymbolAddress(&sym, g_noalloc_scratch);
    if (e != cudaSuccess || !sym)
      return fail(PT_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  }
  unsigned char* base = static_cast<unsigned char*>(sym);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n_pad = (n + 15) / 16 * 16;
  const int64_t v_pad = (v + 255) / 256 * 256;
  const int64_t P_pad = (P + 127) / 128 * 128;
  size_t off = 0;
  auto carve = [&](size_t bytes) {
    unsigned char* p = base + off;
    off += up256(bytes);
    return p;
  };
  uint32_t* status = reinterpret_cast<uint32_t*>(carve(2 * sizeof(uint32_t)));
  float* Xraw = reinterpret_cast<float*>(carve(sizeof(float) * v * n_pad));
  uint8_t* valid = carve(v);
  double* mean = reinterpret_cast<double*>(carve(sizeof(double) * v));
  double* inv_norm = reinterpret_cast<double*>(carve(sizeof(double) * v));
  float* u_obs_m = reinterpret_cast<float*>(carve(sizeof(float) * v));
  int32_t* valid_map = reinterpret_cast<int32_t*>(carve(sizeof(int32_t) * v));
  float* u_obs = reinterpret_cast<float*>(carve(sizeof(float) * v_pad));
  float* Xn32 = reinterpret_cast<float*>(carve(sizeof(float) * v_pad * n_pad));
  float* L = reinterpret_cast<float*>(carve(sizeof(float) * P_pad * n_pad));
  uint8_t* rowflag = carve(P_pad);
  uint8_t* blockflag = carve(P_pad / 128);
  unsigned long long* maxkey = reinterpret_cast<unsigned long long*>(carve(sizeof(unsigned long long) * P));
  uint32_t* cnt = reinterpret_cast<uint32_t*>(carve(sizeof(uint32_t) * (v + 1)));

  // The array keeps the previous call's contents: clear what must start at zero.
  NA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(uint32_t), st));
  NA_TRY(cudaMemsetAsync(maxkey, 0, sizeof(unsigned long long) * P, st));
  NA_TRY(cudaMemsetAsync(cnt, 0, sizeof(uint32_t) * (v + 1), st));
  NA_TRY(cudaMemsetAsync(blockflag, 0, P_pad / 128, st));
  if (counts) NA_TRY(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * v, st));

  noalloc_moments_kernel<<<unsigned((v + 127) / 128), 128, 0, st>>>(
      X, n, n1, n_pad, v, Xraw, mean, inv_norm, u_obs_m, valid, status);
  noalloc_compact_kernel<<<1, 1024, 0, st>>>(valid, v, valid_map, status + 1);
  NA_TRY(cudaGetLastError());
  uint32_t hb[2] = {0, 0};
  NA_TRY(cudaMemcpyAsync(hb, status, sizeof(hb), cudaMemcpyDeviceToHost, st));
  NA_TRY(cudaStreamSynchronize(st));
  if (hb[0] & kErrBadData) return fail(PT_ERR_INVALID, "X holds NaN or Inf");
  const int64_t v_valid = hb[1];

  noalloc_xn32_kernel<<<blocks_for(v_pad * n_pad, 256), 256, 0, st>>>(
      Xraw, n, n_pad, valid_map, v_valid, v_pad, mean, inv_norm, u_obs_m, u_obs, Xn32);
  labels_kernel<<<unsigned((P_pad + 7) / 8), 256, 0, st>>>(perms, P, P_pad, n, n1, n_pad, 0, L,
                                                           rowflag, blockflag, cnt + v_valid,
                                                           status);
  if (v_valid > 0) {
    const int64_t vt = (v_valid + 127) / 128;
    const int64_t ptiles = P_pad / 128;
    int64_t chunks = (152 * 2 * 4 + vt - 1) / vt;
    if (chunks > ptiles) chunks = ptiles;
    if (chunks < 1) chunks = 1;
    if (chunks > 65535) chunks = 65535;
    const int per = int((ptiles + chunks - 1) / chunks);
    chunks = (ptiles + per - 1) / per;
    const dim3 grid{unsigned(vt), unsigned(chunks), 1u};
    simt_contract_kernel<<<grid, 256, 0, st>>>(L, Xn32, n_pad, P, v_valid, per, 0, two_sided,
                                               u_obs, rowflag, maxkey, cnt, nullptr);
  }
  const int fin_blocks = blocks_for((P + kFinRowsPerBlock - 1) / kFinRowsPerBlock, 1);
  finalize_max_kernel<<<fin_blocks, 256, 0, st>>>(
      maxkey, P, valid_map, Xraw, n, n1, n_pad, perms, two_sided, maxnull, argmax);
  if (counts && v_valid > 0)
    scatter_counts_kernel<<<blocks_for(v_valid, 256), 256, 0, st>>>(cnt, v_valid, valid_map,
                                                                    counts, 0);
  NA_TRY(cudaGetLastError());
  uint32_t bits = 0;
  NA_TRY(cudaMemcpyAsync(&bits, status, sizeof(bits), cudaMemcpyDeviceToHost, st));
  NA_TRY(cudaStreamSynchronize(st));
  if (bits & kErrBadPerm) return fail(PT_ERR_INVALID, "a relabelling row is not a permutation");
  return PT_OK;
}
