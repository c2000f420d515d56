// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/pt.h"

namespace pt {

// Device-side error bits, OR-ed into the context's status word by kernels.
enum : uint32_t {
  kErrBadPerm = 1u,   // a relabelling row is not a permutation of 0..n-1
  kErrTimeout = 2u,   // a bounded spin-wait expired
  kErrBadData = 4u,   // NaN / Inf in the input data
  kErrGlmSpan = 8u,   // a relabelled group column lies in the span of the covariates
};

// Relabelling rows finished per 256-thread CTA by finalize_max_kernel.
constexpr int kFinRowsPerBlock = 16;

// Covariate-adjusted statistic: at most this many columns in [1, Z].
constexpr int kGlmMaxQ1 = 17;

// Caching device allocator: blocks are keyed by (device, rounded size) and
// recycled, so steady-state calls never reach cudaMalloc.
void* dev_alloc(size_t bytes);
void dev_free(void* p);
// Frees blocks once ev (owned by the cache from here) has completed.
void dev_free_after(const std::vector<void*>& ps, cudaEvent_t ev);

// A device buffer owned by a context; grows on demand, never shrinks.
struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
  bool ensure(size_t want);  // false on allocation failure
  void release();
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

}  // namespace pt

struct pt_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int32_t n = 0, n1 = 0, n2 = 0, n_pad = 0;
  int64_t n_grid = 0;
  int64_t v = 0;        // mask voxels
  int64_t v_valid = 0;  // voxels with a defined t
  int64_t v_pad = 0;    // v_valid rounded up to 256
  double k = 0.0;       // 1/n1 + 1/n2
  double c_t = 0.0;     // sqrt(k (n - 2)): t = c_t u / sqrt(1 - k u^2)
  std::string last_error;

  pt::Buf status;       // uint32 error bits
  pt::Buf vox_grid;     // int64[v]: grid index of masked voxel j
  pt::Buf valid_map;    // int32[v_valid]: masked index of compact voxel c
  pt::Buf t_obs64;      // double[v]: observed t (NaN if degenerate)
  pt::Buf Xraw;         // float[v][n_pad]: input values, masked order, voxel-major
  pt::Buf vstat;        // float4[v_pad]: (mean hi, mean lo, 1/sqrt(SS) hi, lo), compact order
  pt::Buf u_obs;        // float[v_pad]: observed group-1 share of the unit-norm voxel, compact
  pt::Buf Xn32;         // float[v_pad][n_pad]: unit-norm centred data (built on first FP32 use)
  pt::Buf Xnb;          // bf16 pieces 3 x [v_pad/8][n_pad/8][8][8] (built on first tensor-core use)
  bool have_xn32 = false, have_xnb = false;
  bool xnb_f16 = false;  // Xnb holds the FP16 pieces (PT_PREC_FP16X2), else BF16 pieces

  // Per-call workspaces (grown on demand).
  pt::Buf labels;       // float or bf16 labels
  pt::Buf rowflag;      // uint8[P_pad]: relabelling has the observed group-1 set
  pt::Buf blockflag;    // uint8[P_pad/128]: 128-row block holds such a row
  pt::Buf maxkey;       // uint64[P]
  pt::Buf cnt;          // uint32[v_valid + 1]; the last word counts observed-set rows
  pt::Buf scratch;      // misc
  pt::Buf moments;      // pt_prepare's per-voxel FP64 moments (read by kernels it enqueues)
  pt::Buf tcdesc;       // device copy of the tensor-core launch descriptor

  // Covariate-adjusted statistic (pt_prepare_glm); glm_q1 = 0 for the plain t.
  int32_t glm_q1 = 0;   // columns of [1, Z]
  double glm_a_obs = 0.0, glm_df = 0.0;
  pt::Buf glmQ;         // double[n][q1]: orthonormal basis of [1, Z]
  pt::Buf glm_coef;     // double[v][q1]: Q^T x per masked voxel
  pt::Buf glm_inv;      // double[v]: 1 / ||x - Q Q^T x||
  pt::Buf rowscale;     // float[P_pad]: sqrt(a_obs / a(l)) per relabelling

  // Cluster-level summaries: grid index -> compact voxel (-1 outside the mask or
  // without a statistic), built on first use for the grid shape in grid_dims.
  pt::Buf grid_inv;
  int64_t grid_dims[3] = {0, 0, 0};

  // Profiling of the dominant kernel (events on `stream`).
  bool profile = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pending, ev_pool;
};

namespace pt {

// NVTX range over a host-side phase (prepare, max-null, training, recovery,
// tuning): shows in profilers' timelines, free when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

void set_error(pt_ctx* ctx, const std::string& msg);
void count_launch();
void add_launch_count(int64_t k);
int64_t launch_counter();
// Event pair around the dominant kernel when profiling is on (no-ops otherwise).
void prof_begin(pt_ctx* ctx);
void prof_end(pt_ctx* ctx);
void set_thread_error(const std::string& msg);

// ---- prepare (pt_prepare.cu) ----
pt_status prepare_impl(pt_ctx* ctx, const float* X, const uint8_t* mask);

// ---- covariate-adjusted statistic (pt_glm.cu) ----
pt_status glm_setup(pt_ctx* ctx, const double* Z, int q);      // host basis, before prepare
pt_status glm_moments(pt_ctx* ctx, uint8_t* valid, float* u_obs_m);
pt_status glm_build_xnb(pt_ctx* ctx);
pt_status glm_rowscale(pt_ctx* ctx, const int32_t* perms, int64_t P, int64_t P_pad);
pt_status glm_finalize(pt_ctx* ctx, const int32_t* perms, int64_t P, int two_sided,
                       float* maxnull, int32_t* argmax);
// Operand layouts built from Xraw on first use (FP32 rows / BF16 pieces).
pt_status ensure_xn32(pt_ctx* ctx);
pt_status ensure_xnb(pt_ctx* ctx, int precision);

// Tensor-core operand forms of each precision: data pieces per k-step, label
// layout (0 FP32 rows, 1 BF16 core matrices, 2 FP16 core matrices), and the
// power-of-two scale of the FP16 data pieces (|Xn| < 1, so 2^15 Xn < 32768 is
// in FP16 range and the low piece stays a normal FP16 number for |Xn| >= 2^-18).
inline int prec_pieces(int precision) { return precision == PT_PREC_BF16X3 ? 3 : 2; }
inline int prec_label_layout(int precision) {
  return precision == PT_PREC_FP32 ? 0 : (precision == PT_PREC_FP16X2 ? 2 : 1);
}
constexpr float kF16Scale = 32768.0f;

// ---- RapidPT (pt_rapid.cu) ----
pt_status rapid_train_impl(pt_ctx* ctx, const int32_t* perms, int32_t n_train, int32_t rank,
                           double sample_rate, const pt_rapid_opts& o, float* U_out,
                           float* train_max, uint32_t* counts, float* w_hist,
                           pt_rapid_info* info);
pt_status t_rows_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, int precision, float* T);
pt_status rapid_recover_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, int64_t first_row,
                             const float* U_in, int32_t rank, double sample_rate, double sigma,
                             double mu, const pt_rapid_opts& o, float* maxnull, float* W_out);

// ---- reconstruction with noise on the tensor cores (pt_recon_tc.cu) ----
// keys[i] (zero or an earlier key on entry) <- max with the packed (value,
// voxel) maximum over voxels j of (W_i . U_j) + sigma z(tag, j, label0 + i);
// W rows x RP, U V x RP (FP32, padded columns zero), RP <= 128.
pt_status recon_tc(pt_ctx* ctx, const float* W, int64_t rows, int64_t label0, const float* U,
                   int64_t V, int RP, float sigma, uint32_t tag, uint32_t k0, uint32_t k1,
                   unsigned long long* keys);

// ---- naive path (pt_naive.cu) ----
pt_status naive_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, const pt_naive_opts& o,
                     float* maxnull, int32_t* argmax, uint32_t* counts);
pt_status naive_batched_impl(pt_ctx* const* ctxs, int n, const int32_t* const* perms,
                             const int64_t* P, const pt_naive_opts& o, float* const* maxnull,
                             int32_t* const* argmax, uint32_t* const* counts);
// The F of a g-group factor in the fused kernel (FG = 2 or 4 label rows per
// relabelling): per-relabelling maxima of B = u^T W u into keys, counts B >= B_obs.
pt_status tc_f_reduce(pt_ctx* ctx, const void* Lb, int64_t rows, int precision, int fg,
                      const float* b_obs, const float* fmat, int64_t fstride,
                      unsigned long long* keys, uint32_t* cnt);
pt_status anova_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, const int32_t* sizes, int g,
                     int precision, float* maxnull, int32_t* argmax, uint32_t* counts);
pt_status cluster_maxnull_impl(pt_ctx* ctx, const int32_t* perms, int64_t P, double tau,
                               const int32_t* dims, int connectivity, int precision,
                               int32_t* maxsize);
pt_status cluster_observed_impl(pt_ctx* ctx, double tau, const int32_t* dims, int connectivity,
                                int32_t* label, int32_t* size);
pt_status fwer_pvalues_impl(pt_ctx* ctx, const float* maxnull, int64_t P, int two_sided,
                            float* p_out);
// Drops a cached batched graph that names this context (from pt_destroy);
// true if it did.
bool batch_forget(const pt_ctx* ctx);
// Drops the cached batched graph (the tuned configurations changed).
void batch_drop_graph();

}  // namespace pt

#define PT_CUDA_TRY(ctx, call)                                                        \
  do {                                                                                \
    cudaError_t _e = (call);                                                          \
    if (_e != cudaSuccess) {                                                          \
      pt::set_error((ctx), std::string(#call) + ": " + cudaGetErrorString(_e));       \
      return _e == cudaErrorMemoryAllocation ? PT_ERR_NOMEM : PT_ERR_CUDA;            \
    }                                                                                 \
  } while (0)

#define PT_LAUNCH_CHECK(ctx)                                                          \
  do {                                                                                \
    cudaError_t _e = cudaGetLastError();                                              \
    if (_e != cudaSuccess) {                                                          \
      pt::set_error((ctx), std::string("kernel launch: ") + cudaGetErrorString(_e));  \
      return PT_ERR_CUDA;                                                             \
    }                                                                                 \
    pt::count_launch();                                                               \
  } while (0)
