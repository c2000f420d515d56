// C-ABI entry points, context lifetime, caching device allocator, errors.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "pt_internal.h"

namespace pt {

// ---------------------------------------------------------------------------
// Caching allocator. Sizes are rounded up (256 B below 1 MiB, 2 MiB above) and
// freed blocks wait in a per-(device, size) free list until reused.
// ---------------------------------------------------------------------------
namespace {
std::mutex g_alloc_mu;
std::map<std::pair<int, size_t>, std::vector<void*>> g_free;
std::map<void*, std::pair<int, size_t>> g_live;
// Blocks of destroyed contexts whose work may still be queued: reusable once
// the event recorded behind that work has completed.
struct Deferred {
  cudaEvent_t ev;
  std::vector<std::pair<void*, std::pair<int, size_t>>> blocks;
};
std::vector<Deferred> g_deferred;

// Moves every block whose event has completed to the free lists (lock held).
void reclaim_locked() {
  for (size_t i = 0; i < g_deferred.size();) {
    if (cudaEventQuery(g_deferred[i].ev) == cudaErrorNotReady) {
      ++i;
      continue;
    }
    for (auto& b : g_deferred[i].blocks) g_free[b.second].push_back(b.first);
    cudaEventDestroy(g_deferred[i].ev);
    g_deferred[i] = std::move(g_deferred.back());
    g_deferred.pop_back();
  }
}

size_t round_size(size_t b) {
  if (b == 0) b = 1;
  if (b < (1u << 20)) return (b + 255) & ~size_t(255);
  const size_t g = size_t(2) << 20;
  return (b + g - 1) / g * g;
}
}  // namespace

namespace {
// Allocation-failure injection (pt_debug_fail_allocations): allocations left
// before every later one fails; negative = off.
std::atomic<int64_t> g_fail_after{-1};
}  // namespace

void* dev_alloc(size_t bytes) {
  for (int64_t left = g_fail_after.load(); left >= 0;) {
    if (left == 0) return nullptr;
    if (g_fail_after.compare_exchange_weak(left, left - 1)) break;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  const size_t sz = round_size(bytes);
  {
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    if (!g_deferred.empty()) reclaim_locked();
    auto it = g_free.find({dev, sz});
    if (it != g_free.end() && !it->second.empty()) {
      void* p = it->second.back();
      it->second.pop_back();
      g_live[p] = {dev, sz};
      return p;
    }
  }
  void* p = nullptr;
  if (cudaMalloc(&p, sz) != cudaSuccess) {
    cudaGetLastError();  // clear the sticky-free allocation error
    // Give back cached blocks of this device and retry once.
    std::vector<void*> drop;
    {
      std::lock_guard<std::mutex> lk(g_alloc_mu);
      for (auto& kv : g_free)
        if (kv.first.first == dev) {
          drop.insert(drop.end(), kv.second.begin(), kv.second.end());
          kv.second.clear();
        }
    }
    for (void* q : drop) cudaFree(q);
    if (cudaMalloc(&p, sz) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
  }
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  g_live[p] = {dev, sz};
  return p;
}

void dev_free(void* p) {
  if (!p) return;
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  auto it = g_live.find(p);
  if (it == g_live.end()) return;
  g_free[it->second].push_back(p);
  g_live.erase(it);
}

// The blocks become reusable when ev (recorded behind the last work that
// reads them; the cache owns it from here) has completed.
void dev_free_after(const std::vector<void*>& ps, cudaEvent_t ev) {
  std::lock_guard<std::mutex> lk(g_alloc_mu);
  Deferred d{ev, {}};
  for (void* p : ps) {
    auto it = g_live.find(p);
    if (it == g_live.end()) continue;
    d.blocks.push_back({p, it->second});
    g_live.erase(it);
  }
  g_deferred.push_back(std::move(d));
}

bool Buf::ensure(size_t want) {
  if (want <= bytes && p) return true;
  release();
  p = dev_alloc(want);
  if (!p) return false;
  bytes = want;
  return true;
}

void Buf::release() {
  if (p) dev_free(p);
  p = nullptr;
  bytes = 0;
}

namespace {
thread_local std::string t_last_error;
}

void set_error(pt_ctx* ctx, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  t_last_error = msg;
}

void set_thread_error(const std::string& msg) { t_last_error = msg; }

namespace {
std::atomic<int64_t> g_launches{0};
}
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void add_launch_count(int64_t k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
int64_t launch_counter() { return g_launches.load(std::memory_order_relaxed); }

void prof_begin(pt_ctx* ctx) {
  if (!ctx->profile) return;
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!ctx->ev_pool.empty()) {
    ev = ctx->ev_pool.back();
    ctx->ev_pool.pop_back();
  } else {
    cudaEventCreate(&ev.first);
    cudaEventCreate(&ev.second);
  }
  cudaEventRecord(ev.first, ctx->stream);
  ctx->ev_pending.push_back(ev);
}

void prof_end(pt_ctx* ctx) {
  if (!ctx->profile || ctx->ev_pending.empty()) return;
  cudaEventRecord(ctx->ev_pending.back().second, ctx->stream);
}

}  // namespace pt

using pt::set_error;

extern "C" {

void pt_naive_opts_default(pt_naive_opts* o) {
  if (!o) return;
  o->precision = PT_PREC_BF16X3;
  o->two_sided = 0;
  o->accumulate_counts = 0;
}

pt_status pt_prepare(const float* X, int32_t n, int64_t n_grid, const uint8_t* mask, int32_t n1,
                     void* stream, pt_ctx** out) {
  pt::NvtxRange nvtx_range("pt_prepare");
  try {
    if (!out || !X) {
      pt::set_thread_error("pt_prepare: X and out must be non-NULL");
      return PT_ERR_INVALID;
    }
    if (n < 3 || n > 1024 || n1 < 1 || n1 > n - 1 || n_grid < 1 || n_grid >= (int64_t(1) << 31)) {
      pt::set_thread_error("pt_prepare: need 3 <= n <= 1024, 1 <= n1 <= n-1, 1 <= n_grid < 2^31");
      return PT_ERR_INVALID;
    }
    pt_ctx* ctx = new (std::nothrow) pt_ctx();
    if (!ctx) {
      pt::set_thread_error("pt_prepare: out of host memory");
      return PT_ERR_NOMEM;
    }
    cudaGetDevice(&ctx->device);
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->n = n;
    ctx->n1 = n1;
    ctx->n2 = n - n1;
    ctx->n_pad = (n + 15) / 16 * 16;
    ctx->n_grid = n_grid;
    ctx->k = 1.0 / n1 + 1.0 / (n - n1);
    ctx->c_t = std::sqrt(ctx->k * (n - 2));
    pt_status st = pt::prepare_impl(ctx, X, mask);
    if (st != PT_OK) {
      pt::set_thread_error(ctx->last_error);
      pt_destroy(ctx);
      return st;
    }
    *out = ctx;
    return PT_OK;
  } catch (...) {
    pt::set_thread_error("pt_prepare: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_prepare_glm(const float* X, int32_t n, int64_t n_grid, const uint8_t* mask,
                         int32_t n1, const double* Z, int32_t q, void* stream, pt_ctx** out) {
  pt::NvtxRange nvtx_range("pt_prepare_glm");
  try {
    if (!out || !X || q < 0 || q > pt::kGlmMaxQ1 - 1 || (q > 0 && !Z)) {
      pt::set_thread_error("pt_prepare_glm: need X, out non-NULL, 0 <= q <= 16, Z non-NULL if q > 0");
      return PT_ERR_INVALID;
    }
    if (n < 3 || n > 1024 || n1 < 1 || n1 > n - 1 || n_grid < 1 || n_grid >= (int64_t(1) << 31) ||
        n - q - 2 < 1) {
      pt::set_thread_error(
          "pt_prepare_glm: need 3 <= n <= 1024, 1 <= n1 <= n-1, 1 <= n_grid < 2^31, q <= n - 3");
      return PT_ERR_INVALID;
    }
    pt_ctx* ctx = new (std::nothrow) pt_ctx();
    if (!ctx) {
      pt::set_thread_error("pt_prepare_glm: out of host memory");
      return PT_ERR_NOMEM;
    }
    cudaGetDevice(&ctx->device);
    ctx->stream = static_cast<cudaStream_t>(stream);
    ctx->n = n;
    ctx->n1 = n1;
    ctx->n2 = n - n1;
    ctx->n_pad = (n + 15) / 16 * 16;
    ctx->n_grid = n_grid;
    ctx->k = 1.0 / n1 + 1.0 / (n - n1);
    ctx->c_t = std::sqrt(ctx->k * (n - 2));
    pt_status st = pt::glm_setup(ctx, Z, q);
    if (st == PT_OK) st = pt::prepare_impl(ctx, X, mask);
    if (st != PT_OK) {
      pt::set_thread_error(ctx->last_error);
      pt_destroy(ctx);
      return st;
    }
    *out = ctx;
    return PT_OK;
  } catch (...) {
    pt::set_thread_error("pt_prepare_glm: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_maxnull_naive_ex(pt_ctx* ctx, const int32_t* perms, int64_t P,
                              const pt_naive_opts* opts, float* maxnull, int32_t* argmax,
                              uint32_t* counts) {
  pt::NvtxRange nvtx_range("pt_maxnull_naive");
  if (!ctx) {
    pt::set_thread_error("pt_maxnull_naive: ctx is NULL");
    return PT_ERR_INVALID;
  }
  try {
    pt_naive_opts o;
    pt_naive_opts_default(&o);
    if (opts) o = *opts;
    if (!perms || !maxnull || !argmax || P < 1 || P > INT32_MAX) {
      set_error(ctx, "pt_maxnull_naive: need perms, maxnull, argmax non-NULL and 1 <= P < 2^31");
      return PT_ERR_INVALID;
    }
    if (o.precision < PT_PREC_FP32 || o.precision > PT_PREC_FP16X2 || o.two_sided < 0 ||
        o.two_sided > 1 || o.accumulate_counts < 0 || o.accumulate_counts > 1) {
      set_error(ctx, "pt_maxnull_naive: bad options");
      return PT_ERR_INVALID;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      set_error(ctx, "pt_maxnull_naive: cudaSetDevice failed");
      return PT_ERR_CUDA;
    }
    return pt::naive_impl(ctx, perms, P, o, maxnull, argmax, counts);
  } catch (...) {
    set_error(ctx, "pt_maxnull_naive: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_maxnull_naive_batched(pt_ctx* const* ctxs, int32_t n_studies,
                                   const int32_t* const* perms, const int64_t* P,
                                   const pt_naive_opts* opts, float* const* maxnull,
                                   int32_t* const* argmax, uint32_t* const* counts) {
  pt::NvtxRange nvtx_range("pt_maxnull_naive_batched");
  if (!ctxs || n_studies < 1 || n_studies > 4096 || !perms || !P || !maxnull || !argmax) {
    pt::set_thread_error(
        "pt_maxnull_naive_batched: need 1 <= n_studies <= 4096 and non-NULL arrays");
    return PT_ERR_INVALID;
  }
  pt_ctx* lead = ctxs[0];
  try {
    pt_naive_opts o;
    pt_naive_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision < PT_PREC_FP32 || o.precision > PT_PREC_FP16X2 || o.two_sided < 0 ||
        o.two_sided > 1 || o.accumulate_counts < 0 || o.accumulate_counts > 1) {
      pt::set_thread_error("pt_maxnull_naive_batched: bad options");
      return PT_ERR_INVALID;
    }
    for (int32_t i = 0; i < n_studies; ++i) {
      if (!ctxs[i] || !perms[i] || !maxnull[i] || !argmax[i] || P[i] < 1 || P[i] > INT32_MAX) {
        pt::set_thread_error("pt_maxnull_naive_batched: study " + std::to_string(i) +
                             ": need ctx, perms, maxnull, argmax non-NULL and 1 <= P < 2^31");
        return PT_ERR_INVALID;
      }
      for (int32_t j = 0; j < i; ++j)
        if (ctxs[j] == ctxs[i]) {
          pt::set_thread_error("pt_maxnull_naive_batched: a context appears twice");
          return PT_ERR_INVALID;
        }
    }
    if (cudaSetDevice(lead->device) != cudaSuccess) {
      set_error(lead, "pt_maxnull_naive_batched: cudaSetDevice failed");
      return PT_ERR_CUDA;
    }
    const pt_status s =
        pt::naive_batched_impl(ctxs, n_studies, perms, P, o, maxnull, argmax, counts);
    if (s != PT_OK) pt::set_thread_error(lead->last_error);
    return s;
  } catch (...) {
    set_error(lead, "pt_maxnull_naive_batched: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_maxnull_naive(pt_ctx* ctx, const int32_t* perms, int64_t P, float* maxnull,
                           int32_t* argmax, uint32_t* counts) {
  return pt_maxnull_naive_ex(ctx, perms, P, nullptr, maxnull, argmax, counts);
}

pt_status pt_fwer_pvalues(pt_ctx* ctx, const float* maxnull, int64_t P, int32_t two_sided,
                          float* p_out) {
  pt::NvtxRange nvtx_range("pt_fwer_pvalues");
  if (!ctx) {
    pt::set_thread_error("pt_fwer_pvalues: ctx is NULL");
    return PT_ERR_INVALID;
  }
  if (!maxnull || !p_out || P < 1 || two_sided < 0 || two_sided > 1) {
    set_error(ctx, "pt_fwer_pvalues: need maxnull, p_out non-NULL, P >= 1, two_sided 0 or 1");
    return PT_ERR_INVALID;
  }
  try {
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      set_error(ctx, "pt_fwer_pvalues: cudaSetDevice failed");
      return PT_ERR_CUDA;
    }
    return pt::fwer_pvalues_impl(ctx, maxnull, P, two_sided, p_out);
  } catch (...) {
    set_error(ctx, "pt_fwer_pvalues: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_sync(pt_ctx* ctx) {
  if (!ctx) {
    pt::set_thread_error("pt_sync: ctx is NULL");
    return PT_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  PT_CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  uint32_t bits = 0;
  PT_CUDA_TRY(ctx, cudaMemcpy(&bits, ctx->status.p, sizeof(bits), cudaMemcpyDeviceToHost));
  if (bits) {
    PT_CUDA_TRY(ctx, cudaMemset(ctx->status.p, 0, sizeof(uint32_t)));
    if (bits & pt::kErrTimeout) {
      set_error(ctx, "a bounded device-side wait expired");
      return PT_ERR_TIMEOUT;
    }
    if (bits & pt::kErrBadPerm) {
      set_error(ctx, "a relabelling row is not a permutation of 0..n-1");
      return PT_ERR_INVALID;
    }
    if (bits & pt::kErrGlmSpan) {
      set_error(ctx, "a relabelled group column lies in the span of the covariates");
      return PT_ERR_INVALID;
    }
    set_error(ctx, "invalid input data (NaN or Inf)");
    return PT_ERR_INVALID;
  }
  return PT_OK;
}

pt_status pt_t_obs(pt_ctx* ctx, float* t_obs);  // defined in pt_prepare.cu

pt_status pt_voxel_grid_index(pt_ctx* ctx, int64_t* grid_index) {
  if (!ctx || !grid_index) {
    set_error(ctx, "pt_voxel_grid_index: NULL argument");
    return PT_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  PT_CUDA_TRY(ctx, cudaMemcpyAsync(grid_index, ctx->vox_grid.p, sizeof(int64_t) * ctx->v,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
  return PT_OK;
}

int64_t pt_num_voxels(const pt_ctx* ctx) { return ctx ? ctx->v : -1; }
int64_t pt_num_valid_voxels(const pt_ctx* ctx) { return ctx ? ctx->v_valid : -1; }

const char* pt_last_error(const pt_ctx* ctx) {
  if (ctx) return ctx->last_error.c_str();
  return pt::t_last_error.c_str();
}

pt_status pt_profile_enable(pt_ctx* ctx, int32_t on) {
  if (!ctx) {
    pt::set_thread_error("pt_profile_enable: ctx is NULL");
    return PT_ERR_INVALID;
  }
  ctx->profile = on != 0;
  return PT_OK;
}

pt_status pt_profile_read(pt_ctx* ctx, double* total_ms, int64_t* launches) {
  if (!ctx || !total_ms || !launches) {
    set_error(ctx, "pt_profile_read: NULL argument");
    return PT_ERR_INVALID;
  }
  cudaSetDevice(ctx->device);
  // Waits for the last timed launch only (later work on the stream may run on).
  if (!ctx->ev_pending.empty())
    PT_CUDA_TRY(ctx, cudaEventSynchronize(ctx->ev_pending.back().second));
  double tot = 0.0;
  for (auto& ev : ctx->ev_pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev.first, ev.second) == cudaSuccess) tot += ms;
    ctx->ev_pool.push_back(ev);
  }
  *total_ms = tot;
  *launches = int64_t(ctx->ev_pending.size());
  ctx->ev_pending.clear();
  return PT_OK;
}

int64_t pt_kernel_launch_count(void) { return pt::g_launches.load(); }

void pt_debug_fail_allocations(int64_t after) { pt::g_fail_after.store(after < 0 ? -1 : after); }

pt_status pt_debug_device_reset(void) {
  const cudaError_t e = cudaDeviceReset();
  if (e != cudaSuccess) {
    pt::set_thread_error(std::string("cudaDeviceReset: ") + cudaGetErrorString(e));
    return PT_ERR_CUDA;
  }
  return PT_OK;
}

// Does not wait for the context's queued work: its workspaces go back to the
// cache behind an event recorded on its stream and are handed out again once
// that work has finished. A context that took part in a captured batch (whose
// graph runs on the lead context's stream) is waited for instead.
void pt_destroy(pt_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  const bool member = pt::batch_forget(ctx);
  for (auto& ev : ctx->ev_pending) ctx->ev_pool.push_back(ev);
  for (auto& ev : ctx->ev_pool) {  // released by the runtime once recorded work completes
    cudaEventDestroy(ev.first);
    cudaEventDestroy(ev.second);
  }
  pt::Buf* bufs[] = {&ctx->status,  &ctx->vox_grid, &ctx->valid_map, &ctx->t_obs64,
                     &ctx->Xraw,    &ctx->vstat,    &ctx->u_obs,     &ctx->Xn32,
                     &ctx->Xnb,     &ctx->labels,   &ctx->rowflag,   &ctx->blockflag,
                     &ctx->maxkey,  &ctx->cnt,      &ctx->scratch,   &ctx->tcdesc,
                     &ctx->moments, &ctx->glmQ,     &ctx->glm_coef,  &ctx->glm_inv,
                     &ctx->rowscale, &ctx->grid_inv};
  cudaEvent_t done = nullptr;
  if (!member && cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess &&
      cudaEventRecord(done, ctx->stream) == cudaSuccess) {
    std::vector<void*> ps;
    for (pt::Buf* b : bufs) {
      if (b->p) ps.push_back(b->p);
      b->p = nullptr;
      b->bytes = 0;
    }
    pt::dev_free_after(ps, done);
  } else {
    if (done) cudaEventDestroy(done);
    if (member) cudaDeviceSynchronize();
    else cudaStreamSynchronize(ctx->stream);
    for (pt::Buf* b : bufs) b->release();
  }
  delete ctx;
}

void pt_release_cached_memory(void) {
  std::vector<void*> drop;
  {
    std::lock_guard<std::mutex> lk(pt::g_alloc_mu);
    for (auto& d : pt::g_deferred) {  // blocks of destroyed contexts: after their work
      cudaEventSynchronize(d.ev);
      cudaEventDestroy(d.ev);
      for (auto& b : d.blocks) drop.push_back(b.first);
    }
    pt::g_deferred.clear();
    for (auto& kv : pt::g_free) {
      drop.insert(drop.end(), kv.second.begin(), kv.second.end());
      kv.second.clear();
    }
  }
  for (void* q : drop) cudaFree(q);
}

}  // extern "C"
