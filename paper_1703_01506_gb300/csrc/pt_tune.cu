// Autotuner of the fused tensor-core NaivePT kernel: the process-wide table of
// tuned launch configurations, the entry points that fill it by timing, and
// its text file format.
//
// A configuration only changes how the work is staged and cut (label-ring
// shape, relabelling blocks per work item; the voxel tile is fixed by n);
// every T entry is accumulated over the same k-steps and data pieces in the
// same order whatever the configuration, so the outputs do not depend on it.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "pt_internal.h"
#include "pt_kernels.h"

namespace pt {
namespace {

struct Key {
  int n_pad, precision, two_sided, vb, pb;
  bool operator<(const Key& o) const {
    return std::tie(n_pad, precision, two_sided, vb, pb) <
           std::tie(o.n_pad, o.precision, o.two_sided, o.vb, o.pb);
  }
};
struct Entry {
  pt_tc_config cfg;
  double ms;
};

std::mutex g_mu;
std::map<Key, Entry> g_table;

// Half-octave buckets: voxel or relabelling counts within a factor of about
// 1.41 of each other share an entry.
int bucket(int64_t x) { return x < 1 ? 0 : int(std::floor(2.0 * std::log2(double(x)))); }

int pad16(int n) { return (n + 15) / 16 * 16; }

Key make_key(int n_pad, int precision, int two_sided, int64_t v, int64_t P) {
  return Key{n_pad, precision, two_sided, bucket(v), bucket(P)};
}

void put(const Key& k, const pt_tc_config& c, double ms) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_table[k] = Entry{c, ms};
}

const char kHeader[] = "# pt tuned launch configurations v2";

pt_status tune_one(pt_ctx* ctx, const int32_t* perms, int64_t P, const pt_naive_opts& o,
                   pt_tc_config* chosen, double* chosen_ms) {
  pt_status s = tc_supported(ctx);
  if (s != PT_OK) return s;
  const int pieces = prec_pieces(o.precision);
  pt_tc_config best;
  if (!tc_default_config(ctx->n_pad, pieces, &best)) {
    set_error(ctx, "tensor-core path: n too large for the resident data tile");
    return PT_ERR_UNSUPPORTED;
  }
  double best_ms = 0.0;
  if (ctx->v_valid > 0) {
    if (!ctx->maxkey.ensure(sizeof(unsigned long long) * P) ||
        !ctx->cnt.ensure(sizeof(uint32_t) * (ctx->v_valid + 1))) {
      set_error(ctx, "out of device memory (workspace)");
      return PT_ERR_NOMEM;
    }
    PT_CUDA_TRY(ctx, cudaMemsetAsync(ctx->cnt.p, 0, sizeof(uint32_t) * (ctx->v_valid + 1),
                                     ctx->stream));
    int64_t P_pad = 0;
    s = build_labels(ctx, perms, P, prec_label_layout(o.precision), &P_pad);
    if (s == PT_OK) s = ensure_xnb(ctx, o.precision);
    if (s == PT_OK) s = tc_autotune(ctx, ctx->labels.p, P, o.precision, o.two_sided, &best,
                                    &best_ms, nullptr);
    if (s != PT_OK) return s;
    s = pt_sync(ctx);  // a bad relabelling row or an expired wait voids the timings
    if (s != PT_OK) return s;
    put(make_key(ctx->n_pad, o.precision, o.two_sided, ctx->v_valid, P), best, best_ms);
  }
  if (chosen) *chosen = best;
  if (chosen_ms) *chosen_ms = best_ms;
  return PT_OK;
}

bool opts_ok(const pt_naive_opts& o) {
  return (o.precision == PT_PREC_BF16X2 || o.precision == PT_PREC_BF16X3 ||
          o.precision == PT_PREC_FP16X2) &&
         (o.two_sided == 0 || o.two_sided == 1);
}

}  // namespace

bool tune_find(int n_pad, int precision, int two_sided, int64_t v, int64_t P, pt_tc_config* cfg) {
  std::lock_guard<std::mutex> lk(g_mu);
  auto it = g_table.find(make_key(n_pad, precision, two_sided, v, P));
  if (it == g_table.end()) return false;
  *cfg = it->second.cfg;
  return true;
}

}  // namespace pt

extern "C" {

pt_status pt_autotune_naive(pt_ctx* ctx, const int32_t* perms, int64_t P,
                            const pt_naive_opts* opts, pt_tc_config* chosen, double* chosen_ms) {
  pt::NvtxRange nvtx_range("pt_autotune_naive");
  if (!ctx) {
    pt::set_thread_error("pt_autotune_naive: ctx is NULL");
    return PT_ERR_INVALID;
  }
  try {
    pt_naive_opts o;
    pt_naive_opts_default(&o);
    if (opts) o = *opts;
    if (!perms || P < 1 || P > INT32_MAX || !pt::opts_ok(o)) {
      pt::set_error(ctx,
                    "pt_autotune_naive: need perms non-NULL, 1 <= P < 2^31 and a tensor-core "
                    "precision (BF16X2, BF16X3 or FP16X2)");
      return PT_ERR_INVALID;
    }
    if (cudaSetDevice(ctx->device) != cudaSuccess) {
      pt::set_error(ctx, "pt_autotune_naive: cudaSetDevice failed");
      return PT_ERR_CUDA;
    }
    return pt::tune_one(ctx, perms, P, o, chosen, chosen_ms);
  } catch (...) {
    pt::set_error(ctx, "pt_autotune_naive: internal error");
    return PT_ERR_CUDA;
  }
}

pt_status pt_autotune_naive_batched(pt_ctx* const* ctxs, int32_t n_studies,
                                    const int32_t* const* perms, const int64_t* P,
                                    const pt_naive_opts* opts) {
  pt::NvtxRange nvtx_range("pt_autotune_naive_batched");
  if (!ctxs || n_studies < 1 || n_studies > 4096 || !perms || !P) {
    pt::set_thread_error("pt_autotune_naive_batched: need 1 <= n_studies <= 4096 and arrays");
    return PT_ERR_INVALID;
  }
  try {
    pt_naive_opts o;
    pt_naive_opts_default(&o);
    if (opts) o = *opts;
    if (!pt::opts_ok(o)) {
      pt::set_thread_error("pt_autotune_naive_batched: needs a tensor-core precision");
      return PT_ERR_INVALID;
    }
    for (int32_t i = 0; i < n_studies; ++i)
      if (!ctxs[i] || !perms[i] || P[i] < 1 || P[i] > INT32_MAX) {
        pt::set_thread_error("pt_autotune_naive_batched: study " + std::to_string(i) +
                             ": need ctx, perms non-NULL and 1 <= P < 2^31");
        return PT_ERR_INVALID;
      }
    // One tuning run per distinct shape key, on the first study that has it.
    std::map<pt::Key, int> seen;
    for (int32_t i = 0; i < n_studies; ++i) {
      pt_ctx* c = ctxs[i];
      const pt::Key k = pt::make_key(c->n_pad, o.precision, o.two_sided, c->v_valid, P[i]);
      if (seen.count(k)) continue;
      seen[k] = i;
      if (cudaSetDevice(c->device) != cudaSuccess) {
        pt::set_thread_error("pt_autotune_naive_batched: cudaSetDevice failed");
        return PT_ERR_CUDA;
      }
      const pt_status s = pt::tune_one(c, perms[i], P[i], o, nullptr, nullptr);
      if (s != PT_OK) {
        pt::set_thread_error("pt_autotune_naive_batched: study " + std::to_string(i) + ": " +
                             c->last_error);
        return s;
      }
    }
    pt::batch_drop_graph();  // the next batched call plans with the new table
    return PT_OK;
  } catch (...) {
    pt::set_thread_error("pt_autotune_naive_batched: internal error");
    return PT_ERR_CUDA;
  }
}

int32_t pt_tune_lookup(int32_t n, int32_t precision, int32_t two_sided, int64_t v, int64_t P,
                       pt_tc_config* out) {
  if (!out || n < 3 || n > 1024 || v < 1 || P < 1 || precision < PT_PREC_BF16X2 ||
      precision > PT_PREC_FP16X2 || two_sided < 0 || two_sided > 1)
    return -1;
  const int n_pad = pt::pad16(n);
  const int pieces = pt::prec_pieces(precision);
  if (!pt::tc_default_config(n_pad, pieces, out)) return -1;
  return pt::tune_find(n_pad, precision, two_sided, v, P, out) ? 1 : 0;
}

pt_status pt_tune_set(int32_t n, int32_t precision, int32_t two_sided, int64_t v, int64_t P,
                      const pt_tc_config* cfg) {
  if (!cfg || n < 3 || n > 1024 || v < 1 || P < 1 || precision < PT_PREC_BF16X2 ||
      precision > PT_PREC_FP16X2 || two_sided < 0 || two_sided > 1) {
    pt::set_thread_error("pt_tune_set: bad shape or options");
    return PT_ERR_INVALID;
  }
  const int n_pad = pt::pad16(n);
  if (!pt::tc_config_valid(*cfg, n_pad, pt::prec_pieces(precision))) {
    pt::set_thread_error("pt_tune_set: configuration does not fit this n (voxel_tile as n "
                         "fixes it, ksteps_per_stage 1/2/4/8, 2 <= stages <= what fits, "
                         "1 <= items_per_sm <= 64)");
    return PT_ERR_INVALID;
  }
  pt::put(pt::make_key(n_pad, precision, two_sided, v, P), *cfg, 0.0);
  pt::batch_drop_graph();
  return PT_OK;
}

pt_status pt_tune_save(const char* path) {
  if (!path) {
    pt::set_thread_error("pt_tune_save: path is NULL");
    return PT_ERR_INVALID;
  }
  std::vector<std::pair<pt::Key, pt::Entry>> rows;
  {
    std::lock_guard<std::mutex> lk(pt::g_mu);
    rows.assign(pt::g_table.begin(), pt::g_table.end());
  }
  FILE* f = std::fopen(path, "w");
  if (!f) {
    pt::set_thread_error(std::string("pt_tune_save: cannot open ") + path);
    return PT_ERR_INVALID;
  }
  std::fprintf(f, "%s\n# n_pad precision two_sided v_bucket P_bucket voxel_tile stages "
                  "ksteps_per_stage items_per_sm ms\n", pt::kHeader);
  for (const auto& r : rows)
    std::fprintf(f, "%d %d %d %d %d %d %d %d %d %.6f\n", r.first.n_pad, r.first.precision,
                 r.first.two_sided, r.first.vb, r.first.pb, r.second.cfg.voxel_tile,
                 r.second.cfg.stages, r.second.cfg.ksteps_per_stage, r.second.cfg.items_per_sm,
                 r.second.ms);
  const bool ok = std::fclose(f) == 0;
  if (!ok) {
    pt::set_thread_error(std::string("pt_tune_save: write failed: ") + path);
    return PT_ERR_INVALID;
  }
  return PT_OK;
}

pt_status pt_tune_load(const char* path) {
  if (!path) {
    pt::set_thread_error("pt_tune_load: path is NULL");
    return PT_ERR_INVALID;
  }
  FILE* f = std::fopen(path, "r");
  if (!f) {
    pt::set_thread_error(std::string("pt_tune_load: cannot open ") + path);
    return PT_ERR_INVALID;
  }
  std::vector<std::pair<pt::Key, pt::Entry>> rows;
  char line[512];
  int lineno = 0;
  bool header = false;
  std::string err;
  while (std::fgets(line, sizeof line, f)) {
    ++lineno;
    if (lineno == 1) {
      header = std::strncmp(line, pt::kHeader, sizeof(pt::kHeader) - 1) == 0;
      if (!header) {
        err = "not a pt tuning file (first line)";
        break;
      }
      continue;
    }
    if (line[0] == '#' || line[0] == '\n') continue;
    pt::Key k;
    pt::Entry e;
    if (std::sscanf(line, "%d %d %d %d %d %d %d %d %d %lf", &k.n_pad, &k.precision,
                    &k.two_sided, &k.vb, &k.pb, &e.cfg.voxel_tile, &e.cfg.stages,
                    &e.cfg.ksteps_per_stage, &e.cfg.items_per_sm, &e.ms) != 10 ||
        k.n_pad < 16 || k.n_pad % 16 != 0 || k.n_pad > 1024 || k.precision < PT_PREC_BF16X2 ||
        k.precision > PT_PREC_FP16X2 || k.two_sided < 0 || k.two_sided > 1 ||
        !pt::tc_config_valid(e.cfg, k.n_pad, pt::prec_pieces(k.precision))) {
      err = "malformed or invalid entry on line " + std::to_string(lineno);
      break;
    }
    rows.push_back({k, e});
  }
  std::fclose(f);
  if (!header && err.empty()) err = "empty file";
  if (!err.empty()) {
    pt::set_thread_error(std::string("pt_tune_load: ") + path + ": " + err);
    return PT_ERR_INVALID;
  }
  {
    std::lock_guard<std::mutex> lk(pt::g_mu);
    for (const auto& r : rows) pt::g_table[r.first] = r.second;
  }
  pt::batch_drop_graph();
  return PT_OK;
}

void pt_tune_clear(void) {
  {
    std::lock_guard<std::mutex> lk(pt::g_mu);
    pt::g_table.clear();
  }
  pt::batch_drop_graph();
}

}  // extern "C"
