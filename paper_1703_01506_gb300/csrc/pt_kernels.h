// Device helpers (inline PTX for sm_103a: mbarrier, TMA, tcgen05) and the
// host-side launchers shared between translation units.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "pt_internal.h"

namespace pt {

// ---- packed (value, index) keys: larger value wins, then smaller index ----
__device__ __forceinline__ uint32_t orderable_bits(float f) {
  const uint32_t u = __float_as_uint(f);
  return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float from_orderable_bits(uint32_t o) {
  const uint32_t u = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
  return __uint_as_float(u);
}
__device__ __forceinline__ unsigned long long pack_key(float value, uint32_t index) {
  return (static_cast<unsigned long long>(orderable_bits(value)) << 32) |
         static_cast<unsigned long long>(~index);
}
__device__ __forceinline__ float unpack_key_value(unsigned long long key) {
  return from_orderable_bits(static_cast<uint32_t>(key >> 32));
}
__device__ __forceinline__ uint32_t unpack_key_index(unsigned long long key) {
  return ~static_cast<uint32_t>(key & 0xffffffffull);
}

// ---- float-float arithmetic (an unevaluated pair h + l, ~44 significant bits) ----
// s + e = a + b exactly (Knuth's branch-free two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// (h, l) += (bh, bl), renormalised so that |l| <= ulp(h)/2.
__device__ __forceinline__ void ff_acc(float& h, float& l, float bh, float bl) {
  float s, e;
  two_sum(h, bh, s, e);
  e += l + bl;
  h = s + e;
  l = e - (h - s);
}

__device__ __forceinline__ double ff_d(float h, float l) { return double(h) + double(l); }

// B = u^T W u for the F of a g-group factor: u and W (FG x FG, row-major,
// zero-padded past g - 1) in a fixed order of FMAs, so that the fused kernel
// and the observed statistic's kernel round identically.
template <int FG>
__device__ __forceinline__ float f_quad(const float (&u)[FG], const float* W) {
  float bq = 0.0f;
#pragma unroll
  for (int m = 0; m < FG; ++m) {
    float t = 0.0f;
#pragma unroll
    for (int m2 = 0; m2 < FG; ++m2) t = fmaf(W[m * FG + m2], u[m2], t);
    bq = fmaf(u[m], t, bq);
  }
  return bq;
}

// ---- bounded waits ----
// Every spin-wait in this library gives up after kWaitLimitNs of wall time,
// records kErrTimeout in the context's status word and returns false.
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// A thread whose phase is not complete sleeps in try_wait until the phase
// completes or kSuspendHintNs pass: waiting warps do not keep polling the
// barrier's shared-memory word while the tensor core streams operands.
constexpr uint32_t kSuspendHintNs = 20000u;
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(kSuspendHintNs)
      : "memory");
  return ok != 0;
}
// Waits for the phase with the given parity to complete. Returns false (after
// recording a timeout, or at once if *abort is set) when it gives up.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, uint32_t* status,
                                          volatile int* abort_flag,
                                          unsigned long long limit_ns = kWaitLimitNs,
                                          bool honour_abort = true) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 63u) == 0) {
      if (honour_abort && *abort_flag) return false;
      if (globaltimer_ns() - t0 > limit_ns) {
        atomicOr(status, kErrTimeout);
        *abort_flag = 1;
        return false;
      }
    }
  }
}

// ---- TMA (bulk tensor copy, global -> shared, completes on an mbarrier) ----
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int32_t c0, int32_t c1,
                                            uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(c0), "r"(c1), "r"(bar)
      : "memory");
}

// ---- tcgen05 ----
__device__ __forceinline__ void tmem_alloc(uint32_t dst_slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(dst_slot),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// D[tmem] (+)= A[smem desc] * B[smem desc]^T, kind::f16 (BF16 in, FP32 accumulate).
__device__ __forceinline__ void tc_mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                           uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// Arrive (once) on an mbarrier when all previously issued tcgen05 ops of this thread complete.
__device__ __forceinline__ void tc_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
      : "memory");
}
__device__ __forceinline__ void tc_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// 32 lanes x 32 consecutive 32-bit columns: thread t of the warp gets lane (base+t).
__device__ __forceinline__ void tc_ld_32x32b_x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
}

__device__ __forceinline__ void tc_ld_32x32b_x8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                 "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
}

__device__ __forceinline__ void tc_ld_32x32b_x16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}

// Shared-memory matrix descriptor, no swizzle, K-major operand stored as
// 8x8 (rows x 16-byte) core matrices: lbo = byte step between core matrices
// adjacent in K, sbo = byte step between adjacent 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= uint64_t((addr >> 4) & 0x3FFFu);
  d |= uint64_t((lbo >> 4) & 0x3FFFu) << 16;
  d |= uint64_t((sbo >> 4) & 0x3FFFu) << 32;
  d |= uint64_t(1) << 46;  // descriptor version for tcgen05
  return d;                 // base offset 0, absolute LBO mode, swizzle none (bits 61-63 = 0)
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// Same with A = B = F16 (type fields 0): both operands of one MMA share a type.
__host__ __device__ constexpr uint32_t idesc_f16_f32(int M, int N) {
  return (1u << 4) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

// ---- TMA descriptors (pt_naive_tc.cu) ----
// 2D view [rows][256] of a BF16 buffer, box [box_rows][256], no swizzle;
// false if the driver entry point is missing or rejects the view.
bool make_map(CUtensorMap* m, const void* base, uint64_t rows, uint32_t box_rows);

// ---- launchers implemented in pt_naive_tc.cu ----
pt_status tc_supported(pt_ctx* ctx);
// Fused contraction + max / count reduction over P relabellings (labels from
// build_labels, layout 1); rowflag/blockflag from the labels kernel.
pt_status tc_reduce(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int two_sided,
                    const float* u_obs, unsigned long long* maxkey, uint32_t* cnt);
// Same contraction writing rows: write_mode 1 -> u, 2 -> t (optionally also
// reducing); 3 -> one bit per entry, u >= uthr, or-ed into rows of
// (v + 31) / 32 uint32 words at out (zeroed by the caller; no reduction).
pt_status tc_rows(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int write_mode,
                  float* out, int do_reduce, int two_sided, const float* u_obs,
                  unsigned long long* maxkey, uint32_t* cnt, float uthr = 0.0f);

// Several studies in one persistent launch per tile class. tc_batch_plan
// encodes every study's tensor maps and work split (labels and workspaces of
// every context already allocated) and uploads them; tc_batch_launch enqueues
// one fused launch per tile class on lead->stream and can be graph-captured.
struct TcGroup {
  int NT, first, count, n_pad_max;
  int64_t items;
  int stages, kps;  // label ring: stages of kps k-steps
};
pt_status tc_batch_plan(pt_ctx* lead, pt_ctx* const* ctxs, const int64_t* P, int n,
                        const pt_naive_opts& o, Buf& descbuf, std::vector<char>& host_desc,
                        std::vector<TcGroup>& groups);
pt_status tc_batch_launch(pt_ctx* lead, const Buf& descbuf, const std::vector<TcGroup>& groups,
                          int precision, int two_sided);

// ---- launch configuration of the fused kernel (pt_naive_tc.cu) ----
// Label-ring stages of kps k-steps that fit beside a resident tile of NT voxels (0: none).
int tc_max_stages(int NT, int n_pad, int pieces, int kps);
// Configuration used when none is recorded: the largest voxel tile that fits,
// the largest stage of which two fit (8, 4, 2 or 1 k-steps), a ring of about
// 16 k-steps, 8 work items per SM. false if no tile fits.
bool tc_default_config(int n_pad, int pieces, pt_tc_config* out);
bool tc_config_valid(const pt_tc_config& c, int n_pad, int pieces);
struct TcTrial {
  pt_tc_config cfg;
  double ms;
};
// Times the candidate configurations of the reduce-only launch on ctx's
// problem (labels in Lb, operand pieces built, maxkey/cnt sized for P).
pt_status tc_autotune(pt_ctx* ctx, const void* Lb, int64_t P, int precision, int two_sided,
                      pt_tc_config* best, double* best_ms, std::vector<TcTrial>* trials);

// ---- table of tuned configurations (pt_tune.cu) ----
// Overwrites *cfg and returns true when a configuration is recorded for this
// shape (padded n, precision, sidedness, voxel and relabelling counts).
bool tune_find(int n_pad, int precision, int two_sided, int64_t v, int64_t P, pt_tc_config* cfg);

// ---- shared with pt_naive.cu ----
pt_status build_labels(pt_ctx* ctx, const int32_t* perms, int64_t P, int layout,
                       int64_t* P_pad_out);

}  // namespace pt
