// The random numbers of RapidPT on the device: Philox4x32-10 (Salmon, Moraes,
// Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC 2011) keyed by
// the 64-bit seed, counters (a, b, c, tag), and the draws built on its words:
//   normal        Box-Muller from words (x0, x1): u1 = (x0 + 1) 2^-32 in (0, 1],
//                 u2 = x1 2^-32, z = sqrt(-2 ln u1) cos(2 pi u2);
//   voxel noise   one counter (floor(j / 4), b, 0, tag) serves voxels 4p .. 4p + 3:
//                 words (x0, x1) the Box-Muller pair of 4p, 4p + 1 and (x2, x3)
//                 that of 4p + 2, 4p + 3 (cos for the even, sin for the odd voxel);
//   index         floor((x1 2^32 + x0) v / 2^64), uniform on [0, v).
// Every |z| is at most sqrt(-2 ln 2^-32) = 6.66035...
#pragma once
#include <cstdint>

namespace pt {

constexpr uint32_t TAG_U0 = 1, TAG_TRAIN = 2, TAG_REC = 3, TAG_NOISE = 4, TAG_SHIFT = 5;
constexpr float kNoiseBound = 6.6604f;  // sqrt(-2 ln 2^-32) rounded up: |z| of every draw
constexpr float kTwoPow32Inv = 2.3283064365386963e-10f;

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

// u1 in (0, 1] from the first word of a Box-Muller pair.
__device__ __forceinline__ float bm_u1(uint32_t w) {
  return fmaf(__uint2float_rn(w), kTwoPow32Inv, kTwoPow32Inv);
}

__device__ __forceinline__ float draw_normal(uint32_t k0, uint32_t k1, uint32_t tag, uint32_t a,
                                             uint32_t b) {
  const uint4 o = philox(make_uint4(a, b, 0u, tag), k0, k1);
  const float u2 = __uint2float_rn(o.y) * kTwoPow32Inv;
  return sqrtf(-2.0f * logf(bm_u1(o.x))) * cospif(2.0f * u2);
}

// The Box-Muller pair of words (wa, wb): r cos(2 pi u2) for the even voxel,
// r sin(2 pi u2) for the odd one.
__device__ __forceinline__ void bm_pair(uint32_t wa, uint32_t wb, float& z_even, float& z_odd) {
  const float r = sqrtf(-2.0f * logf(bm_u1(wa)));
  float sv, cv;
  sincospif(2.0f * (__uint2float_rn(wb) * kTwoPow32Inv), &sv, &cv);
  z_even = r * cv;
  z_odd = r * sv;
}

__device__ __forceinline__ uint32_t draw_index(uint32_t k0, uint32_t k1, uint32_t tag, uint32_t q,
                                               uint32_t i, uint32_t p, uint32_t V) {
  const uint4 o = philox(make_uint4(q, i, p, tag), k0, k1);
  const unsigned long long t =
      (unsigned long long)o.y * V + (((unsigned long long)o.x * V) >> 32);
  return uint32_t(t >> 32);
}

}  // namespace pt
