// Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11):
// ten rounds, each multiplying counter words 0 and 2 by the Philox constants,
// exchanging product halves with words 1 and 3 and xoring the key, with the key
// advanced by the Weyl constants between rounds. Plus the uniform / normal
// conversions of the library's counter layout:
//   key = (seed mod 2^32, (seed >> 32) ^ stream_id)
//   counter = (kind << 24 | step, sub, particle, block).
#pragma once
#include "common.cuh"

namespace phi4 {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u, kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u, kPhiloxW1 = 0xBB67AE85u;

enum : uint32_t { RNG_INIT = 1, RNG_RESAMPLE = 2, RNG_PROPOSE = 3, RNG_ACCEPT = 4,
                  RNG_NS_START = 5, RNG_NS_DIRECTION = 6, RNG_NS_SLICE = 7, RNG_FLIP = 8 };

struct PhiloxKey { uint32_t k0, k1; };

__host__ __device__ __forceinline__ PhiloxKey philox_key(uint64_t seed, uint64_t stream_id) {
  return PhiloxKey{(uint32_t)(seed & 0xffffffffu), (uint32_t)((seed >> 32) ^ stream_id)};
}
__host__ __device__ __forceinline__ uint32_t counter_word0(uint32_t kind, uint32_t step) {
  return (kind << 24) | (step & 0xffffffu);
}

PHI4_DEV uint4 philox4x32_10(uint4 c, PhiloxKey k) {
  uint32_t k0 = k.k0, k1 = k.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
    const uint32_t hi0 = __umulhi(kPhiloxM0, c.x), lo0 = kPhiloxM0 * c.x;
    const uint32_t hi1 = __umulhi(kPhiloxM1, c.z), lo1 = kPhiloxM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

// Host twin used only for scalar words the host needs (e.g. launch-time offsets).
inline uint4 philox4x32_10_host(uint4 c, PhiloxKey k) {
  uint32_t k0 = k.k0, k1 = k.k1;
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += kPhiloxW0; k1 += kPhiloxW1; }
    const uint64_t p0 = (uint64_t)kPhiloxM0 * c.x, p1 = (uint64_t)kPhiloxM1 * c.z;
    c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ k0, (uint32_t)p1, (uint32_t)(p0 >> 32) ^ c.w ^ k1, (uint32_t)p0);
  }
  return c;
}

// Box-Muller on two 32-bit words, double precision: u1 in (0,1], u2 in [0,1).
PHI4_DEV double2 box_muller_f64(uint32_t a, uint32_t b) {
  const double u1 = ((double)a + 1.0) * 0x1p-32;
  const double u2 = (double)b * 0x1p-32;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  return make_double2(r * c, r * s);
}

// Box-Muller on the top 24 bits of two words, single precision.
PHI4_DEV float2 box_muller_f32(uint32_t a, uint32_t b) {
  const float u1 = (float)((a >> 8) + 1u) * 0x1p-24f;
  const float u2 = (float)(b >> 8) * 0x1p-24f;
  const float r = sqrtf(-2.0f * logf(u1));
  float s, c;
  sincospif(2.0f * u2, &s, &c);
  return make_float2(r * c, r * s);
}

// 53-bit uniform in (0, 1] from two words: x = (w0 << 21) | (w1 >> 11), u = (x+1) 2^-53.
PHI4_DEV double uniform53(uint32_t w0, uint32_t w1) {
  const uint64_t x = ((uint64_t)w0 << 21) | (uint64_t)(w1 >> 11);
  return (double)(x + 1ull) * 0x1p-53;
}

}  // namespace phi4
