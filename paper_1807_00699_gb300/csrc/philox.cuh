// Counter-based normal deviates for the noise term of Eq. (2).
//
// Philox4x32-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random
// numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64-bit
// multiplies, with the key bumped by two Weyl constants between rounds.
// Uniforms use the top 23 bits plus one half ulp, so they are exact in FP32
// and never 0 or 1; normals come from Box-Muller on word pairs.
#pragma once
#include <cstdint>

namespace gda {

struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

__device__ __forceinline__ float philox_u01(uint32_t x) {
  return (float(x >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// Four N(0,1) deviates for counter (c0, c1, c2, c3) under a 64-bit key.
__device__ __forceinline__ void philox_normal4(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint64_t seed, float z[4]) {
  const U4 o = philox4x32_10(U4{c0, c1, c2, c3}, uint32_t(seed), uint32_t(seed >> 32));
  float s, c;
  float r = sqrtf(-2.0f * logf(philox_u01(o.x)));
  sincospif(2.0f * philox_u01(o.y), &s, &c);
  z[0] = r * c; z[1] = r * s;
  r = sqrtf(-2.0f * logf(philox_u01(o.z)));
  sincospif(2.0f * philox_u01(o.w), &s, &c);
  z[2] = r * c; z[3] = r * s;
}

}  // namespace gda
