// Philox4x32-10 counter-based generator, written from its published definition
// (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11):
// 10 rounds; each multiplies counter words 0 and 2 by fixed odd constants into 64-bit
// products, then recombines high halves with words 1 and 3 and the round key; the key advances
// by the Weyl increments (golden ratio and sqrt(3) - 1 in 32-bit fixed point) between rounds.
#pragma once
#include <stdint.h>

namespace negf {

struct PhiloxKey { uint32_t k0, k1; };

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, PhiloxKey key) {
  constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
  constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
  uint32_t k0 = key.k0, k1 = key.k1;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kM0, c.x), lo0 = kM0 * c.x;
    const uint32_t hi1 = __umulhi(kM1, c.z), lo1 = kM1 * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += kW0;
    k1 += kW1;
  }
  return c;
}

}  // namespace negf
