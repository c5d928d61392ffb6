// Fixed-point helpers of the exact integer alias construction: scaling a weight by a power of
// two and truncating it to an integer, without overflow of the intermediate for any finite
// weight of a row whose largest weight sets the shift.
#pragma once

#include <stdint.h>

namespace negf {

__device__ __forceinline__ uint64_t small_pack(uint32_t thr, uint32_t alias) {
  return (uint64_t)thr | ((uint64_t)alias << 32);
}
// 2^e as a float for e in [-126, 127]
__device__ __forceinline__ float small_pow2f(int e) { return __int_as_float((e + 127) << 23); }
// trunc(w 2^sh) for w 2^sh < 2^32: w scaled by two exact power-of-two factors (each within the
// normal range for any finite float w and the sh of its row)
__device__ __forceinline__ uint32_t small_fixp(float w, int sh) {
  const int h = sh / 2;
  return __float2uint_rz((w * small_pow2f(h)) * small_pow2f(sh - h));
}
__device__ __forceinline__ uint32_t small_fixp(double w, int sh) {
  return __double2uint_rz(ldexp(w, sh));
}

}  // namespace negf
