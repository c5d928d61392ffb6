// Level-2 blocks of two-level tables: the inverse-CDF draw of a site within a slice (the paper's
// cumulative-sum search of Step 6', in integers behind a guide).  Shared by the level-2 pass over
// stored weights (k_alias.cu) and the CTA-wide chain that emits the blocks directly
// (k_chain_cta.cu), so that both produce the same bits from the same FP32 weights.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace negf {
namespace {

constexpr uint32_t kCdfOne = 1u << 31;
__device__ __forceinline__ float pow2f_l2(int e) { return __int_as_float((e + 127) << 23); }

// floor(2^62 / T) for T in [2^29 - 64, 2^31), exactly, without a 64-bit division (its emulation
// runs on the FP64 pipe, narrow on this GPU): q0 from a float reciprocal (within ~2^11 of the
// quotient), one correction by the remainder r = 2^62 - q T divided in floats (|r| < 2^42, so
// r / 2^10 fits 32 bits; the corrected q is within one), then unit steps until 0 <= r < T.
__device__ __forceinline__ uint64_t recip_2p62(uint32_t T) {
  const float rt = __frcp_rn((float)T);
  uint64_t q = (uint64_t)__float2uint_rz(rt * 2305843009213693952.0f) << 1;   // 2 (2^61 / T)
  const uint64_t two62 = 1ull << 62;
  int64_t r = (int64_t)(two62 - q * (uint64_t)T);
  const float rf = (float)(int32_t)(r >> 10) * 1024.0f;
  q += (uint64_t)(int64_t)__float2int_rz(rf * rt);
  r = (int64_t)(two62 - q * (uint64_t)T);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (r < 0) {
      --q;
      r += T;
    } else if (r >= (int64_t)T) {
      ++q;
      r -= T;
    }
  }
  return q;
}

// Thresholds of one slice's W <= WB FP32 weights wt(0) .. wt(W - 1) (WB a multiple of 16, or
// below 16): the exact fixed-point prefix c_a = floor(2^31 P_a / T) (c = 2^31 where P_a
// reaches the total), with the weights scaled by a power of two so that their integer total T
// lies in [2^29, 2^31) and divided by T through a 64-bit reciprocal; an empty slice gives all
// 2^31.  *total: the slice's weight as
// the integer total scaled back.  Returns false on a negative or non-finite sum.
template <int WB, typename Wf>
__device__ __forceinline__ bool level2_fp32(Wf wt, int W, uint32_t (&c)[WB], float* total) {
  bool ok = true;
  float tot = 0.f;
  // chunks of 16 weights: the float sum S (it only sets the scale) as the sum of the chunks'
  // sums combined pairwise, and the integer total and prefix chunk by chunk (exact in any order)
  constexpr int kCh = WB < 16 ? WB : 16;
  constexpr int nCh = WB / kCh;
  float cs[nCh];
#pragma unroll
  for (int h = 0; h < nCh; ++h) cs[h] = 0.f;
#pragma unroll
  for (int a = 0; a < WB; ++a)
    if (a < W) cs[a / kCh] += wt(a);
  float S = cs[0];
  if (nCh == 2) S = cs[0] + cs[1];
  if (nCh == 4) S = (cs[0] + cs[1]) + (cs[2 % nCh] + cs[3 % nCh]);
  if (!(S >= 0.f && S < INFINITY)) ok = false;
  if (S > 0.f && S < INFINITY) {
    int e = 0;
    frexpf(S, &e);                             // S = f 2^e, f in [1/2, 1)
    const int sh = 30 - e, sh1 = sh / 2, sh2 = sh - sh / 2;
    const float p1 = pow2f_l2(sh1), p2 = pow2f_l2(sh2);
#pragma unroll
    for (int a = 0; a < WB; ++a) {
      const float v = a < W ? wt(a) : 0.f;
      c[a] = v > 0.f ? __float2uint_rz((v * p1) * p2) : 0u;
    }
    // prefix within chunks of 16, then the chunks' offsets
#pragma unroll
    for (int a = 0; a < WB; ++a)
      if (a % kCh) c[a] += c[a - 1];
    uint32_t off[nCh];
    off[0] = 0;
#pragma unroll
    for (int h = 1; h < nCh; ++h) off[h] = off[h - 1] + c[h * kCh - 1];
    const uint32_t T = off[nCh - 1] + c[WB - 1];
    tot = (__uint2float_rn(T) * pow2f_l2(-sh1)) * pow2f_l2(-sh2);
    const uint64_t Rr = recip_2p62(T);                 // floor(2^62 / T), T >= 2^29 - W
#pragma unroll
    for (int a = 0; a < WB; ++a) {
      const uint32_t P = off[a / kCh] + c[a];
      const uint32_t q = (uint32_t)(((uint64_t)P * Rr) >> 31);
      c[a] = P == T ? kCdfOne : min(q, kCdfOne - 1u);
    }
  } else {
#pragma unroll
    for (int a = 0; a < WB; ++a) c[a] = kCdfOne;
  }
  *total = tot;
  return ok;
}

// level2_fp32 for a 64-weight slice on a pair of adjacent lanes (lane parity h): each takes
// weights 32 h .. 32 h + 31 (wt(a) for a < 32 gives the lane's own a + 32 h); the chunk sums and
// chunk totals are exchanged so that both lanes form the same S, T and offsets as level2_fp32
// does alone, hence the same thresholds, of which c holds the lane's half.  Every lane of the
// warp must call it (shuffles).
template <typename Wf>
__device__ __forceinline__ bool level2_fp32_pair(Wf wt, int h, uint32_t (&c)[32], float* total) {
  bool ok = true;
  float tot = 0.f;
  float cs0 = 0.f, cs1 = 0.f;                   // the lane's chunks 2h, 2h + 1
#pragma unroll
  for (int a = 0; a < 16; ++a) cs0 += wt(a);
#pragma unroll
  for (int a = 16; a < 32; ++a) cs1 += wt(a);
  const float mine = cs0 + cs1;                 // (cs[0] + cs[1]) or (cs[2] + cs[3])
  const float other = __shfl_xor_sync(0xffffffffu, mine, 1);
  const float S = h == 0 ? mine + other : other + mine;
  if (!(S >= 0.f && S < INFINITY)) ok = false;
  uint32_t t0 = 0, t1 = 0;
  int sh1 = 0, sh2 = 0;
  const bool pos = S > 0.f && S < INFINITY;
  if (pos) {
    int e = 0;
    frexpf(S, &e);
    const int sh = 30 - e;
    sh1 = sh / 2;
    sh2 = sh - sh / 2;
    const float p1 = pow2f_l2(sh1), p2 = pow2f_l2(sh2);
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      const float v = wt(a);
      c[a] = v > 0.f ? __float2uint_rz((v * p1) * p2) : 0u;
    }
#pragma unroll
    for (int a = 0; a < 32; ++a)
      if (a % 16) c[a] += c[a - 1];
    t0 = c[15];
    t1 = c[31];
  }
  // chunk totals of the partner: offsets of chunks 0..3 and T as level2_fp32 forms them
  const uint32_t u0 = __shfl_xor_sync(0xffffffffu, t0, 1);
  const uint32_t u1 = __shfl_xor_sync(0xffffffffu, t1, 1);
  if (pos) {
    const uint32_t a0 = h == 0 ? t0 : u0, a1 = h == 0 ? t1 : u1;   // chunks 0, 1
    const uint32_t a2 = h == 0 ? u0 : t0, a3 = h == 0 ? u1 : t1;   // chunks 2, 3
    const uint32_t off1 = a0, off2 = off1 + a1, off3 = off2 + a2;
    const uint32_t T = off3 + a3;
    const uint32_t o0 = h == 0 ? 0u : off2, o1 = h == 0 ? off1 : off3;
    tot = (__uint2float_rn(T) * pow2f_l2(-sh1)) * pow2f_l2(-sh2);
    const uint64_t Rr = recip_2p62(T);
#pragma unroll
    for (int a = 0; a < 32; ++a) {
      const uint32_t P = (a < 16 ? o0 : o1) + c[a];
      const uint32_t q = (uint32_t)(((uint64_t)P * Rr) >> 31);
      c[a] = P == T ? kCdfOne : min(q, kCdfOne - 1u);
    }
  } else {
#pragma unroll
    for (int a = 0; a < 32; ++a) c[a] = kCdfOne;
  }
  *total = tot;
  return ok;
}

// The block of thresholds c, four words at a time (put4(word index, words)): for W > 8 an
// 8-word guide (the last threshold of each octet but the last, then 2^31) followed by
// ceil(W / 8) octets; for W <= 8 one octet.  The slice's last threshold and the padding of the
// last octet are 2^31.
template <int WB, typename Put4>
__device__ __forceinline__ void level2_pack4(const uint32_t (&c)[WB], int W, Put4 put4) {
  const int G = (W + 7) >> 3;
  int base = 0;
  if (G > 1) {
    uint32_t g[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      constexpr int dummy = 0;
      const int idx = 8 * q + 7 < WB ? 8 * q + 7 : dummy;
      g[q] = (q < G - 1 && 8 * q + 7 < WB) ? c[idx] : kCdfOne;
    }
    put4(0, make_uint4(g[0], g[1], g[2], g[3]));
    put4(4, make_uint4(g[4], g[5], g[6], g[7]));
    base = 8;
  }
#pragma unroll
  for (int a = 0; a < WB; a += 4) {
    if (a < 8 * G) {
      uint32_t v[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) v[j] = a + j < W - 1 ? c[a + j] : kCdfOne;
      put4(base + a, make_uint4(v[0], v[1], v[2], v[3]));
    }
  }
}

}  // namespace
}  // namespace negf
