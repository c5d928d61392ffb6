// Alias row of k <= 64 weights built by one thread in exact integer arithmetic (no scratch
// memory): the level-2 rows of two-level Step 6' tables.
//
// Quantisation as in the warp-wide row build: the largest weight is scaled into [2^31, 2^32)
// by a power of two and every weight truncated to an integer m_i; T = sum m_i.  Slot units
// u_i = floor(m_i k 2^32 / T) are evaluated with the per-row reciprocal R0 = floor((2^64-1)/T)
// (each low by at most 65 units), and the shortfall k 2^32 - sum u_i goes to the largest item,
// so that every one of the k slots holds exactly 2^32 units.  Small items (u < 2^32) are then
// paired with the current large item, lowest indices first; a large item whose remainder drops
// below 2^32 is paired next.  u_i is recomputed from w_i when needed.  Zero rows get all-full
// slots.  Entry = threshold (low 32 bits) | alias (high 32 bits); full slots alias themselves.
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

// wget(i) returns weight i (float or double); put(i, entry) stores slot i.  Returns false when
// a weight is negative or not finite (it is treated as 0).
template <typename R, typename Get, typename Put>
__device__ bool alias_small(int k, Get wget, Put put) {
  constexpr uint64_t kSlot = 1ull << 32;
  bool ok = true;
  R wmax = 0;
  int imax = 0;
  for (int i = 0; i < k; ++i) {
    const R v = wget(i);
    if (!(v >= (R)0) || !isfinite(v)) {
      ok = false;
    } else if (v > wmax) {
      wmax = v;
      imax = i;
    }
  }
  if (!(wmax > (R)0)) {
    for (int i = 0; i < k; ++i) put(i, small_pack(0xffffffffu, (uint32_t)i));
    return ok;
  }
  int e = 0;
  frexp((double)wmax, &e);
  const int sh = 32 - e;                         // wmax 2^sh in [2^31, 2^32)
  auto m_of = [&](int i) -> uint64_t {
    const R v = wget(i);
    return (v >= (R)0 && isfinite(v)) ? (uint64_t)small_fixp(v, sh) : 0ull;
  };
  uint64_t T = 0;
  for (int i = 0; i < k; ++i) T += m_of(i);
  const uint64_t R0 = ~0ull / T;
  auto u_base = [&](int i) -> uint64_t {
    const uint64_t X = m_of(i) * (uint64_t)k;
    return (__umul64hi(X, R0) << 32) | ((X * R0) >> 32);
  };
  uint64_t sum = 0;
  for (int i = 0; i < k; ++i) sum += u_base(i);
  const uint64_t rem = ((uint64_t)k << 32) - sum;
  auto u_of = [&](int i) -> uint64_t { return u_base(i) + (i == imax ? rem : 0ull); };
  uint64_t small = 0, large = 0;
  for (int i = 0; i < k; ++i) {
    if (u_of(i) < kSlot) small |= 1ull << i;
    else large |= 1ull << i;
  }
  int cur = -1;
  uint64_t ul = 0;
  if (large) {
    cur = __ffsll((long long)large) - 1;
    large &= large - 1;
    ul = u_of(cur);
  }
  int pend = -1;
  uint64_t pv = 0;
  while (true) {
    int s;
    uint64_t us;
    if (pend >= 0) {
      s = pend;
      us = pv;
      pend = -1;
    } else if (small) {
      s = __ffsll((long long)small) - 1;
      small &= small - 1;
      us = u_of(s);
    } else {
      break;
    }
    if (cur < 0) {
      put(s, small_pack(0xffffffffu, (uint32_t)s));
      continue;
    }
    put(s, small_pack((uint32_t)us, (uint32_t)cur));
    ul -= kSlot - us;
    if (ul < kSlot) {
      pend = cur;
      pv = ul;
      if (large) {
        cur = __ffsll((long long)large) - 1;
        large &= large - 1;
        ul = u_of(cur);
      } else {
        cur = -1;
      }
    }
  }
  if (cur >= 0) put(cur, small_pack(0xffffffffu, (uint32_t)cur));
  while (large) {
    const int i = __ffsll((long long)large) - 1;
    large &= large - 1;
    put(i, small_pack(0xffffffffu, (uint32_t)i));
  }
  return ok;
}

}  // namespace negf

namespace negf {

// The same construction with the slot units kept in u[0..k) (shared memory of the caller):
// u is filled with u_i, and every slot's entry then overwrites its own u_i (a slot's u is read
// before its entry is written).  Same entries as alias_small.  *total receives the fixed-point
// sum T 2^-sh of the weights (within k 2^-32 of the largest weight below the exact sum), *sum64
// (if given) their FP64 sum in index order.  The weights may live in u's memory (each row's
// weights packed from its start): every weight is read before u overwrites it.
template <typename R, typename Get>
__device__ bool alias_small_inplace(int k, Get wget, uint64_t* u, double* total,
                                    double* sum64 = nullptr) {
  constexpr uint64_t kSlot = 1ull << 32;
  bool ok = true;
  R wmax = 0;
  int imax = 0;
  double s64 = 0.0;
  for (int i = 0; i < k; ++i) {
    const R v = wget(i);
    if (sum64) s64 += (double)v;
    if (!(v >= (R)0) || !isfinite(v)) {
      ok = false;
    } else if (v > wmax) {
      wmax = v;
      imax = i;
    }
  }
  if (sum64) *sum64 = s64;
  if (!(wmax > (R)0)) {
    for (int i = 0; i < k; ++i) u[i] = small_pack(0xffffffffu, (uint32_t)i);
    *total = 0.0;
    return ok;
  }
  int e = 0;
  frexp((double)wmax, &e);
  const int sh = 32 - e;
  uint64_t T = 0;
  // descending, so that u may share its memory with the weights: u[i] covers bytes [8i, 8i + 8)
  // of the row, which hold weights of index >= i, all read by then
  for (int i = k - 1; i >= 0; --i) {
    const R v = wget(i);
    const uint64_t m = (v >= (R)0 && isfinite(v)) ? (uint64_t)small_fixp(v, sh) : 0ull;
    u[i] = m;
    T += m;
  }
  *total = ldexp((double)T, -sh);
  const uint64_t R0 = ~0ull / T;
  uint64_t sum = 0;
  for (int i = 0; i < k; ++i) {
    const uint64_t X = u[i] * (uint64_t)k;
    const uint64_t ui = (__umul64hi(X, R0) << 32) | ((X * R0) >> 32);
    u[i] = ui;
    sum += ui;
  }
  u[imax] += ((uint64_t)k << 32) - sum;
  uint64_t small = 0, large = 0;
  for (int i = 0; i < k; ++i) {
    if (u[i] < kSlot) small |= 1ull << i;
    else large |= 1ull << i;
  }
  int cur = -1;
  uint64_t ul = 0;
  if (large) {
    cur = __ffsll((long long)large) - 1;
    large &= large - 1;
    ul = u[cur];
  }
  int pend = -1;
  uint64_t pv = 0;
  while (true) {
    int s;
    uint64_t us;
    if (pend >= 0) {
      s = pend;
      us = pv;
      pend = -1;
    } else if (small) {
      s = __ffsll((long long)small) - 1;
      small &= small - 1;
      us = u[s];
    } else {
      break;
    }
    if (cur < 0) {
      u[s] = small_pack(0xffffffffu, (uint32_t)s);
      continue;
    }
    u[s] = small_pack((uint32_t)us, (uint32_t)cur);
    ul -= kSlot - us;
    if (ul < kSlot) {
      pend = cur;
      pv = ul;
      if (large) {
        cur = __ffsll((long long)large) - 1;
        large &= large - 1;
        ul = u[cur];
      } else {
        cur = -1;
      }
    }
  }
  if (cur >= 0) u[cur] = small_pack(0xffffffffu, (uint32_t)cur);
  while (large) {
    const int i = __ffsll((long long)large) - 1;
    large &= large - 1;
    u[i] = small_pack(0xffffffffu, (uint32_t)i);
  }
  return ok;
}

}  // namespace negf
