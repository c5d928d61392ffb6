// Alias-table construction for the Step 6' categorical draw.
//
// Sec. III.B draws the next index by a cumulative sum and a search (O(K) per step).  The walk
// here uses Walker's alias method (one table entry per draw), so each row of weights is turned
// into K slots (threshold, alias).  One warp builds one row, in exact integer arithmetic on a
// quantised copy of the row, by a parallel "sweep" construction (in the spirit of
// Hubschle-Schneider and Sanders, "Parallel weighted random sampling", ESA 2019), written from
// this derivation:
//
//   Quantise: scale the row by a power of two so that its largest weight lies in [2^31, 2^32)
//   and truncate to integers m_i (exact scaling, no rounding of the others beyond 2^-32 of the
//   largest); T = sum m_i is exact.  Then u_i = floor(m_i K 2^32 / T) (by a 64 x 64 -> 128-bit
//   product with a per-row reciprocal), and the integer remainder K 2^32 - sum(u) goes to the
//   largest item, so that sum(u) = K 2^32 exactly and every slot holds exactly 2^32 units.  Light items (u < 2^32) in index order carry deficits 2^32 - u with
//   inclusive prefix sums Lc_r; heavy items (u >= 2^32) carry excesses u - 2^32 with inclusive
//   prefix sums Ec_j.  Heavy j owns the interval [Ec_{j-1}, Ec_j) of the deficit line.
//   * light r keeps thr = u and aliases the heavy whose interval contains its start Lc_{r-1};
//   * heavy j (not the last) is consumed past its excess by the light interval (Lc_{r-1}, Lc_r]
//     that contains Ec_j; its slot keeps thr = 2^32 - (Lc_r - Ec_j) and aliases heavy j+1.
//     If no light interval contains Ec_j (Ec_j == 0) the slot is full;
//   * the last heavy is full (sum of deficits == sum of excesses exactly).
//   Every item then holds exactly u_i of the K 2^32 units.
// Full slots store thr = 2^32 - 1 and alias = self.  The FP64 row sum is also the sum-rule check
// of Sec. II.D (each row must add up to <i|A|i>, which the diagonal-block kernel stored).
#include <cuda_runtime.h>
#include <math.h>

#include "alias_small.cuh"
#include "level2.cuh"
#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr uint64_t kSlot = 1ull << 32;

__device__ __forceinline__ uint64_t pack(uint32_t thr, uint32_t alias) {
  return (uint64_t)thr | ((uint64_t)alias << 32);
}

// Each lane owns a block of npl = ceil(K/32) consecutive items.  Per-item values live in shared
// memory at slot (i / npl) * pitch + i % npl, with an odd pitch (npl or npl + 1) so that the 32
// lanes walking their blocks in step touch 32 different banks.
__host__ __device__ inline int alias_npl(int K) { return (K + 31) >> 5; }
__host__ __device__ inline int alias_pitch(int K) { return alias_npl(K) | 1; }
// Per-warp shared memory: s_u, s_c : u64 [32 pitch] | s_x : u32 [cap] | staging buffer for the
// next row's weights (cap elements of `elem` bytes, or 64 FP64 mode weights), 16-byte aligned.
__host__ __device__ inline size_t alias_stage_off(int cap) {
  const size_t slots = (size_t)32 * alias_pitch(cap);
  return (2 * slots * sizeof(uint64_t) + (size_t)cap * sizeof(uint32_t) + 15) & ~(size_t)15;
}
__host__ __device__ inline size_t alias_warp_bytes(int cap, int elem) {
  const size_t stage = (size_t)cap * elem > 64 * sizeof(double) ? (size_t)cap * elem
                                                                  : 64 * sizeof(double);
  return alias_stage_off(cap) + ((stage + 15) & ~(size_t)15);
}

// Asynchronous global -> shared copies of 4 or 8 bytes (the weights of the next row).
template <int kBytes>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(kBytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

__device__ __forceinline__ uint32_t fixp(float w, int sh) { return small_fixp(w, sh); }
__device__ __forceinline__ uint32_t fixp(double w, int sh) { return __double2uint_rz(ldexp(w, sh)); }

// First index in [lo, hi) whose key is > x (pred gt) or >= x (pred ge); hi when none.  key(i) is
// non-decreasing.  Starts with a gallop from lo, so that a cursor that moves little costs a few
// loads.
template <bool kStrict, typename Key>
__device__ __forceinline__ int gallop_first(int lo, int hi, uint64_t x, Key key) {
  auto past = [&](int i) { return kStrict ? key(i) > x : key(i) >= x; };
  if (lo >= hi || past(lo)) return lo;
  int step = 1;                                   // key(lo) fails the test
  int a = lo;                                     // invariant: key(a) fails
  while (a + step < hi && !past(a + step)) {
    a += step;
    step <<= 1;
  }
  int b = min(a + step, hi);                      // b == hi or key(b) passes
  ++a;
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (past(mid)) b = mid; else a = mid + 1;
  }
  return a;
}

// Build one row.  w: the K weights, staged in shared memory; A: the value the row must sum to
// (checked when check_A, to tol A + atol: a row whose spectral weight is at the rounding level
// of G, such as an orbital no open channel reaches, carries only rounding noise); out: K
// entries; rowsum_out: receives the row sum.  s_u, s_c:
// 32 * alias_pitch(K) u64 each; s_x: K u32.  after_stage() is called by every lane once w has
// been read (the caller reuses w's buffer for the next row).
template <typename R, typename After>
__device__ void alias_row(const R* w, int K, double A, bool check_A, double tol, double atol,
                          uint64_t* __restrict__ out, double* rowsum_out, uint64_t* s_u,
                          uint64_t* s_c, uint32_t* s_x, int32_t* err, After after_stage) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const int npl = alias_npl(K), pitch = alias_pitch(K);
  // slots of items lane, lane + 32, ...: (quotient, remainder) by npl, stepped by 32
  const int q32 = 32 / npl, r32 = 32 - q32 * npl;
  const int qlane = lane / npl, rlane = lane - qlane * npl;
  const int i0 = lane * npl;                                    // this lane's items [i0, i1)
  const int i1 = min(K, i0 + npl);
  const int mine = max(0, i1 - i0);
  uint64_t* my_u = s_u + lane * pitch;
  R* s_w = reinterpret_cast<R*>(s_c);
  R* my_w = s_w + lane * pitch;
  // pass 1 (coalesced): stage the row, largest weight; FP64 rows also take their FP64 sum here
  // (lane-strided order, tree to lane 0)
  R wmax = 0;
  bool bad = false;
  double part = 0.0;
  for (int i = lane, q = qlane, rm = rlane; i < K; i += 32) {
    const R v = w[i];
    s_w[q * pitch + rm] = v;
    q += q32;
    rm += r32;
    if (rm >= npl) { rm -= npl; ++q; }
    bad |= !(v >= 0) || !isfinite(v);
    if (v > wmax && isfinite(v)) wmax = v;
    if (sizeof(R) == 8) part += (double)v;
  }
  __syncwarp();
  after_stage();
  for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(FULL, wmax, off));
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
  if (!(wmax > 0)) {
    if (lane == 0) *rowsum_out = 0.0;
    if (lane == 0 && check_A && A > 1e-300 && A > atol) atomicOr(err, ERR_ROWSUM);
    for (int i = lane; i < K; i += 32) out[i] = pack(0xffffffffu, (uint32_t)i);
    return;
  }
  int ex = 0;
  if (sizeof(R) == 4) frexpf((float)wmax, &ex);   // wmax = f 2^ex, f in [0.5, 1)
  else frexp((double)wmax, &ex);
  const int sh = 32 - ex;                          // wmax 2^sh in [2^31, 2^32)
  // pass 2 (own block): integer weights m_i, T = sum m_i
  uint64_t T = 0;
  for (int k = 0; k < mine; ++k) {
    const R v = my_w[k];
    const uint32_t m = (v > 0 && isfinite(v)) ? fixp(v, sh) : 0u;
    my_u[k] = m;
    T += m;
  }
  for (int off = 16; off > 0; off >>= 1) T += __shfl_xor_sync(FULL, T, off);
  // row sum: FP64 weights are summed in FP64; FP32 weights use the exact fixed-point sum
  // (within K 2^-32 of the largest weight)
  if (sizeof(R) == 8)
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(FULL, part, off);
  // the FP64 steps run on lane 0 only (FP64 throughput is low); the reciprocal is broadcast
  uint64_t rcp = 0;
  if (lane == 0) {
    const double total = sizeof(R) == 8 ? part : ldexp((double)T, -sh);
    rcp = (uint64_t)(ldexp(1.0, 94) / (double)T);   // < 2^63 since T >= 2^31
    *rowsum_out = total;
    if (check_A && A > 1e-300 && fabs(total - A) > tol * A + atol) atomicOr(err, ERR_ROWSUM);
  }
  // pass 3: u_i = floor(m_i K 2^32 / T) = (m_i K) (2^94 / T) / 2^62, with the 128-bit product
  rcp = __shfl_sync(FULL, rcp, 0);
  const uint64_t target = (uint64_t)K << 32;
  uint64_t usum = 0, umax = 0;
  int imax = 0x7fffffff;
  for (int k = 0; k < mine; ++k) {
    const uint64_t q = my_u[k] * (uint64_t)K;
    const uint64_t hi = __umul64hi(q, rcp), lo = q * rcp;
    uint64_t u = (hi << 2) | (lo >> 62);
    if (u > target) u = target;
    my_u[k] = u;
    usum += u;
    if (u > umax) { umax = u; imax = i0 + k; }   // first index of the lane's maximum
  }
  for (int off = 16; off > 0; off >>= 1) {
    usum += __shfl_xor_sync(FULL, usum, off);
    const uint64_t om = __shfl_xor_sync(FULL, umax, off);
    const int oi = __shfl_xor_sync(FULL, imax, off);
    if (om > umax || (om == umax && oi < imax)) { umax = om; imax = oi; }
  }
  if (i0 <= imax && imax < i1) my_u[imax - i0] += target - usum;   // signed remainder
  // pass 4: lights (u < 2^32) carry deficits 2^32 - u, heavies excesses u - 2^32; exclusive
  // prefix over the lanes of counts and sums
  uint32_t cnt = 0;                               // lights | heavies << 16
  uint64_t dl = 0, dh = 0;
  for (int k = 0; k < mine; ++k) {
    const uint64_t u = my_u[k];
    if (u >= kSlot) { cnt += 1u << 16; dh += u - kSlot; }
    else { cnt += 1u; dl += kSlot - u; }
  }
  uint32_t cx = cnt;
  uint64_t lx = dl, hx = dh;                      // inclusive scans
  for (int off = 1; off < 32; off <<= 1) {
    const uint32_t oc = __shfl_up_sync(FULL, cx, off);
    const uint64_t ol = __shfl_up_sync(FULL, lx, off);
    const uint64_t oh = __shfl_up_sync(FULL, hx, off);
    if (lane >= off) { cx += oc; lx += ol; hx += oh; }
  }
  const uint32_t ctot = __shfl_sync(FULL, cx, 31);
  const int nl = (int)(ctot & 0xffffu), nh = (int)(ctot >> 16);
  int r = (int)((cx - cnt) & 0xffffu), j = (int)((cx - cnt) >> 16);   // first light / heavy
  uint64_t runl = lx - dl, runh = hx - dh;                             // of this lane
  __syncwarp();                                   // s_w (in s_c) is dead from here
  // pass 5: Lc_r (inclusive deficit prefix, light order) from the front of s_c, Ec_j (inclusive
  // excess prefix, heavy order) from the back; s_x holds the item index of each
  for (int k = 0; k < mine; ++k) {
    const uint64_t u = my_u[k];
    if (u >= kSlot) {
      runh += u - kSlot;
      s_c[K - 1 - j] = runh;
      s_x[K - 1 - j] = (uint32_t)(i0 + k);
      ++j;
    } else {
      runl += kSlot - u;
      s_c[r] = runl;
      s_x[r] = (uint32_t)(i0 + k);
      ++r;
    }
  }
  __syncwarp();
  if (nh == 0) {   // cannot happen when sum(u) == K 2^32; keep the row drawable anyway
    for (int i = lane; i < K; i += 32) out[i] = pack(0xffffffffu, (uint32_t)i);
    return;
  }
  auto Ec = [&](int jj) { return s_c[K - 1 - jj]; };
  auto Lc = [&](int rr) { return s_c[rr]; };
  // pass 6: entries, into s_u by item index (s_u is dead from here).  The lanes split the light
  // list, then the heavy list, into contiguous ranges, each searched from a cursor that moves
  // forward.
  // Light r (start Lc_{r-1}, u_r = 2^32 - (Lc_r - Lc_{r-1})) aliases the heavy whose excess
  // interval [Ec_{j-1}, Ec_j) contains its start.
  {
    const int ra = (lane * nl) >> 5, rb = ((lane + 1) * nl) >> 5;
    uint64_t st = ra == 0 ? 0ull : Lc(ra - 1);
    int jc = 0;
    for (int rr = ra; rr < rb; ++rr) {
      const uint64_t Lr = Lc(rr);
      jc = gallop_first<true>(jc, nh, st, Ec);          // first j with Ec_j > st
      const int jj = jc < nh ? jc : nh - 1;
      s_u[s_x[rr]] = pack((uint32_t)(kSlot - (Lr - st)), s_x[K - 1 - jj]);
      st = Lr;
    }
  }
  // Heavy j (not the last, Ec_j > 0) is consumed past its excess by the light interval
  // (Lc_{r-1}, Lc_r] containing Ec_j: it keeps 2^32 - (Lc_r - Ec_j) and aliases heavy j + 1.
  {
    const int ja = (lane * nh) >> 5, jb = ((lane + 1) * nh) >> 5;
    int rc = 0;
    for (int jj = ja; jj < jb; ++jj) {
      const uint32_t self = s_x[K - 1 - jj];
      uint64_t e = pack(0xffffffffu, self);
      const uint64_t Ej = Ec(jj);
      if (jj < nh - 1 && Ej > 0) {
        rc = gallop_first<false>(rc, nl, Ej, Lc);       // first r with Lc_r >= Ej
        if (rc < nl) {
          const uint64_t used = Lc(rc) - Ej;            // consumed beyond the excess, <= 2^32
          if (used > 0) e = pack((uint32_t)(kSlot - used), s_x[K - 1 - (jj + 1)]);
        }
      }
      s_u[self] = e;
    }
  }
  __syncwarp();
  for (int i = lane; i < K; i += 32) out[i] = s_u[i];
}

template <typename R>
__global__ void alias_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t total_jobs,
                             int cap, double tol, const R* __restrict__ weights,
                             double* __restrict__ rowsum, const double* __restrict__ mode_w,
                             uint64_t* __restrict__ tab, uint64_t* __restrict__ mode_tab,
                             int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  unsigned char* base = smem_raw + (size_t)warp * alias_warp_bytes(cap, (int)sizeof(R));
  uint64_t* s_u = reinterpret_cast<uint64_t*>(base);
  uint64_t* s_c = s_u + (size_t)32 * alias_pitch(cap);
  uint32_t* s_x = reinterpret_cast<uint32_t*>(s_c + (size_t)32 * alias_pitch(cap));
  unsigned char* s_stage = base + alias_stage_off(cap);
  const uint32_t stride = gridDim.x * nwarps;
  // task owning a job: jobs of a warp only increase, so the search starts at the last task found
  int hint = 0;
  auto find = [&](uint32_t jb) {
    int lo = hint, hi = n_tasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].row_base <= jb) lo = mid; else hi = mid - 1;
    }
    return lo;
  };
  // the weights of job jb go to s_stage by asynchronous copies (one commit group)
  auto stage = [&](uint32_t jb) {
    const TaskDesc& d = tasks[find(jb)];
    const int row = (int)(jb - d.row_base);
    if (row < d.rows) {
      const R* src = weights + d.wt_off + (uint64_t)row * d.K;
      R* dst = reinterpret_cast<R*>(s_stage);
      for (int i = lane; i < d.K; i += 32) cp_async<(int)sizeof(R)>(dst + i, src + i);
    } else {
      const double* src = mode_w + d.mode_off + (row - d.rows) * d.W;
      double* dst = reinterpret_cast<double*>(s_stage);
      for (int i = lane; i < d.W; i += 32) cp_async<8>(dst + i, src + i);
    }
    cp_async_commit();
  };
  uint32_t job = blockIdx.x * nwarps + warp;
  if (job < total_jobs) stage(job);
  for (; job < total_jobs; job += stride) {
    hint = find(job);
    const TaskDesc& d = tasks[hint];
    const int row = (int)(job - d.row_base);
    const double A = rowsum[job];                 // <i|A|i> (rows) or c_p (mode rows)
    const uint32_t next = job + stride;
    auto after = [&]() {
      if (next < total_jobs) stage(next);
    };
    cp_async_wait_all();
    __syncwarp();
    if (row < d.rows) {
      alias_row<R>(reinterpret_cast<const R*>(s_stage), d.K, A, true, tol, 1e-13 / d.t,
                   tab + d.tab_off + (uint64_t)row * d.K, rowsum + job, s_u, s_c, s_x, err,
                   after);
    } else {
      const int p = row - d.rows;
      alias_row<double>(reinterpret_cast<const double*>(s_stage), d.W, A, true, 1e-9, 1e-13 / d.t,
                        mode_tab + d.mode_off + p * d.W, rowsum + job, s_u, s_c, s_x, err,
                        after);
    }
    __syncwarp();
  }
  cp_async_wait_all();
}

// ---- Level-2 inverse-CDF blocks of two-level tables --------------------------------------
//
// Within a slice the site is drawn by the paper's own categorical draw (Sec. III.B: cumulative
// sum of the weights, normalised, the first entry above a uniform), in integers: for the W site
// weights w_a of (table row, slice), c_a = floor(2^31 P_a / S) with P_a = sum_{b <= a} w_b and
// S = P_{W-1}, for a < W - 1; c_{W-1} and the padding of the last octet are 2^31.  Octet g holds
// c_{8g .. 8g+7}; for W > 8 an 8-word guide precedes the octets, guide_g = c_{8g+7} for
// g < G - 1 and 2^31 after (G = ceil(W / 8)).  The walk draws v = x >> 1 (31 bits), takes
// g = #{guide words <= v} and the site 8g + #{words of octet g <= v}, so site a has probability
// (c_a - c_{a-1}) / 2^31 and a zero weight is never drawn.  A slice whose weights sum to zero
// gets 2^31 everywhere (its level-1 weight is zero, so it is never drawn).
// FP32 weights: s = 2^sh with (FP32 sum) s in [2^29, 2^30); m_a = floor(w_a s) (exact scaling
// and truncation), P_a = sum m (exact integers, < 2^31), T = P_{W-1}, c_a = floor(P_a R / 2^31)
// with R = floor(2^62 / T) (within one unit below floor(2^31 P_a / T), nondecreasing in P_a),
// c_a = 2^31 where P_a = T; the slice's level-1 weight is T / s.  FP64 weights: P_a, S and c_a
// in FP64, level-1 weight S.
// One warp per table row, chunks of 32 slices: the chunk's weights are staged by coalesced loads,
// each lane forms one slice's block in registers and writes it into its shared region (odd pitch
// in 4-byte words), and the chunk's blocks (32 consecutive blocks of the row) leave by coalesced
// stores.
constexpr int kL2Warps = 4;

// Region pitch in 4-byte words: holds W weights of type R and a block of B2 words; odd for
// 4-byte accesses, 2 mod 4 for 8-byte ones (conflict-free across a half-warp).
template <typename R>
__host__ __device__ inline int level2_pitch(int W, int B2) {
  const int need = (int)(W * sizeof(R) / 4) > B2 ? (int)(W * sizeof(R) / 4) : B2;
  if (sizeof(R) == 4) return need | 1;
  int p = (need + 1) & ~1;
  if ((p & 3) == 0) p += 2;
  return p;
}

template <typename R, int WB>
__device__ __forceinline__ bool level2_block(uint32_t* reg, int W, int B2, R* total) {
  const R* wk = reinterpret_cast<const R*>(reg);
  uint32_t c[WB];
  bool ok = true;
  R tot = 0;
  if constexpr (sizeof(R) == 4) {
    float t32 = 0.f;
    ok = level2_fp32<WB>([&](int a) { return wk[a]; }, W, c, &t32);
    tot = t32;
  } else {
    double S = 0.0;
#pragma unroll
    for (int a = 0; a < WB; ++a)
      if (a < W) S += wk[a];
    if (!(S >= 0.0 && S < INFINITY)) ok = false;
    if (S > 0.0 && S < INFINITY) {
      const double scale = 2147483648.0 / S;
      double P = 0.0;
#pragma unroll
      for (int a = 0; a < WB; ++a) {
        P += a < W ? wk[a] : 0.0;
        c[a] = P >= S ? kCdfOne : min(__double2uint_rz(P * scale), kCdfOne - 1u);
      }
      tot = S;
    } else {
#pragma unroll
      for (int a = 0; a < WB; ++a) c[a] = kCdfOne;
    }
  }
  // c_{W-1} and the padding of the last octet are 2^31 (the weights have been read)
  const int G = (W + 7) >> 3;
  uint32_t* oct = G > 1 ? reg + 8 : reg;
#pragma unroll
  for (int a = 0; a < WB; ++a)
    if (a < 8 * G) oct[a] = a < W - 1 ? c[a] : kCdfOne;
  if (G > 1) {
#pragma unroll
    for (int g = 0; g < 8; ++g) reg[g] = (g < G - 1 && 8 * g + 7 < WB) ? c[8 * g + 7] : kCdfOne;
  }
  *total = tot;
  return ok;
}

template <typename R, int WB>
__global__ void __launch_bounds__(32 * kL2Warps) level2_cdf_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs, R* __restrict__ weights,
    uint64_t* __restrict__ tab, int32_t* err) {
  extern __shared__ __align__(16) unsigned char l2_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t job = blockIdx.x * kL2Warps + warp;
  if (job >= n_jobs) return;
  int lo = 0, hi = n_tasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].row_base <= job) lo = mid; else hi = mid - 1;
  }
  const TaskDesc& d = tasks[lo];
  if (d.layout != NEGF_LAYOUT_TWO_LEVEL || d.l2_fused) return;   // fused: written by the chain
  const int row = (int)(job - d.row_base);
  if (row >= d.rows) return;
  const int W = d.W, L = d.L, n = d.n;
  const int B2 = level2_words(W);
  const int PW = level2_pitch<R>(W, B2);
  uint32_t* wbase = reinterpret_cast<uint32_t*>(l2_smem) + (size_t)warp * 32 * PW;
  const R* wr = weights + d.wt_off + (uint64_t)row * d.K;
  R* l1 = weights + d.l1w_off + (uint64_t)row * (L + 2);
  uint32_t* l2 = reinterpret_cast<uint32_t*>(tab + d.tab_off) + (uint64_t)row * L * B2;
  constexpr int EW = (int)(sizeof(R) / 4);          // words per weight
  const int eq = 32 / W, er = 32 - (32 / W) * W;
  bool ok = true;
  for (int k0 = 0; k0 < L; k0 += 32) {
    const int ns = min(32, L - k0);
    const R* wc = wr + (uint64_t)k0 * W;
    if (EW == 1 && (W & 1) == 0 && (reinterpret_cast<uintptr_t>(wc) & 7) == 0) {
      // FP32 pairs (a pair never straddles two slices when W is even)
      const int hw = W >> 1;
      const int pq = 32 / hw, pr = 32 - (32 / hw) * hw;
      int q = lane / hw, r = lane - q * hw;
      for (int p = lane; p < ns * hw; p += 32) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(wc) + p);
        float* dst = reinterpret_cast<float*>(wbase + q * PW) + 2 * r;
        dst[0] = v.x;
        dst[1] = v.y;
        q += pq;
        r += pr;
        if (r >= hw) { r -= hw; ++q; }
      }
    } else {
      int q = lane / W, r = lane - q * W;
      for (int i = lane; i < ns * W; i += 32) {
        reinterpret_cast<R*>(wbase + q * PW)[r] = wc[i];
        q += eq;
        r += er;
        if (r >= W) { r -= W; ++q; }
      }
    }
    __syncwarp();
    if (lane < ns) {
      R tot = 0;
      ok &= level2_block<R, WB>(wbase + lane * PW, W, B2, &tot);
      l1[k0 + lane] = tot;
    }
    __syncwarp();
    // the chunk's ns blocks are contiguous; blocks are multiples of 8 words, the row's level 2
    // starts 32-byte aligned, so four consecutive words of one block leave as one 16-byte store
    uint32_t* oc = l2 + (uint64_t)k0 * B2;
    {
      int q = (4 * lane) / B2, r = 4 * lane - q * B2;
      const int sq = 128 / B2, sr = 128 - (128 / B2) * B2;
      for (int i = 4 * lane; i < ns * B2; i += 128) {
        const uint32_t* src = wbase + q * PW + r;
        *reinterpret_cast<uint4*>(oc + i) = make_uint4(src[0], src[1], src[2], src[3]);
        q += sq;
        r += sr;
        while (r >= B2) { r -= B2; ++q; }
      }
    }
    __syncwarp();
  }
  if (lane == 0) {
    l1[L] = wr[n];
    l1[L + 1] = wr[n + 1];
  }
  if (__any_sync(0xffffffffu, !ok) && lane == 0) atomicOr(err, ERR_NONFINITE);
}

// Step 7' energy rows of inelastic Buttiker probes (Sec. II.F, Eq. draw_E_last): for task t (the
// energy E_e of its wire) and site i, the alias row over the wire's grid energies e' of
//   w_e' K(E_e' - E_e) A_ii(E_e'),   K(dE) = exp(-dE^2 / (2 sigma^2)) (the identity for
// sigma = 0), A_ii(E_e') the row sum of site row i of the wire's task at e' (after the alias
// build), w_e' the energy's quadrature weight.  One warp per (task, site) row, into
// etab + eoff(t) + i nE.
__global__ void energy_alias_kernel(const TaskDesc* __restrict__ tasks, int n_tasks,
                                    const EnergyDesc* __restrict__ edesc,
                                    const uint32_t* __restrict__ job_base, uint32_t total_jobs,
                                    int cap, double sigma, const double* __restrict__ rowsum,
                                    uint64_t* __restrict__ etab, int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  unsigned char* base = smem_raw + (size_t)warp * alias_warp_bytes(cap, (int)sizeof(double));
  uint64_t* s_u = reinterpret_cast<uint64_t*>(base);
  uint64_t* s_c = s_u + (size_t)32 * alias_pitch(cap);
  uint32_t* s_x = reinterpret_cast<uint32_t*>(s_c + (size_t)32 * alias_pitch(cap));
  double* s_w = reinterpret_cast<double*>(base + alias_stage_off(cap));
  for (uint32_t job = blockIdx.x * nwarps + warp; job < total_jobs; job += gridDim.x * nwarps) {
    int lo = 0, hi = n_tasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (job_base[mid] <= job) lo = mid; else hi = mid - 1;
    }
    const TaskDesc& d = tasks[lo];
    const EnergyDesc ed = edesc[lo];
    const int i = (int)(job - job_base[lo]);
    const int nE = ed.nE;
    const double inv2s2 = sigma > 0.0 ? 0.5 / (sigma * sigma) : 0.0;
    for (int ep = lane; ep < nE; ep += 32) {
      const TaskDesc& dp = tasks[ed.t0 + ep];
      const double dE = dp.E - d.E;
      const double K = sigma > 0.0 ? exp(-dE * dE * inv2s2) : (ep == d.e_idx ? 1.0 : 0.0);
      s_w[ep] = dp.w_E * K * rowsum[dp.row_base + i];
    }
    __syncwarp();
    double total = 0.0;
    alias_row<double>(s_w, nE, 0.0, false, 0.0, 0.0, etab + ed.eoff + (uint64_t)i * nE, &total,
                      s_u, s_c, s_x, err, [] {});
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_two_level_split(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs,
                                   int precision, void* d_weights, uint64_t* d_tab,
                                   int32_t* d_err, cudaStream_t s, int max_W) {
  if (n_jobs == 0 || n_tasks == 0) return cudaSuccess;
  const unsigned blocks = (n_jobs + kL2Warps - 1) / kL2Warps;
  auto run = [&](auto kernel, auto tag, int wb) -> cudaError_t {
    using R = decltype(tag);
    // shared memory for the widest slice the kernel instance takes (W <= wb)
    int pw = 0;
    for (int W = 1; W <= wb; ++W) {
      const int p = level2_pitch<R>(W, level2_words(W));
      pw = p > pw ? p : pw;
    }
    const size_t smem = (size_t)kL2Warps * 32 * pw * 4;
    const cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return e;
    kernel<<<blocks, 32 * kL2Warps, smem, s>>>(d_tasks, n_tasks, n_jobs, static_cast<R*>(d_weights),
                                               d_tab, d_err);
    return cudaGetLastError();
  };
  if (precision == NEGF_FP64) {
    if (max_W <= 16) return run(level2_cdf_kernel<double, 16>, 0.0, 16);
    if (max_W <= 32) return run(level2_cdf_kernel<double, 32>, 0.0, 32);
    return run(level2_cdf_kernel<double, 64>, 0.0, 64);
  }
  if (max_W <= 16) return run(level2_cdf_kernel<float, 16>, 0.f, 16);
  if (max_W <= 32) return run(level2_cdf_kernel<float, 32>, 0.f, 32);
  return run(level2_cdf_kernel<float, 64>, 0.f, 64);
}

cudaError_t launch_energy_tables(const TaskDesc* d_tasks, int n_tasks, const EnergyDesc* d_edesc,
                                 const uint32_t* d_job_base, uint32_t total_jobs, int max_nE,
                                 double sigma, const double* d_rowsum, uint64_t* d_etab,
                                 int32_t* d_err, cudaStream_t s) {
  if (total_jobs == 0) return cudaSuccess;
  const int cap = max_nE < 64 ? 64 : max_nE;
  const size_t per_warp = alias_warp_bytes(cap, (int)sizeof(double));
  int warps = 4;
  while (warps > 1 && per_warp * warps > 200 * 1024) --warps;
  const size_t smem = per_warp * warps;
  if (smem > 220 * 1024) return cudaErrorInvalidValue;     // energy grids beyond shared memory
  cudaError_t e = cudaFuncSetAttribute(energy_alias_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t blocks = (total_jobs + warps - 1) / warps;
  if (blocks > (uint32_t)sms * 16) blocks = (uint32_t)sms * 16;
  energy_alias_kernel<<<blocks, warps * 32, smem, s>>>(d_tasks, n_tasks, d_edesc, d_job_base,
                                                      total_jobs, cap, sigma, d_rowsum, d_etab,
                                                      d_err);
  return cudaGetLastError();
}

int alias_warps_max(int max_K) {
  const int cap = max_K < 64 ? 64 : max_K;
  const size_t per_warp = alias_warp_bytes(cap, (int)sizeof(double));
  int w = 16;
  while (w > 1 && per_warp * w > 200 * 1024) --w;
  return w;
}

cudaError_t launch_alias_build(const TaskDesc* d_tasks, int n_tasks, uint32_t total_jobs,
                               int max_K, int precision, const void* d_weights,
                               double* d_rowsum, const double* d_mode_w, uint64_t* d_tab,
                               uint64_t* d_mode_tab, int32_t* d_err, cudaStream_t s,
                               int warps_req) {
  if (total_jobs == 0) return cudaSuccess;
  const int cap = max_K < 64 ? 64 : max_K;
  const size_t per_warp =
      alias_warp_bytes(cap, precision == NEGF_FP64 ? (int)sizeof(double) : (int)sizeof(float));
  const int wmax = alias_warps_max(max_K);
  int warps = 8;
  while (warps > 1 && per_warp * warps > 96 * 1024) --warps;
  if (warps_req > 0) warps = warps_req < wmax ? warps_req : wmax;
  const size_t smem = per_warp * warps;
  if (smem > 220 * 1024) return cudaErrorInvalidValue;   // rows beyond the shared-memory path
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t blocks = (total_jobs + warps - 1) / warps;
  const uint32_t cap_blocks = (uint32_t)sms * 32;
  if (blocks > cap_blocks) blocks = cap_blocks;
  // sum-rule tolerance: FP64 weights agree with A to rounding; FP32 propagation to ~1e-5
  const double tol = precision == NEGF_FP64 ? 1e-8 : 1e-3;
  cudaError_t e;
  if (precision == NEGF_FP64) {
    e = cudaFuncSetAttribute(alias_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    alias_kernel<double><<<blocks, warps * 32, smem, s>>>(
        d_tasks, n_tasks, total_jobs, cap, tol, static_cast<const double*>(d_weights), d_rowsum,
        d_mode_w, d_tab, d_mode_tab, d_err);
  } else {
    e = cudaFuncSetAttribute(alias_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    alias_kernel<float><<<blocks, warps * 32, smem, s>>>(
        d_tasks, n_tasks, total_jobs, cap, tol, static_cast<const float*>(d_weights), d_rowsum,
        d_mode_w, d_tab, d_mode_tab, d_err);
  }
  return cudaGetLastError();
}

}  // namespace negf
