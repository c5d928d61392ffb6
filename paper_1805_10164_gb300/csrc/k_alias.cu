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
#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr uint64_t kSlot = 1ull << 32;

__device__ __forceinline__ uint64_t pack(uint32_t thr, uint32_t alias) {
  return (uint64_t)thr | ((uint64_t)alias << 32);
}

__host__ __device__ inline size_t alias_warp_bytes(int cap) {
  // lc, hc, stage : u64 [cap] | li, hi : u32 [cap]
  return (size_t)cap * (3 * sizeof(uint64_t) + 2 * sizeof(uint32_t));
}

__device__ __forceinline__ uint32_t fixp(float w, int sh) { return small_fixp(w, sh); }
__device__ __forceinline__ uint32_t fixp(double w, int sh) { return __double2uint_rz(ldexp(w, sh)); }

// Build one row.  w: K weights; A: the value the row must sum to (checked when check_A);
// out: K entries; rowsum_out: receives the row sum.
template <typename R>
__device__ void alias_row(const R* __restrict__ w, int K, double A, bool check_A, double tol,
                          uint64_t* __restrict__ out, double* rowsum_out, uint64_t* s_lc,
                          uint64_t* s_hc, uint64_t* s_st, uint32_t* s_li, uint32_t* s_hi,
                          int32_t* err) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const unsigned lt_mask = (1u << lane) - 1u;
  // largest weight (non-finite or negative weights are reported; they are treated as 0)
  R wmax = 0;
  bool bad = false;
  for (int i = lane; i < K; i += 32) {
    const R v = w[i];
    bad |= !(v >= 0) || !isfinite(v);
    if (v > wmax && isfinite(v)) wmax = v;
  }
  for (int off = 16; off > 0; off >>= 1) wmax = max(wmax, __shfl_xor_sync(FULL, wmax, off));
  if (__any_sync(FULL, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
  if (!(wmax > 0)) {
    if (lane == 0) *rowsum_out = 0.0;
    if (lane == 0 && check_A && A > 1e-300) atomicOr(err, ERR_ROWSUM);
    for (int i = lane; i < K; i += 32) out[i] = pack(0xffffffffu, (uint32_t)i);
    return;
  }
  int ex = 0;
  frexp((double)wmax, &ex);                   // wmax = f 2^ex, f in [0.5, 1)
  const int sh = 32 - ex;                      // wmax 2^sh in [2^31, 2^32)
  uint64_t T = 0;
  for (int i = lane; i < K; i += 32) {
    const R v = w[i];
    const uint32_t m = (v > 0 && isfinite(v)) ? fixp(v, sh) : 0u;
    s_st[i] = m;
    T += m;
  }
  for (int off = 16; off > 0; off >>= 1) T += __shfl_xor_sync(FULL, T, off);
  // row sum: FP64 weights are summed in FP64 (fixed order: lane-strided, tree to lane 0);
  // FP32 weights use the exact fixed-point sum (within K 2^-32 of the largest weight)
  double total = ldexp((double)T, -sh);
  if (sizeof(R) == 8) {
    double part = 0.0;
    for (int i = lane; i < K; i += 32) part += (double)w[i];
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(FULL, part, off);
    total = __shfl_sync(FULL, part, 0);
  }
  if (lane == 0) {
    *rowsum_out = total;
    if (check_A && A > 1e-300 && fabs(total - A) > tol * A) atomicOr(err, ERR_ROWSUM);
  }
  // u_i = floor(m_i K 2^32 / T) = (m_i K) (2^94 / T) / 2^62, with the 128-bit product
  const uint64_t target = (uint64_t)K << 32;
  const uint64_t rcp = (uint64_t)(ldexp(1.0, 94) / (double)T);   // < 2^63 since T >= 2^31
  uint64_t usum = 0, umax = 0;
  int imax = 0x7fffffff;
  __syncwarp();
  for (int i = lane; i < K; i += 32) {
    const uint64_t q = s_st[i] * (uint64_t)K;
    const uint64_t hi = __umul64hi(q, rcp), lo = q * rcp;
    uint64_t u = (hi << 2) | (lo >> 62);
    if (u > target) u = target;
    s_st[i] = u;
    usum += u;
    if (u > umax || (u == umax && i < imax)) { umax = u; imax = i; }
  }
  for (int off = 16; off > 0; off >>= 1) {
    usum += __shfl_xor_sync(FULL, usum, off);
    const uint64_t om = __shfl_xor_sync(FULL, umax, off);
    const int oi = __shfl_xor_sync(FULL, imax, off);
    if (om > umax || (om == umax && oi < imax)) { umax = om; imax = oi; }
  }
  __syncwarp();
  if (lane == 0) s_st[imax] += target - usum;   // two's-complement add of a signed remainder
  __syncwarp();
  // integer prefix sums of deficits (lights) and excesses (heavies), index order
  int nl = 0, nh = 0;
  uint64_t runl = 0, runh = 0;
  for (int base = 0; base < K; base += 32) {
    const int i = base + lane;
    const bool valid = i < K;
    const uint64_t u = valid ? s_st[i] : 0ull;
    const bool heavy = valid && u >= kSlot;
    const bool light = valid && !heavy;
    const unsigned bh = __ballot_sync(FULL, heavy);
    const unsigned bl = __ballot_sync(FULL, light);
    uint64_t dl = light ? kSlot - u : 0ull;
    uint64_t dh = heavy ? u - kSlot : 0ull;
    for (int off = 1; off < 32; off <<= 1) {
      const uint64_t ol = __shfl_up_sync(FULL, dl, off);
      const uint64_t oh = __shfl_up_sync(FULL, dh, off);
      if (lane >= off) { dl += ol; dh += oh; }
    }
    if (light) {
      const int r = nl + __popc(bl & lt_mask);
      s_lc[r] = runl + dl;
      s_li[r] = (uint32_t)i;
    }
    if (heavy) {
      const int j = nh + __popc(bh & lt_mask);
      s_hc[j] = runh + dh;
      s_hi[j] = (uint32_t)i;
    }
    runl += __shfl_sync(FULL, dl, 31);
    runh += __shfl_sync(FULL, dh, 31);
    nl += __popc(bl);
    nh += __popc(bh);
  }
  __syncwarp();
  if (nh == 0) {   // cannot happen when sum(u) == K 2^32; keep the row drawable anyway
    for (int i = lane; i < K; i += 32) out[i] = pack(0xffffffffu, (uint32_t)i);
    return;
  }
  // lights: alias = heavy whose interval [Ec_{j-1}, Ec_j) contains the light's start
  for (int r = lane; r < nl; r += 32) {
    const uint64_t st = r == 0 ? 0ull : s_lc[r - 1];
    int lo = 0, hi = nh;                         // first j with Ec_j > st
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_hc[mid] > st) hi = mid; else lo = mid + 1;
    }
    if (lo >= nh) lo = nh - 1;
    const uint32_t i = s_li[r];
    s_st[i] = pack((uint32_t)s_st[i], s_hi[lo]);
  }
  // heavies
  for (int j = lane; j < nh; j += 32) {
    const uint32_t i = s_hi[j];
    uint64_t e = pack(0xffffffffu, i);
    const uint64_t Ej = s_hc[j];
    if (j < nh - 1 && Ej > 0) {
      int lo = 0, hi = nl;                       // first r with Lc_r >= Ej
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (s_lc[mid] >= Ej) hi = mid; else lo = mid + 1;
      }
      if (lo < nl) {
        const uint64_t used = s_lc[lo] - Ej;     // consumed beyond the excess, <= 2^32
        if (used > 0) e = pack((uint32_t)(kSlot - used), s_hi[j + 1]);
      }
    }
    s_st[i] = e;
  }
  __syncwarp();
  for (int i = lane; i < K; i += 32) out[i] = s_st[i];
}

template <typename R>
__global__ void alias_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t total_jobs,
                             int cap, double tol, const R* __restrict__ weights,
                             double* __restrict__ rowsum, const double* __restrict__ mode_w,
                             uint64_t* __restrict__ tab, uint64_t* __restrict__ mode_tab,
                             int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  unsigned char* base = smem_raw + (size_t)warp * alias_warp_bytes(cap);
  uint64_t* s_lc = reinterpret_cast<uint64_t*>(base);
  uint64_t* s_hc = s_lc + cap;
  uint64_t* s_st = s_hc + cap;
  uint32_t* s_li = reinterpret_cast<uint32_t*>(s_st + cap);
  uint32_t* s_hi = s_li + cap;
  for (uint32_t job = blockIdx.x * nwarps + warp; job < total_jobs; job += gridDim.x * nwarps) {
    int lo = 0, hi = n_tasks - 1;                // task owning this job
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].row_base <= job) lo = mid; else hi = mid - 1;
    }
    const TaskDesc& d = tasks[lo];
    const int row = (int)(job - d.row_base);
    const double A = rowsum[job];                 // <i|A|i> (rows) or c_p (mode rows)
    if (row < d.rows) {
      alias_row<R>(weights + d.wt_off + (uint64_t)row * d.K, d.K, A, true, tol,
                   tab + d.tab_off + (uint64_t)row * d.K, rowsum + job, s_lc, s_hc, s_st, s_li,
                   s_hi, err);
    } else {
      const int p = row - d.rows;
      alias_row<double>(mode_w + d.mode_off + p * d.W, d.W, A, true, 1e-9,
                        mode_tab + d.mode_off + p * d.W, rowsum + job, s_lc, s_hc, s_st, s_li,
                        s_hi, err);
    }
    __syncwarp();
  }
}

// One warp per table row of a two-level task.  The row is taken in chunks of 32 slices: the
// chunk's weights are staged in shared memory by coalesced loads, each lane builds one slice's
// level-1 weight (FP64 sum) and level-2 alias row in shared memory, and the chunk's entries
// (32 consecutive level-2 rows) leave by coalesced stores.
constexpr int kTlWarps = 4;
constexpr int kTlPitch = 65;                         // padded slice pitch (W <= 64)

template <typename R>
__global__ void __launch_bounds__(32 * kTlWarps) two_level_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs, R* __restrict__ weights,
    uint64_t* __restrict__ tab, int32_t* err) {
  extern __shared__ __align__(16) unsigned char tl_smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* so = reinterpret_cast<uint64_t*>(tl_smem) + (size_t)warp * 32 * kTlPitch;
  R* sw = reinterpret_cast<R*>(reinterpret_cast<uint64_t*>(tl_smem) + (size_t)kTlWarps * 32 * kTlPitch) +
          (size_t)warp * 32 * kTlPitch;
  const uint32_t job = blockIdx.x * kTlWarps + warp;
  if (job >= n_jobs) return;
  int lo = 0, hi = n_tasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (tasks[mid].row_base <= job) lo = mid; else hi = mid - 1;
  }
  const TaskDesc& d = tasks[lo];
  if (d.layout != NEGF_LAYOUT_TWO_LEVEL) return;
  const int row = (int)(job - d.row_base);
  if (row >= d.rows) return;
  const int W = d.W, L = d.L, n = d.n;
  const R* wr = weights + d.wt_off + (uint64_t)row * d.K;
  R* l1 = weights + d.l1w_off + (uint64_t)row * (L + 2);
  uint64_t* l2 = tab + d.tab_off + (uint64_t)row * n;
  bool ok = true;
  for (int k0 = 0; k0 < L; k0 += 32) {
    const int ns = min(32, L - k0);
    const R* wc = wr + (uint64_t)k0 * W;
    for (int i = lane; i < ns * W; i += 32) sw[(i / W) * kTlPitch + (i % W)] = wc[i];
    __syncwarp();
    if (lane < ns) {
      const R* ws = sw + lane * kTlPitch;
      double S = 0.0;
      ok &= alias_small_inplace<R>(W, [&](int i) { return ws[i]; }, so + lane * kTlPitch, &S);
      if (sizeof(R) == 8) {            // FP64 tables: the FP64 sum
        S = 0.0;
        for (int a = 0; a < W; ++a) S += (double)ws[a];
      }
      l1[k0 + lane] = (R)S;            // FP32 tables: the exact fixed-point sum
    }
    __syncwarp();
    uint64_t* oc = l2 + (uint64_t)k0 * W;
    for (int i = lane; i < ns * W; i += 32) oc[i] = so[(i / W) * kTlPitch + (i % W)];
    __syncwarp();
  }
  if (lane == 0) {
    l1[L] = wr[n];
    l1[L + 1] = wr[n + 1];
  }
  if (__any_sync(0xffffffffu, !ok) && lane == 0) atomicOr(err, ERR_NONFINITE);
}

}  // namespace

cudaError_t launch_two_level_split(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs,
                                   int precision, void* d_weights, uint64_t* d_tab,
                                   int32_t* d_err, cudaStream_t s) {
  if (n_jobs == 0 || n_tasks == 0) return cudaSuccess;
  const unsigned blocks = (n_jobs + kTlWarps - 1) / kTlWarps;
  const size_t stage = (size_t)kTlWarps * 32 * kTlPitch;      // entries per staging array
  cudaError_t e;
  if (precision == NEGF_FP64) {
    const size_t smem = stage * (sizeof(uint64_t) + sizeof(double));
    e = cudaFuncSetAttribute(two_level_kernel<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    two_level_kernel<double><<<blocks, 32 * kTlWarps, smem, s>>>(
        d_tasks, n_tasks, n_jobs, static_cast<double*>(d_weights), d_tab, d_err);
  } else {
    const size_t smem = stage * (sizeof(uint64_t) + sizeof(float));
    e = cudaFuncSetAttribute(two_level_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    two_level_kernel<float><<<blocks, 32 * kTlWarps, smem, s>>>(
        d_tasks, n_tasks, n_jobs, static_cast<float*>(d_weights), d_tab, d_err);
  }
  return cudaGetLastError();
}

int alias_warps_max(int max_K) {
  const int cap = max_K < 64 ? 64 : max_K;
  const size_t per_warp = alias_warp_bytes(cap);
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
  const size_t per_warp = alias_warp_bytes(cap);
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
