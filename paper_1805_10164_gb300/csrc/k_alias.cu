// Alias-table construction for the Step 6' categorical draw.
//
// Sec. III.B draws the next index by a cumulative sum and a search (O(K) per step).  The walk
// here uses Walker's alias method (one table entry per draw), so each row of weights is turned
// into K slots (threshold, alias).  One warp builds one row with a parallel "sweep" alias
// construction (in the spirit of Hubschle-Schneider and Sanders, "Parallel weighted random
// sampling", ESA 2019), written from this derivation:
//
//   q_i = w_i K / sum(w).  Light items (q < 1) in index order carry deficits 1 - q with
//   inclusive prefix sums Lc_r; heavy items (q >= 1) in index order carry excesses q - 1 with
//   inclusive prefix sums Ec_j.  Heavy j owns the interval [Ec_{j-1}, Ec_j) of the deficit line.
//   * light r keeps prob q and aliases the heavy whose interval contains its start Lc_{r-1};
//   * heavy j (not the last) is consumed past its excess by the light interval (Lc_{r-1}, Lc_r]
//     that contains Ec_j; its own slot keeps prob 1 - (Lc_r - Ec_j) and aliases heavy j+1.
//     If no light interval contains Ec_j (Ec_j == 0 or beyond the deficit total) it is full;
//   * the last heavy is full.
//   Every item then receives exactly mass q_i / K (each heavy gets its own slot remainder plus
//   the deficits of the slots aliasing it, a contiguous stretch of the deficit line).
// Slots store thr = floor(prob 2^32) (full slots: thr = 2^32 - 1 and alias = self).
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr int kWarpsMax = 8;

__device__ __forceinline__ uint64_t pack(uint32_t thr, uint32_t alias) {
  return (uint64_t)thr | ((uint64_t)alias << 32);
}

__device__ __forceinline__ uint32_t to_thr(double prob) {
  // prob in [0, 1): floor(prob * 2^32) fits in 32 bits
  double x = floor(prob * 4294967296.0);
  if (x < 0.0) x = 0.0;
  if (x > 4294967295.0) x = 4294967295.0;
  return (uint32_t)x;
}

template <typename R>
__device__ __forceinline__ double load_w(const R* p, int i) { return (double)p[i]; }

// Build one row.  w: K weights; total: their FP64 sum; out: K entries.  s_*: per-warp smem
// arrays of capacity K.
template <typename R>
__device__ void alias_row(const R* __restrict__ w, int K, double total, uint64_t* __restrict__ out,
                          double* s_lc, int* s_li, double* s_hc, int* s_hi, int32_t* err) {
  const int lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  if (!(total > 0.0) || !isfinite(total)) {
    for (int i = lane; i < K; i += 32) out[i] = pack(0xffffffffu, (uint32_t)i);
    return;
  }
  const double scale = (double)K / total;
  int nl = 0, nh = 0;
  double runl = 0.0, runh = 0.0;
  const unsigned lt_mask = (1u << lane) - 1u;
  for (int base = 0; base < K; base += 32) {
    const int i = base + lane;
    double q = 0.0;
    bool valid = i < K;
    if (valid) q = load_w(w, i) * scale;
    const bool heavy = valid && q >= 1.0;
    const bool light = valid && !heavy;
    const unsigned bh = __ballot_sync(FULL, heavy);
    const unsigned bl = __ballot_sync(FULL, light);
    double dl = light ? 1.0 - q : 0.0;
    double dh = heavy ? q - 1.0 : 0.0;
    // inclusive warp scans (fixed order -> deterministic)
    for (int off = 1; off < 32; off <<= 1) {
      const double ol = __shfl_up_sync(FULL, dl, off);
      const double oh = __shfl_up_sync(FULL, dh, off);
      if (lane >= off) { dl += ol; dh += oh; }
    }
    if (light) {
      const int r = nl + __popc(bl & lt_mask);
      s_lc[r] = runl + dl;
      s_li[r] = i;
    }
    if (heavy) {
      const int j = nh + __popc(bh & lt_mask);
      s_hc[j] = runh + dh;
      s_hi[j] = i;
    }
    runl += __shfl_sync(FULL, dl, 31);
    runh += __shfl_sync(FULL, dh, 31);
    nl += __popc(bl);
    nh += __popc(bh);
  }
  __syncwarp();
  if (nh == 0) {
    // every q rounded just below 1 (sum q = K in exact arithmetic), i.e. a uniform row:
    // full slots realise it to rounding accuracy
    for (int i = lane; i < K; i += 32) out[i] = pack(0xffffffffu, (uint32_t)i);
    return;
  }
  // lights: alias = heavy whose interval [Ec_{j-1}, Ec_j) contains the light's start
  for (int r = lane; r < nl; r += 32) {
    const double start = r == 0 ? 0.0 : s_lc[r - 1];
    int lo = 0, hi = nh;                    // first j with Ec_j > start
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (s_hc[mid] > start) hi = mid; else lo = mid + 1;
    }
    if (lo >= nh) lo = nh - 1;
    const int i = s_li[r];
    const double q = load_w(w, i) * scale;
    out[i] = pack(to_thr(q), (uint32_t)s_hi[lo]);
  }
  // heavies
  for (int j = lane; j < nh; j += 32) {
    const int i = s_hi[j];
    uint64_t e = pack(0xffffffffu, (uint32_t)i);
    if (j < nh - 1) {
      const double Ej = s_hc[j];
      if (Ej > 0.0 && nl > 0) {
        int lo = 0, hi = nl;                // first r with Lc_r >= Ej
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (s_lc[mid] >= Ej) hi = mid; else lo = mid + 1;
        }
        if (lo < nl) {
          const double prob = 1.0 - (s_lc[lo] - Ej);
          if (prob < 1.0) e = pack(to_thr(prob), (uint32_t)s_hi[j + 1]);
        }
      }
    }
    out[i] = e;
  }
}

template <typename R>
__global__ void alias_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t total_jobs,
                             int cap, const R* __restrict__ weights,
                             const double* __restrict__ rowsum, const double* __restrict__ mode_w,
                             uint64_t* __restrict__ tab, uint64_t* __restrict__ mode_tab,
                             int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  double* s_lc = reinterpret_cast<double*>(smem_raw) + (size_t)warp * 2 * cap;
  double* s_hc = s_lc + cap;
  int* s_li = reinterpret_cast<int*>(reinterpret_cast<double*>(smem_raw) + (size_t)nwarps * 2 * cap) +
              (size_t)warp * 2 * cap;
  int* s_hi = s_li + cap;
  for (uint32_t job = blockIdx.x * nwarps + warp; job < total_jobs; job += gridDim.x * nwarps) {
    // task owning this job: last task with row_base <= job
    int lo = 0, hi = n_tasks - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tasks[mid].row_base <= job) lo = mid; else hi = mid - 1;
    }
    const TaskDesc& d = tasks[lo];
    const int row = (int)(job - d.row_base);
    if (row < d.rows) {
      alias_row<R>(weights + d.wt_off + (uint64_t)row * d.K, d.K, rowsum[job],
                   tab + d.tab_off + (uint64_t)row * d.K, s_lc, s_li, s_hc, s_hi, err);
    } else {
      const int p = row - d.rows;
      alias_row<double>(mode_w + d.mode_off + p * d.W, d.W, rowsum[job],
                        mode_tab + d.mode_off + p * d.W, s_lc, s_li, s_hc, s_hi, err);
    }
    __syncwarp();
  }
}

}  // namespace

cudaError_t launch_alias_build(const TaskDesc* d_tasks, int n_tasks, uint32_t total_jobs,
                               int max_K, int precision, const void* d_weights,
                               const double* d_rowsum, const double* d_mode_w,
                               uint64_t* d_tab, uint64_t* d_mode_tab, int32_t* d_err,
                               cudaStream_t s) {
  if (total_jobs == 0) return cudaSuccess;
  const int cap = max_K;
  const size_t per_warp = (size_t)cap * 2 * (sizeof(double) + sizeof(int));
  int warps = kWarpsMax;
  while (warps > 1 && per_warp * warps > 96 * 1024) --warps;
  const size_t smem = per_warp * warps;
  if (smem > 220 * 1024) return cudaErrorInvalidValue;   // rows beyond the smem path
  int dev = 0, sms = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint32_t blocks = (total_jobs + warps - 1) / warps;
  const uint32_t cap_blocks = (uint32_t)sms * 16;
  if (blocks > cap_blocks) blocks = cap_blocks;
  cudaError_t e;
  if (precision == NEGF_FP64) {
    e = cudaFuncSetAttribute(alias_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    alias_kernel<double><<<blocks, warps * 32, smem, s>>>(
        d_tasks, n_tasks, total_jobs, cap, static_cast<const double*>(d_weights), d_rowsum,
        d_mode_w, d_tab, d_mode_tab, d_err);
  } else {
    e = cudaFuncSetAttribute(alias_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    alias_kernel<float><<<blocks, warps * 32, smem, s>>>(
        d_tasks, n_tasks, total_jobs, cap, static_cast<const float*>(d_weights), d_rowsum,
        d_mode_w, d_tab, d_mode_tab, d_err);
  }
  return cudaGetLastError();
}

}  // namespace negf
