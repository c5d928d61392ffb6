// Linear conductance with continuous energies: each walker draws its energy from the thermal
// window Th(E) = -df/dE (Eq. Gqp_expression; the sampling density of Eq. gpq_formula) restricted
// to the span of a wire's energy grid, and walks the Step 6' chain whose transition
// probabilities are interpolated linearly between the two grid energies around it (the
// interpolation of the p_i in the paper's Sec. "Interpolation"): each draw takes the upper grid
// energy's alias table with probability alpha, else the lower one's (an interval where the start
// lead has no open channel at one end walks with the other end's table).  A walker absorbed at
// q = 1 - p scores c(E) = (1 - alpha) c_i + alpha c_{i+1} (Eq. elast_lin_xpq); the tally keeps,
// per grid interval, the absorbed count, sum of a = floor(alpha 2^32) and sum of (a >> 16)^2 in
// integers, from which the host forms the mean and variance of the score exactly.
//
// Random numbers (Philox4x32-10, counter (b, id_lo, id_hi, 0x80000000 | wire)): block 0 -> the
// energy (x0, x1: a 53-bit word v whose CDF value F = F0 + (v + 1/2) 2^-53 window gives the
// interval, found by comparing v with the host's integer thresholds of the grid points, and
// the energy) and the injection table (x2); block 1 -> the injection mode (x0, x1); block
// b >= 2 -> transition b - 1, (x0, x1) on the row (two-level tables: on the level-1 row, and x3
// for the site within a drawn slice) and x2 < a for the table.  One thread per walker
// (grid-stride); the block's tally sits in shared memory and is added to global memory
// once.
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"
#include "philox.cuh"

namespace negf {
namespace {

constexpr int kThermalThreads = 256;

__device__ __forceinline__ void smem_add64(unsigned* lohi, unsigned v) {
  const unsigned old = atomicAdd(lohi, v);
  if (old + v < old) atomicAdd(lohi + 1, 1u);
}
// 64-bit add to a shared counter kept as two 32-bit words
__device__ __forceinline__ void add64(unsigned* lohi, uint64_t v) {
  if (v == 0) return;
  smem_add64(lohi, (unsigned)v);
  if (v >> 32) atomicAdd(lohi + 1, (unsigned)(v >> 32));
}

// kTwo: the grid's tables are two-level (level 1 an alias row over the slices and leads, level 2
// the inverse-CDF blocks of the slices): a transition draws the slice or lead with (x0, x1),
// the table with x2, and the site within the slice with x3 (v = x3 >> 1).
template <bool kTwo>
__global__ void __launch_bounds__(kThermalThreads) thermal_walk_kernel(
    const TaskDesc* __restrict__ tasks, int task0, int M, uint32_t wire,
    const uint64_t* __restrict__ tab, const uint64_t* __restrict__ mode_tab,
    const double* __restrict__ cvals, int p, PhiloxKey key, uint64_t walkers, uint64_t id_offset,
    uint32_t max_steps, double mu, double kT, double F0, double window,
    const unsigned long long* __restrict__ thr, unsigned long long* __restrict__ tally,
    int32_t* __restrict__ t_lead,
    uint32_t* __restrict__ t_steps, int32_t* __restrict__ t_interval, uint32_t* __restrict__ t_a) {
  // shared tally: per interval (absorbed at q, sum a, sum (a >> 16)^2), then absorbed L, R,
  // closed, truncated, steps; each a 64-bit counter kept as two 32-bit words
  extern __shared__ unsigned s_t[];
  const int n_fields = 3 * (M - 1) + 5;
  for (int i = threadIdx.x; i < 2 * n_fields; i += blockDim.x) s_t[i] = 0u;
  __syncthreads();
  const int q = 1 - p;
  const int G0 = 3 * (M - 1);
  const uint32_t ctr3 = 0x80000000u | wire;
  const TaskDesc& d0 = tasks[task0];
  const uint32_t n = (uint32_t)d0.n, W = (uint32_t)d0.W, K = (uint32_t)d0.K;
  const uint32_t L = (uint32_t)d0.L, K1 = L + 2, B2 = (uint32_t)level2_words(d0.W);
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  uint64_t my_abs0 = 0, my_abs1 = 0, my_closed = 0, my_trunc = 0, my_steps = 0;
  for (uint64_t g = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g < walkers; g += stride) {
    const uint64_t wid = id_offset + g;
    const uint32_t lo = (uint32_t)wid, hi = (uint32_t)(wid >> 32);
    const uint4 r0 = philox4x32_10(make_uint4(0u, lo, hi, ctr3), key);
    const uint64_t v = (((uint64_t)r0.x << 32) | r0.y) >> 11;
    const double u = ((double)v + 0.5) * 0x1p-53;
    const double pE = F0 + u * window;                // F(E) of the drawn energy
    // last grid index with F(E_e) <= F(E): the number of grid points 1 .. M - 1 whose
    // threshold v reaches (an integer search, no FP64 compares)
    int lo_i = 0, hi_i = M - 1;
    while (lo_i < hi_i) {
      const int mid = (lo_i + hi_i) >> 1;
      if (thr[mid] <= v) lo_i = mid + 1; else hi_i = mid;
    }
    const int iv = lo_i < M - 2 ? lo_i : M - 2;
    // E - E_i = kT ln(F / (1 - F)) - (E_i - mu): the logarithms in FP32 of F and 1 - F (the
    // latter formed in FP64, so that both keep their relative precision); alpha to ~2^-20
    const float lnr = logf((float)pE) - logf((float)(1.0 - pE));
    const float dE = (float)kT * lnr - (float)(tasks[task0 + iv].E - mu);
    float alpha = dE / (float)(tasks[task0 + iv + 1].E - tasks[task0 + iv].E);
    alpha = alpha < 0.f ? 0.f : (alpha > 1.f ? 1.f : alpha);
    const float af = floorf(alpha * 4294967296.f);
    const uint32_t a = af >= 4294967295.f ? 0xffffffffu : (uint32_t)af;
    // an interval open at both ends mixes the two tables; one open at a single end walks with
    // that end's table alone (a chain without an open lead never absorbs)
    const bool open_lo = cvals[2 * (task0 + iv) + p] > 0.0;
    const bool open_hi = cvals[2 * (task0 + iv + 1) + p] > 0.0;
    const bool mix = open_lo && open_hi;
    auto upper = [&](uint32_t word) { return mix ? word < a : open_hi; };
    const int t = upper(r0.z) ? iv + 1 : iv;
    int outcome = (open_lo || open_hi) ? -3 : -1;
    uint32_t steps = 0;
    if (outcome == -3) {
      const uint4 r1 = philox4x32_10(make_uint4(1u, lo, hi, ctr3), key);
      const uint64_t* mrow = mode_tab + tasks[task0 + t].mode_off + p * W;
      const uint32_t c = __umulhi(r1.x, W);
      const uint64_t e = __ldg(mrow + c);
      uint32_t row = n + p * W + (r1.y < (uint32_t)e ? c : (uint32_t)(e >> 32));
      const uint64_t* tab_lo = tab + tasks[task0 + iv].tab_off;
      const uint64_t* tab_hi = tab + tasks[task0 + iv + 1].tab_off;
      const uint64_t* l1_lo = tab + tasks[task0 + iv].l1_off;
      const uint64_t* l1_hi = tab + tasks[task0 + iv + 1].l1_off;
      for (uint32_t b = 2;; ++b) {
        const uint4 r = philox4x32_10(make_uint4(b, lo, hi, ctr3), key);
        const bool up = upper(r.z);
        uint32_t j;
        if (kTwo) {
          const uint32_t cc = __umulhi(r.x, K1);
          const uint64_t ee = __ldg((up ? l1_hi : l1_lo) + (uint64_t)row * K1 + cc);
          const uint32_t k = r.y < (uint32_t)ee ? cc : (uint32_t)(ee >> 32);
          if (k >= L) {
            j = n + (k - L);
          } else {
            const uint32_t v = r.w >> 1;
            const uint4* blk = reinterpret_cast<const uint4*>(up ? tab_hi : tab_lo) +
                               (((uint64_t)row * L + k) * B2 >> 2);
            uint32_t g = 0;
            if (W > 8) {
              const uint4 q0 = __ldg(blk), q1 = __ldg(blk + 1);
              g = (q0.x <= v) + (q0.y <= v) + (q0.z <= v) + (q0.w <= v) + (q1.x <= v) +
                  (q1.y <= v) + (q1.z <= v) + (q1.w <= v);
              blk += 2 + 2 * g;
            }
            const uint4 o0 = __ldg(blk), o1 = __ldg(blk + 1);
            j = k * W + 8 * g + (o0.x <= v) + (o0.y <= v) + (o0.z <= v) + (o0.w <= v) +
                (o1.x <= v) + (o1.y <= v) + (o1.z <= v) + (o1.w <= v);
          }
        } else {
          const uint32_t cc = __umulhi(r.x, K);
          const uint64_t ee = __ldg((up ? tab_hi : tab_lo) + (uint64_t)row * K + cc);
          j = r.y < (uint32_t)ee ? cc : (uint32_t)(ee >> 32);
        }
        ++steps;
        if (j >= n) { outcome = (int)(j - n); break; }
        if (steps >= max_steps) { outcome = -2; break; }
        row = j;
      }
    }
    // per-interval sums: lanes with the same interval pool theirs and one of them adds them
    {
      const unsigned act = __activemask();
      const int key_iv = outcome == q ? iv : -1;
      const unsigned grp = __match_any_sync(act, key_iv);
      if (key_iv >= 0) {
        const uint32_t a16 = a >> 16, sq = a16 * a16;
        const uint32_t cnt = __popc(grp);
        const uint32_t a_hi = __reduce_add_sync(grp, a >> 16), a_lo = __reduce_add_sync(grp, a & 0xffffu);
        const uint32_t s_hi = __reduce_add_sync(grp, sq >> 16), s_lo = __reduce_add_sync(grp, sq & 0xffffu);
        if ((threadIdx.x & 31) == __ffs(grp) - 1) {
          smem_add64(&s_t[2 * (3 * iv + 0)], cnt);
          add64(&s_t[2 * (3 * iv + 1)], ((uint64_t)a_hi << 16) + a_lo);
          add64(&s_t[2 * (3 * iv + 2)], ((uint64_t)s_hi << 16) + s_lo);
        }
      }
    }
    if (outcome == 0) ++my_abs0;
    else if (outcome == 1) ++my_abs1;
    else if (outcome == -1) ++my_closed;
    else ++my_trunc;
    my_steps += steps;
    if (t_lead) t_lead[g] = outcome;
    if (t_steps) t_steps[g] = steps;
    if (t_interval) t_interval[g] = iv;
    if (t_a) t_a[g] = a;
  }
  add64(&s_t[2 * (G0 + 0)], my_abs0);
  add64(&s_t[2 * (G0 + 1)], my_abs1);
  add64(&s_t[2 * (G0 + 2)], my_closed);
  add64(&s_t[2 * (G0 + 3)], my_trunc);
  add64(&s_t[2 * (G0 + 4)], my_steps);
  __syncthreads();
  for (int f = threadIdx.x; f < n_fields; f += blockDim.x) {
    const unsigned long long v = ((unsigned long long)s_t[2 * f + 1] << 32) | s_t[2 * f];
    if (v) atomicAdd(tally + f, v);
  }
}

}  // namespace

// ---- interval distances of the interpolating sampler's grid (Sec. "Interpolation") ----------
// For consecutive grid energies e, e + 1 of one wire: d_e = the largest of the rows' total-
// variation distances (1/2) sum_b |w_ab(e) / S_a(e) - w_ab(e+1) / S_a(e+1)| (S the FP64 row
// sums; a row of zero sum counts as all zeros), the same between the injection-mode
// distributions of lead p, and |c_e - c_{e+1}| / max(c_e, c_{e+1}).  One warp per (interval,
// row), FP64 sums; d (doubles >= 0, zeroed by the caller) takes the maximum through atomicMax
// on the bit patterns, which order like the values for non-negative doubles.
namespace {
template <typename R>
__global__ void interval_distance_kernel(const TaskDesc* __restrict__ tasks, int task0, int M,
                                         const R* __restrict__ weights,
                                         const double* __restrict__ rowsum,
                                         const double* __restrict__ mode_w,
                                         const double* __restrict__ cvals, int p,
                                         unsigned long long* __restrict__ d) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const TaskDesc& t0 = tasks[task0];
  const int rows = t0.rows, K = t0.K, W = t0.W;
  const int per = rows + 1;                           // the rows, then the modes and c
  if (warp >= (M - 1) * per) return;
  const int e = warp / per, row = warp - e * per;
  const TaskDesc& da = tasks[task0 + e];
  const TaskDesc& db = tasks[task0 + e + 1];
  double tv = 0.0;
  if (row < rows) {
    const double sa = rowsum[da.row_base + row], sb = rowsum[db.row_base + row];
    const double ia = sa > 0.0 ? 1.0 / sa : 0.0, ib = sb > 0.0 ? 1.0 / sb : 0.0;
    const R* wa = weights + da.wt_off + (uint64_t)row * K;
    const R* wb = weights + db.wt_off + (uint64_t)row * K;
    for (int j = lane; j < K; j += 32) tv += fabs((double)wa[j] * ia - (double)wb[j] * ib);
  } else {
    const double* ma = mode_w + da.mode_off + p * W;
    const double* mb = mode_w + db.mode_off + p * W;
    double sa = 0.0, sb = 0.0;
    for (int j = 0; j < W; ++j) {
      sa += ma[j];
      sb += mb[j];
    }
    const double ia = sa > 0.0 ? 1.0 / sa : 0.0, ib = sb > 0.0 ? 1.0 / sb : 0.0;
    for (int j = lane; j < W; j += 32) tv += fabs(ma[j] * ia - mb[j] * ib);
  }
  for (int o = 16; o > 0; o >>= 1) tv += __shfl_down_sync(0xffffffffu, tv, o);
  if (lane == 0) {
    double v = 0.5 * tv;
    if (row == rows) {
      const double ca = cvals[2 * (task0 + e) + p], cb = cvals[2 * (task0 + e + 1) + p];
      const double cm = fmax(ca, cb);
      if (cm > 0.0) v = fmax(v, fabs(ca - cb) / cm);
    }
    atomicMax(d + e, (unsigned long long)__double_as_longlong(v));
  }
}

}  // namespace

cudaError_t launch_interval_distance(const TaskDesc* d_tasks, int task0, int M, int rows,
                                     int precision, const void* d_weights,
                                     const double* d_rowsum, const double* d_mode_w,
                                     const double* d_c, int start_lead, double* d_out,
                                     cudaStream_t s) {
  if (M < 2) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(d_out, 0, sizeof(double) * (M - 1), s);
  if (e != cudaSuccess) return e;
  const uint64_t warps = (uint64_t)(M - 1) * (rows + 1);
  const unsigned blocks = (unsigned)((warps + 7) / 8);
  auto* o = reinterpret_cast<unsigned long long*>(d_out);
  if (precision == NEGF_FP64)
    interval_distance_kernel<double><<<blocks, 256, 0, s>>>(
        d_tasks, task0, M, static_cast<const double*>(d_weights), d_rowsum, d_mode_w, d_c,
        start_lead, o);
  else
    interval_distance_kernel<float><<<blocks, 256, 0, s>>>(
        d_tasks, task0, M, static_cast<const float*>(d_weights), d_rowsum, d_mode_w, d_c,
        start_lead, o);
  return cudaGetLastError();
}

cudaError_t launch_thermal_walk(const TaskDesc* d_tasks, int task0, int M, int wire,
                                const uint64_t* d_tab, const uint64_t* d_mode_tab,
                                const double* d_c, int start_lead, uint64_t seed,
                                uint64_t walkers, uint64_t id_offset, uint32_t max_steps,
                                double mu, double kT, double F0, double window,
                                const unsigned long long* d_thr, unsigned long long* d_tally,
                                int32_t* d_lead, uint32_t* d_steps, int32_t* d_interval,
                                uint32_t* d_a, int sm_count, cudaStream_t s, bool two_level) {
  if (walkers == 0 || M < 2) return cudaSuccess;
  const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  const size_t smem = sizeof(unsigned) * 2 * (size_t)(3 * (M - 1) + 5);
  const uint64_t need = (walkers + kThermalThreads - 1) / kThermalThreads;
  uint64_t blocks = (uint64_t)sm_count * 8;
  if (blocks > need) blocks = need;
  auto kern = two_level ? thermal_walk_kernel<true> : thermal_walk_kernel<false>;
  kern<<<(unsigned)blocks, kThermalThreads, smem, s>>>(
      d_tasks, task0, M, (uint32_t)wire, d_tab, d_mode_tab, d_c, start_lead, key, walkers,
      id_offset, max_steps, mu, kT, F0, window, d_thr, d_tally, d_lead, d_steps, d_interval,
      d_a);
  return cudaGetLastError();
}

}  // namespace negf
