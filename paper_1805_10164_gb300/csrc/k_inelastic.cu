// Walks with inelastic Buttiker probes: Step 6' followed by the energy draw of Step 7'
// (Sec. II.F, Eq. draw_E_last).
//
// A walker is injected from lead p at the energy of its task (Step 4, the task's mode alias
// row) and carries its current energy e with its table row.  Philox4x32-10 block b of walker
// wid has counter (b, wid_lo, wid_hi, task) and key (seed_lo, seed_hi), task the injection
// task's number: block 0 is the injection draw (words x0, x1 over the W modes); block s >= 1 is
// transition s: words (x0, x1) draw the next index from the row at energy e (alias over the
// K = n + 2 columns, leads n and n + 1), and when that is a site j, words (x2, x3) draw the
// next energy e' from the energy row (j, e) built by energy_alias_kernel
// (w_e' K(E_e' - E_e) A_jj(E_e'), the model's lambda~ of Eq. condition4_buttiker).  A draw with
// words (x, y) over a K-entry row takes c = (x K) >> 32 and keeps c if y < thr[c], else
// alias[c].  Drawing a lead ends the walk; its count goes to the injection task, so that
// T_qp(E_0) = c_p(E_0) P(q | p, E_0) as for elastic walks.  One walker per thread over a
// persistent grid; counts per task in shared memory (tasks of the launch window), added to the
// global tally once per block.
#include <cuda_runtime.h>

#include "negf_internal.cuh"
#include "philox.cuh"

namespace negf {
namespace {

constexpr int kThreads = 256;
constexpr int kFields = NEGF_TALLY_FIELDS;   // done, absorbed L, absorbed R, truncated, steps
constexpr int kWindow = 1024;                // injection tasks per launch (40 KB shared tally)

// 64-bit counters in shared memory as (lo, hi) words: each addition carries its own overflow
__device__ __forceinline__ void add64(unsigned* lohi, unsigned v) {
  const unsigned old = atomicAdd(lohi, v);
  if (old + v < old) atomicAdd(lohi + 1, 1u);
}

__device__ __forceinline__ uint32_t alias_draw(uint64_t e, uint32_t c, uint32_t y) {
  return y < (uint32_t)e ? c : (uint32_t)(e >> 32);
}

__global__ void __launch_bounds__(kThreads) inelastic_walk_kernel(
    const TaskDesc* __restrict__ tasks, int task0, int n_tasks,
    const EnergyDesc* __restrict__ edesc, const uint64_t* __restrict__ tab,
    const uint64_t* __restrict__ mode_tab, const double* __restrict__ cvals,
    const uint64_t* __restrict__ etab, int start_lead, PhiloxKey key, uint64_t walkers_per_task,
    uint64_t id_offset, uint32_t max_steps, unsigned long long* __restrict__ tally) {
  __shared__ unsigned s_tally[kWindow * kFields * 2];          // [task][field][lo, hi]
  for (int i = threadIdx.x; i < n_tasks * kFields * 2; i += blockDim.x) s_tally[i] = 0u;
  __syncthreads();
  const unsigned long long total = (unsigned long long)n_tasks * walkers_per_task;
  for (unsigned long long g = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; g < total;
       g += (unsigned long long)gridDim.x * blockDim.x) {
    const int tl = (int)(g / walkers_per_task);
    const int t = task0 + tl;
    const TaskDesc& d = tasks[t];
    unsigned* cnt = s_tally + tl * kFields * 2;
    if (!(cvals[2 * t + start_lead] > 0.0)) {            // no open channel: nothing to inject
      add64(cnt, 1u);
      continue;
    }
    const uint64_t w = id_offset + (g - (unsigned long long)tl * walkers_per_task);
    const uint32_t wlo = (uint32_t)w, whi = (uint32_t)(w >> 32), task_id = (uint32_t)t;
    const uint32_t n = (uint32_t)d.n, K = (uint32_t)d.K, W = (uint32_t)d.W;
    const EnergyDesc ed = edesc[t];
    // block 0: the injection mode at the task's energy
    uint4 r = philox4x32_10(make_uint4(0u, wlo, whi, task_id), key);
    const uint32_t c0 = __umulhi(r.x, W);
    const uint32_t mode = alias_draw(__ldg(mode_tab + d.mode_off + start_lead * W + c0), c0, r.y);
    uint32_t row = n + start_lead * W + mode;
    int et = t;                                           // task of the walker's energy
    const uint64_t* trow = tab + d.tab_off;
    uint32_t steps = 0;
    int outcome = -2;
    for (uint32_t b = 1; steps < max_steps; ++b) {
      r = philox4x32_10(make_uint4(b, wlo, whi, task_id), key);
      const uint32_t c = __umulhi(r.x, K);
      const uint32_t j = alias_draw(__ldg(trow + (uint64_t)row * K + c), c, r.y);
      ++steps;
      if (j >= n) {
        outcome = (int)(j - n);
        break;
      }
      // Step 7': the next energy from the energy row (j, e)
      const uint32_t nE = (uint32_t)ed.nE;
      const uint32_t ce = __umulhi(r.z, nE);
      const uint64_t* erow = etab + edesc[et].eoff + (uint64_t)j * nE;
      const uint32_t ep = alias_draw(__ldg(erow + ce), ce, r.w);
      et = ed.t0 + (int)ep;
      trow = tab + tasks[et].tab_off;
      row = j;
    }
    add64(cnt, 1u);
    add64(cnt + 2 * (outcome >= 0 ? 1 + outcome : 3), 1u);
    add64(cnt + 2 * 4, steps);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < n_tasks * kFields; i += blockDim.x) {
    const unsigned long long v =
        (unsigned long long)s_tally[2 * i] | ((unsigned long long)s_tally[2 * i + 1] << 32);
    if (v) atomicAdd(tally + i, v);
  }
}

}  // namespace

cudaError_t launch_inelastic_walk(const TaskDesc* d_tasks, int n_tasks, const EnergyDesc* d_edesc,
                                  const uint64_t* d_tab, const uint64_t* d_mode_tab,
                                  const double* d_c, const uint64_t* d_etab, int start_lead,
                                  uint64_t seed, uint64_t walkers_per_task, uint64_t id_offset,
                                  uint32_t max_steps, uint64_t* d_tally, int sm_count,
                                  cudaStream_t s) {
  if (n_tasks <= 0 || walkers_per_task == 0) return cudaSuccess;
  const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  int per_sm = 0;
  cudaError_t e =
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, inelastic_walk_kernel, kThreads, 0);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  for (int w0 = 0; w0 < n_tasks; w0 += kWindow) {
    const int nt = (n_tasks - w0) < kWindow ? (n_tasks - w0) : kWindow;
    const unsigned long long total = (unsigned long long)nt * walkers_per_task;
    unsigned long long blocks = (unsigned long long)sm_count * per_sm;
    const unsigned long long need = (total + kThreads - 1) / kThreads;
    if (blocks > need) blocks = need;
    inelastic_walk_kernel<<<(unsigned)blocks, kThreads, 0, s>>>(
        d_tasks, w0, nt, d_edesc, d_tab, d_mode_tab, d_c, d_etab, start_lead, key,
        walkers_per_task, id_offset, max_steps,
        reinterpret_cast<unsigned long long*>(d_tally) + (size_t)w0 * kFields);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace negf
