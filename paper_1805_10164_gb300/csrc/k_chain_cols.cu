// Block columns of G with one column per lane (complex64, W <= 32, no gradient outputs).
//
// Sec. III.B obtains the columns of G^r a walker needs by RGF; here each table row's column is
// produced once per task by the recursion
//   G_{k,m} = -t g^L_k G_{k+1,m}  (k < m, direction 0),   G_{k,m} = -t g^R_k G_{k-1,m}  (k > m)
// started from the diagonal block G_mm (or G_mm Phi for the two injection columns), and each
// block is emitted at once as Step 6' weights gamma_(k,a) |G_(k,a),(m,b)|^2 (Eq.
// draw_i_simult), plus the lead weight sum_nu Gamma_nu |(Phi^T G)_nu|^2 at the end slices.
//
// The warp of job (task, y0, dir), y0 a multiple of Y = max(1, 32 / W), carries the Y W columns
// (y, b), y0 <= y < y0 + Y, b < W, lane = (y - y0) W + b: block columns y < L are site slices,
// y = L, L + 1 the left / right injection columns.  Each lane keeps its column of G_{k,y} in
// registers.  Per step the warp has g_k and eta of slice k in shared memory (brought in by
// asynchronous copies one step ahead, double-buffered), every lane forms its next column
// -t g_k X by broadcast reads, and the step's weights leave through a shared-memory transpose so
// that each row's W entries are written together.  One warp per CTA, so that the jobs that do
// no work (y not a multiple of Y) free their slot at once.
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

// kWide: W <= 32 with two g_k buffers filled by asynchronous copies; else W <= 16, one buffer
template <bool kWide>
struct ChainColsSmem {
  float4 g[kWide ? 2 : 1][kWide ? 32 * 16 : 16 * 8];   // g_k, rows padded to an even length
  float eta[kWide ? 2 : 1][32];
  float stage[32 * (kWide ? 33 : 17)];                   // lane l's W weights at l (W + 1)
  int row[32];                 // weight row of lane l's column, -1 for none
  int m0[32];                  // start slice of lane l's column
};

__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int W>
__device__ __forceinline__ void chain_cols_body(const TaskDesc& d, int y0, int dir,
                                                const float* __restrict__ eta_all,
                                                const float* __restrict__ phig,
                                                const double* __restrict__ gam,
                                                const cf* __restrict__ gL,
                                                const cf* __restrict__ gR,
                                                const cf* __restrict__ start,
                                                float* __restrict__ weights,
                                                ChainColsSmem<(W > 16)>* smp) {
  auto& sm = *smp;
  constexpr int Y = W <= 16 ? 32 / W : 1;
  constexpr int Wp = (W + 1) & ~1;                 // padded row of g_k in shared memory
  constexpr int kEm = (Y * W * W + 31) / 32;       // weight writes per lane per step
  constexpr bool kEmPre = kEm <= 8;                // their offsets kept in registers
  const int lane = threadIdx.x & 31;
  const int L = d.L, n = d.n, K = d.K;
  const int y = y0 + lane / W, b = lane % W;
  const bool has = lane < Y * W && y < L + 2;
  const bool inj = y >= L;
  const int m0 = inj ? (y == L ? 0 : L - 1) : y;
  const bool live = has && !(dir == 1 && m0 == L - 1);
  sm.row[lane] = live ? (inj ? n + (y - L) * W : m0 * W) + b : -1;
  sm.m0[lane] = m0;
  const unsigned FULL = 0xffffffffu;
  if (!__any_sync(FULL, live)) return;
  // this lane's column of the start block: X[a] = start[y][a][b]
  cf X[W];
#pragma unroll
  for (int a = 0; a < W; ++a)
    X[a] = live ? start[d.start_off + ((uint64_t)y * W + a) * W + b] : cf{0.f, 0.f};
  const float* eta = eta_all + d.onsite_off / 2;      // FP32 copy of eta
  float* wrow = weights + d.wt_off;
  const float mt = (float)(-d.t);
  const cf* gsrc = dir == 0 ? gL : gR;
  // steps: dir 0 from the largest start slice down to 0 (a lane emits its start block at k = m0
  // and propagates below it); dir 1 from the smallest start slice + 1 up to L - 1
  int k0, k1, step;
  if (dir == 0) {
    k0 = (int)__reduce_max_sync(FULL, live ? (unsigned)m0 : 0u);
    k1 = -1;
    step = -1;
  } else {
    k0 = (int)__reduce_min_sync(FULL, live ? (unsigned)m0 : 0x7fffffffu) + 1;
    k1 = L;
    step = 1;
  }
  auto in_range = [&](int k) { return k != k1 && k >= 0 && k < L; };
  // W <= 16: g_k and eta of the next slice are held in registers one step ahead and stored to
  // buffer 0 at the top of the step; wider blocks come by asynchronous copies into the other of
  // two buffers
  constexpr bool kRegPre = W <= 16;
  constexpr int kPre = kRegPre ? (W * W + 31) / 32 : 1;
  cf gpre[kPre];
  float epre = 0.f;
  auto fetch_reg = [&](int k) {
    const cf* gk = gsrc + d.g_off + (uint64_t)k * W * W;
#pragma unroll
    for (int i = 0; i < kPre; ++i) {
      const int idx = lane + 32 * i;
      if (idx < W * W) gpre[i] = gk[idx];
    }
    if (lane < W) epre = eta[k * W + lane];
  };
  auto fetch = [&](int k, int buf) {
    const cf* gk = gsrc + d.g_off + (uint64_t)k * W * W;
    cf* sg = reinterpret_cast<cf*>(sm.g[kRegPre ? 0 : buf]);
    for (int idx = lane; idx < W * W; idx += 32) {
      const int a = idx / W, c = idx - a * W;
      cp_async8(sg + a * Wp + c, gk + idx);
    }
    if (lane < W) cp_async4(&sm.eta[kRegPre ? 0 : buf][lane], eta + k * W + lane);
    cp_async_commit();
  };
  if (in_range(k0)) {
    if (kRegPre) fetch_reg(k0);
    else fetch(k0, 0);
  }
  __syncwarp();
  // this lane's share of each step's weight writes (elements e = lane + 32 i of the (lane l,
  // entry a) grid, fixed over the steps): row offset, start slice and staging slot
  uint32_t em_off[kEmPre ? kEm : 1];
  int em_m0[kEmPre ? kEm : 1];
  if (kEmPre) {
#pragma unroll
    for (int i = 0; i < (kEmPre ? kEm : 1); ++i) {
      const int e = lane + 32 * i;
      const int l = e / W, a = e - l * W;
      const int r = e < Y * W * W ? sm.row[l] : -1;
      em_off[i] = r >= 0 ? (uint32_t)r * (uint32_t)K + (uint32_t)a : 0u;
      em_m0[i] = r >= 0 ? sm.m0[l] : (dir == 0 ? -1 : 1 << 30);
    }
  }
  int buf = 0;
  for (int k = k0; in_range(k); k += step) {
    if (kRegPre) {
      cf* sg = reinterpret_cast<cf*>(sm.g[0]);
#pragma unroll
      for (int i = 0; i < kPre; ++i) {
        const int idx = lane + 32 * i;
        if (idx < W * W) {
          const int a = idx / W, c = idx - a * W;
          sg[a * Wp + c] = gpre[i];
        }
      }
      if (lane < W) sm.eta[0][lane] = epre;
      if (in_range(k + step)) fetch_reg(k + step);
      __syncwarp();
    } else {
      cp_async_wait_all();
      __syncwarp();
      if (in_range(k + step)) fetch(k + step, buf ^ 1);
    }
    const float4* g4 = sm.g[kRegPre ? 0 : buf];
    const float* seta = sm.eta[kRegPre ? 0 : buf];
    const bool act = live && (dir == 0 ? k <= m0 : k > m0);
    const bool prop = live && (dir == 0 ? k < m0 : k > m0);
    if (prop) {
      cf Xn[W];
#pragma unroll
      for (int a = 0; a < W; ++a) {
        cf acc{0.f, 0.f};
#pragma unroll
        for (int q = 0; q < Wp / 2; ++q) {
          const float4 v = g4[(a * Wp) / 2 + q];
          acc = acc + cf{v.x, v.y} * X[2 * q];
          if (2 * q + 1 < W) acc = acc + cf{v.z, v.w} * X[2 * q + 1];
        }
        Xn[a] = cf{mt * acc.x, mt * acc.y};
      }
#pragma unroll
      for (int a = 0; a < W; ++a) X[a] = Xn[a];
    }
    if (act) {
#pragma unroll
      for (int a = 0; a < W; ++a) sm.stage[lane * (W + 1) + a] = seta[a] * norm2(X[a]);
      if (k == 0 || k == L - 1) {
        // lead weight: sum_nu Gamma_nu |(Phi^T X)_nu|^2
        float sum = 0.f;
        for (int nu = 0; nu < W; ++nu) {
          cf acc{0.f, 0.f};
#pragma unroll
          for (int a = 0; a < W; ++a) acc = acc + phig[d.phi_off + a * W + nu] * X[a];
          sum += (float)gam[d.lead_off + nu] * norm2(acc);
        }
        const int r = sm.row[lane];
        if (k == 0) wrow[(uint64_t)r * K + n + 0] = sum;
        if (k == L - 1) wrow[(uint64_t)r * K + n + 1] = sum;
      }
    }
    __syncwarp();
    // the step's weights: lane l's W entries go to row(l), columns k W .. k W + W - 1
    if (kEmPre) {
#pragma unroll
      for (int i = 0; i < (kEmPre ? kEm : 1); ++i) {
        const bool al = dir == 0 ? k <= em_m0[i] : k > em_m0[i];
        const int e = lane + 32 * i;
        const int l = e / W, a = e - l * W;
        if (al) wrow[(uint64_t)em_off[i] + (uint32_t)(k * W)] = sm.stage[l * (W + 1) + a];
      }
    } else {
#pragma unroll
      for (int i = 0; i < kEm; ++i) {
        const int e = lane + 32 * i;
        const int l = e / W, a = e - l * W;
        if (e < Y * W * W) {
          const int r = sm.row[l], ml = sm.m0[l];
          const bool al = r >= 0 && (dir == 0 ? k <= ml : k > ml);
          if (al) wrow[(uint64_t)r * K + k * W + a] = sm.stage[l * (W + 1) + a];
        }
      }
    }
    __syncwarp();
    if (!kRegPre) buf ^= 1;
  }
  cp_async_wait_all();
}

template <int W>
__device__ __forceinline__ void chain_cols_width(const TaskDesc& d, int y, int dir,
                                                 const float* eta_all, const float* phig,
                                                 const double* gam, const cf* gL, const cf* gR,
                                                 const cf* start, float* weights,
                                                 ChainColsSmem<(W > 16)>* sm) {
  constexpr int Y = W <= 16 ? 32 / W : 1;
  if (y % Y != 0) return;
  chain_cols_body<W>(d, y, dir, eta_all, phig, gam, gL, gR, start, weights, sm);
}

// last task whose first job index (`first(t)`) is <= job
template <typename F>
__device__ __forceinline__ int find_task_cc(int n_tasks, uint32_t job, F first) {
  int lo = 0, hi = n_tasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first(mid) <= job) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Jobs (task, y, dir) as for the other block-column kernels: job = 2 (col_base + y) + dir.
// kWide: the instantiation for 16 < W <= 32 (more registers per thread); the other takes
// W <= 16.  Each skips the tasks of the other.
template <bool kWide>
__global__ void __launch_bounds__(32) chain_cols_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs,
    const float* __restrict__ eta_all, const float* __restrict__ phig,
    const double* __restrict__ gam, const cf* __restrict__ gL, const cf* __restrict__ gR,
    const cf* __restrict__ start, float* __restrict__ weights) {
  __shared__ ChainColsSmem<kWide> s_cc;
  const uint32_t job = blockIdx.x;
  if (job >= n_jobs) return;
  const int task = find_task_cc(n_tasks, job, [&](int t) { return 2 * tasks[t].col_base; });
  const TaskDesc d = tasks[task];
  if (d.fused || d.cta_chain) return;
  const uint32_t local = job - 2 * d.col_base;
  const int y = (int)(local >> 1), dir = (int)(local & 1);
#define NEGF_CC_CASE(w)                                                                       \
  case w:                                                                                     \
    chain_cols_width<w>(d, y, dir, eta_all, phig, gam, gL, gR, start, weights, &s_cc);        \
    break;
  if constexpr (!kWide) {
    switch (d.W) {
      NEGF_CC_CASE(1) NEGF_CC_CASE(2) NEGF_CC_CASE(3) NEGF_CC_CASE(4)
      NEGF_CC_CASE(5) NEGF_CC_CASE(6) NEGF_CC_CASE(7) NEGF_CC_CASE(8)
      NEGF_CC_CASE(9) NEGF_CC_CASE(10) NEGF_CC_CASE(11) NEGF_CC_CASE(12)
      NEGF_CC_CASE(13) NEGF_CC_CASE(14) NEGF_CC_CASE(15) NEGF_CC_CASE(16)
      default: break;
    }
  } else {
    switch (d.W) {
      NEGF_CC_CASE(17) NEGF_CC_CASE(18) NEGF_CC_CASE(19) NEGF_CC_CASE(20)
      NEGF_CC_CASE(21) NEGF_CC_CASE(22) NEGF_CC_CASE(23) NEGF_CC_CASE(24)
      NEGF_CC_CASE(25) NEGF_CC_CASE(26) NEGF_CC_CASE(27) NEGF_CC_CASE(28)
      NEGF_CC_CASE(29) NEGF_CC_CASE(30) NEGF_CC_CASE(31) NEGF_CC_CASE(32)
      default: break;
    }
  }
#undef NEGF_CC_CASE
}

}  // namespace

cudaError_t launch_chain_cols(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs, int max_W,
                              const float* d_eta32, const float* d_phi32, const double* d_gam,
                              const cf* d_gL, const cf* d_gR, const cf* d_start, float* d_w,
                              cudaStream_t s) {
  if (n_jobs == 0 || n_tasks == 0) return cudaSuccess;
  chain_cols_kernel<false><<<n_jobs, 32, 0, s>>>(d_tasks, n_tasks, n_jobs, d_eta32, d_phi32,
                                                 d_gam, d_gL, d_gR, d_start, d_w);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || max_W <= 16) return e;
  chain_cols_kernel<true><<<n_jobs, 32, 0, s>>>(d_tasks, n_tasks, n_jobs, d_eta32, d_phi32,
                                                d_gam, d_gL, d_gR, d_start, d_w);
  return cudaGetLastError();
}

}  // namespace negf
