// Block-column propagation of the RGF on the 5th-generation tensor cores (tcgen05, sm_103a) for
// slices of W = 64 sites, fused with the emission of two-level Step 6' tables.
//
// Sec. III.B: with the left-connected blocks g^L_k the block column of start slice m obeys
// G_{k,m} = -t g^L_k G_{k+1,m} for k < m (towards slice 0), and with the right-connected blocks
// G_{k,m} = -t g^R_k G_{k-1,m} for k > m.  Table row b of block column y (site (m, b), or
// injection mode b of a lead, whose start block is G_mm Phi) needs, for every slice k, the
// weights w_a = eta_{k,a} |X_k[a][b]|^2 of X_k = G_{k,m} (Eq. draw_i_simult), written to the
// task's weight rows like the CUDA-core chains (the two-level table build consumes them).
//
// One CTA (4 warps) runs one job: a pair of block columns of one task in one direction.  Thread
// t owns table row b = t mod 64 of column t / 64 of the pair and TMEM lane t.  A step k is the
// complex 64 x 64 product for both columns at once, written as one real GEMM with M = 128
// (2 columns x 64 rows b), N = K' = 128:
//   A[t]  = (Re X_{k+1}[:, b], Im X_{k+1}[:, b])                 TMEM (the previous step's D)
//   B     = [[Re G^T, Im G^T], [-Im G^T, Re G^T]],  G = -t g_k    shared memory, K-major
//   D[t]  = (Re X_k[:, b], Im X_k[:, b])                          TMEM
// 3xTF32: A = A_hi + A_lo and B = B_hi + B_lo with hi the operand rounded to TF32 and lo the
// exact FP32 remainder; D = A_lo B_hi + A_hi B_lo + A_hi B_hi accumulated in FP32 (the dropped
// A_lo B_lo term is below FP32 rounding).  The epilogue reads D, forms the row's 64 weights
// (staged in shared memory and written out as coalesced rows), and stores the TF32 split of D
// back to TMEM as the next step's A.  The slice-0 and slice-(L-1) blocks of every column are
// also written out (edge blocks): lead_weights_kernel forms the lead weights from them.
// Measured on GB300: the tensor-core accumulation carries a systematic relative bias of about
// 1e-7 per step towards smaller magnitudes (sign-independent; unchanged by rounding the TF32
// parts or by accumulating the corrections separately), so weights at the end of chains of
// 300 - 1000 slices are low by 3 - 5e-5 of their row; the CUDA-core FP32 chains stay within
// a few 1e-6.
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"
#include "tcgen05.cuh"

namespace negf {
namespace {

using namespace tc;

constexpr int kW = 64;
constexpr int kThreads = 128;
constexpr uint32_t kTmemCols = 512;           // D: 0..127, A_hi: 128..255, A_lo: 256..383
constexpr uint32_t kColD = 0, kColAh = 128, kColAl = 256;
constexpr size_t kBBytes = 128 * 128 * 4;     // one B split: N' = 128 rows x K' = 128 TF32
constexpr int kWPitch = kThreads + 1;         // padded weight staging [a][row]
constexpr size_t kWBytes = (size_t)kW * kWPitch * 4;
constexpr uint32_t kStagePitch = 528;         // g_k rows staged with a padded pitch (16-B multiple)
constexpr size_t kStageBytes = (size_t)kW * kStagePitch;
constexpr size_t kSmem = 2 * kBBytes + kWBytes + kStageBytes + 64;
constexpr uint32_t kWaitLimit = 1u << 20;     // bounded mbarrier wait (iterations)

// Byte offset of B^T element (n', k') in the core-matrix layout: the 32 core matrices of an
// 8-row group along K are contiguous (LBO = 128 B); groups are 4096 B apart (SBO).
constexpr uint32_t kLBO = 128, kSBO = 4096;

// B = split TF32 embedding of G = mt g (g: 64 x 64 complex64 staged in shared memory, row a
// at stage + a * kStagePitch).  Thread t writes row n' = t of B^T: t < 64 (real output a = t):
// (Re G[a][c])_c, (-Im G[a][c])_c; t >= 64 (imaginary output a = t - 64): (Im G[a][c])_c,
// (Re G[a][c])_c.
__device__ __forceinline__ void build_b(const unsigned char* stage, float mt, unsigned char* bh,
                                        unsigned char* bl, int t) {
  const int a = t & 63, part = t >> 6;
  const float4* grow = reinterpret_cast<const float4*>(stage + (size_t)a * kStagePitch);
  const uint32_t rowb = (uint32_t)(t >> 3) * 32u * 128u + (uint32_t)(t & 7) * 16u;
  auto put = [&](int q, float v0, float v1, float v2, float v3) {
    const uint32_t h0 = to_tf32(v0), h1 = to_tf32(v1), h2 = to_tf32(v2), h3 = to_tf32(v3);
    uint4 hv = make_uint4(h0, h1, h2, h3);
    uint4 lv = make_uint4(__float_as_uint(v0 - __uint_as_float(h0)),
                          __float_as_uint(v1 - __uint_as_float(h1)),
                          __float_as_uint(v2 - __uint_as_float(h2)),
                          __float_as_uint(v3 - __uint_as_float(h3)));
    *reinterpret_cast<uint4*>(bh + rowb + (uint32_t)q * 128u) = hv;
    *reinterpret_cast<uint4*>(bl + rowb + (uint32_t)q * 128u) = lv;
  };
#pragma unroll 4
  for (int c4 = 0; c4 < 16; ++c4) {
    const float4 p = grow[2 * c4], r = grow[2 * c4 + 1];
    const float re0 = mt * p.x, im0 = mt * p.y, re1 = mt * p.z, im1 = mt * p.w;
    const float re2 = mt * r.x, im2 = mt * r.y, re3 = mt * r.z, im3 = mt * r.w;
    if (part == 0) {
      put(c4, re0, re1, re2, re3);
      put(16 + c4, -im0, -im1, -im2, -im3);
    } else {
      put(c4, im0, im1, im2, im3);
      put(16 + c4, re0, re1, re2, re3);
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1) chain_tc_kernel(
    const TaskDesc* __restrict__ tasks, const TcJob* __restrict__ jobs,
    const float* __restrict__ eta32, const cf* __restrict__ gL, const cf* __restrict__ gR,
    const cf* __restrict__ start, float* __restrict__ weights, cf* __restrict__ edge,
    int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  unsigned char* bh = smem;
  unsigned char* bl = smem + kBBytes;
  float* wbuf = reinterpret_cast<float*>(smem + 2 * kBBytes);     // [a][row], pitch kWPitch
  unsigned char* stage = smem + 2 * kBBytes + kWBytes;           // g_k, padded rows
  uint64_t* mbar = reinterpret_cast<uint64_t*>(stage + kStageBytes);   // MMA completion
  uint64_t* mbar_g = mbar + 1;                                     // g_k arrival
  uint32_t* s_tmem = reinterpret_cast<uint32_t*>(mbar + 2);

  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) {
    tmem_alloc(s_tmem, kTmemCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(mbar, 1);
    mbar_init(mbar_g, 1);
    fence_mbar_init();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *s_tmem;
  const uint32_t tlane = tbase + ((uint32_t)(warp * 32) << 16);   // this warp's lane quarter

  const TcJob job = jobs[blockIdx.x];
  const TaskDesc d = tasks[job.task];
  const int L = d.L, n = d.n, K = d.K;
  const int dir = job.dir;
  const int col = tid >> 6, b = tid & 63;
  const int y = col == 0 ? job.y0 : job.y1;
  const bool has = y >= 0;                      // warp-uniform (64 threads per column)
  auto m0_of = [&](int yy) { return yy < L ? yy : (yy == L ? 0 : L - 1); };
  const int m0 = has ? m0_of(y) : 0;
  auto row_of = [&](int yy, int bb) -> uint64_t {
    return yy < L ? (uint64_t)yy * kW + bb : (uint64_t)n + (uint64_t)(yy - L) * kW + bb;
  };
  const float mt = (float)(-d.t);
  const float* eta = eta32 + d.onsite_off / 2;
  const cf* gsrc = (dir == 0 ? gL : gR) + d.g_off;
  const cf* st = start + d.start_off + (uint64_t)(has ? y : 0) * kW * kW;
  float* wt = weights + d.wt_off;
  cf* ed = edge + d.edge_off + (uint64_t)(has ? y : 0) * 2 * kW * kW;   // [slot][a][b]
  const int ys[2] = {job.y0, job.y1};

  // write the staged weights of slice k of column slot c (all threads; coalesced rows)
  auto flush = [&](int c, int k) {
    for (int i = tid; i < kW * kW; i += kThreads) {
      const int bb = i / kW, a = i % kW;
      wt[row_of(ys[c], bb) * K + (uint64_t)k * kW + a] = wbuf[a * kWPitch + c * kW + bb];
    }
  };

  // ---- direction 0 emits every column's start slice
  if (dir == 0) {
    if (has) {
      for (int a = 0; a < kW; ++a) {
        const cf v = st[a * kW + b];
        wbuf[a * kWPitch + tid] = eta[m0 * kW + a] * (v.x * v.x + v.y * v.y);
        if (m0 == 0) ed[(0 * kW + a) * kW + b] = v;
        if (m0 == L - 1) ed[(1 * kW + a) * kW + b] = v;
      }
    }
    __syncthreads();
    for (int c = 0; c < 2; ++c)
      if (ys[c] >= 0) flush(c, m0_of(ys[c]));
    __syncthreads();
  }

  // ---- propagation over the union of the pair's slices
  const int m0a = m0_of(job.y0), m0b = job.y1 >= 0 ? m0_of(job.y1) : m0a;
  const int k_first = dir == 0 ? max(m0a, m0b) - 1 : min(m0a, m0b) + 1;
  const int k_end = dir == 0 ? -1 : L;
  const int kstep = dir == 0 ? -1 : 1;
  // instruction descriptor: D F32, A and B TF32, K-major both, N = 128, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((128u >> 3) << 17) |
                         ((128u >> 4) << 24);
  const uint64_t dbh = smem_desc(smem_u32(bh), kLBO, kSBO);
  const uint64_t dbl = smem_desc(smem_u32(bl), kLBO, kSBO);
  uint32_t phase = 0, gphase = 0;
  bool timeout = false, g_pending = false;
  // one thread stages g_k: 64 row copies of 512 bytes into the padded rows
  auto issue_g = [&](int k) {
    if (tid == 0) {
      mbar_expect_tx(mbar_g, kW * kW * (uint32_t)sizeof(cf));
      const cf* g = gsrc + (uint64_t)k * kW * kW;
      for (int a = 0; a < kW; ++a)
        bulk_g2s(stage + (size_t)a * kStagePitch, g + (size_t)a * kW, kW * sizeof(cf), mbar_g);
    }
    g_pending = true;
  };
  if (k_first != k_end) issue_g(k_first);
  for (int k = k_first; k != k_end; k += kstep) {
    const bool active = has && (dir == 0 ? k < m0 : k > m0);
    const bool joining = has && (dir == 0 ? k == m0 - 1 : k == m0 + 1);
    if (joining) {
      // A = the split start block column b
      for (int half = 0; half < 2; ++half) {
        uint32_t rh[32], rl[32], ih[32], il[32];
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const cf v = st[(half * 32 + i) * kW + b];
          rh[i] = to_tf32(v.x);
          rl[i] = __float_as_uint(v.x - __uint_as_float(rh[i]));
          ih[i] = to_tf32(v.y);
          il[i] = __float_as_uint(v.y - __uint_as_float(ih[i]));
        }
        tmem_st32(tlane + kColAh + half * 32, rh);
        tmem_st32(tlane + kColAl + half * 32, rl);
        tmem_st32(tlane + kColAh + 64 + half * 32, ih);
        tmem_st32(tlane + kColAl + 64 + half * 32, il);
      }
    }
    bool got = false;
    for (uint32_t it = 0; it < kWaitLimit && !got; ++it) got = mbar_try_wait(mbar_g, gphase);
    gphase ^= 1u;
    g_pending = !got;
    if (__syncthreads_or(!got)) {
      timeout = true;
      break;
    }
    build_b(stage, mt, bh, bl, tid);
    tmem_st_wait();
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    // the stage is free: fetch the next step's block while this step computes
    if (k + kstep != k_end) issue_g(k + kstep);
    if (tid == 0) {
      uint32_t acc = 0;
      for (int pass = 0; pass < 3; ++pass) {
        const uint32_t acol = pass == 0 ? kColAl : kColAh;
        const uint64_t bd = pass == 1 ? dbl : dbh;
        for (int s = 0; s < 16; ++s) {
          mma_tf32_ts(tbase + kColD, tbase + acol + (uint32_t)s * 8u,
                      bd + (uint64_t)((s * 2 * kLBO) >> 4), idesc, acc);
          acc = 1;
        }
      }
      mma_commit(mbar);
    }
    bool done = false;
    for (uint32_t it = 0; it < kWaitLimit && !done; ++it) done = mbar_try_wait(mbar, phase);
    phase ^= 1u;
    if (__syncthreads_or(!done)) {
      timeout = true;
      break;
    }
    tc_fence_after();
    if (active) {
      const bool more = k + kstep != k_end;
      const int slot = (dir == 0 && k == 0) ? 0 : ((dir == 1 && k == L - 1) ? 1 : -1);
      const float* ek = eta + k * kW;
      for (int ch = 0; ch < 4; ++ch) {
        uint32_t v[32];
        tmem_ld32(tlane + kColD + ch * 32, v);
        tmem_ld_wait();
        const int a0 = (ch & 1) * 32;
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          const float x = __uint_as_float(v[i]);
          float* wp = wbuf + (a0 + i) * kWPitch + tid;
          if (ch < 2) *wp = x * x;
          else *wp = ek[a0 + i] * (*wp + x * x);
          if (slot >= 0) {
            float* e = reinterpret_cast<float*>(ed + ((uint64_t)slot * kW + a0 + i) * kW + b);
            e[ch < 2 ? 0 : 1] = x;
          }
        }
        if (more) {
          uint32_t h[32], l[32];
#pragma unroll
          for (int i = 0; i < 32; ++i) {
            const float x = __uint_as_float(v[i]);
            h[i] = to_tf32(x);
            l[i] = __float_as_uint(x - __uint_as_float(h[i]));
          }
          tmem_st32(tlane + kColAh + ch * 32, h);
          tmem_st32(tlane + kColAl + ch * 32, l);
        }
      }
    }
    __syncthreads();
    for (int c = 0; c < 2; ++c) {
      if (ys[c] < 0) continue;
      const int mc = m0_of(ys[c]);
      if (dir == 0 ? k < mc : k > mc) flush(c, k);
    }
  }
  if (timeout && tid == 0) atomicOr(err, ERR_TIMEOUT);
  if (g_pending) {
    // a staged copy may still be in flight after a timeout: wait for it (bounded)
    bool got = false;
    for (uint32_t it = 0; it < kWaitLimit && !got; ++it) got = mbar_try_wait(mbar_g, gphase);
  }
  tmem_st_wait();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, kTmemCols);
}

// Lead weights of the level-1 rows of fused tasks: row b of block column y gets, in slot s
// (0: lead L, 1: lead R), sum_nu Gamma_nu |(Phi^T X)_{nu b}|^2 = <psi_b|Gamma|psi_b> from the
// edge block X of that column (slice 0 or slice L - 1).  One warp per (task, column, slot).
constexpr size_t kLeadSmem = sizeof(cf) * kW * kW + sizeof(float) * kW * kW + sizeof(float) * kW;

__global__ void __launch_bounds__(32) lead_weights_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs,
    const float* __restrict__ phi32, const double* __restrict__ gam,
    const cf* __restrict__ edge, float* __restrict__ weights) {
  extern __shared__ __align__(16) unsigned char lsm[];
  cf* s_x = reinterpret_cast<cf*>(lsm);                          // [a][b]
  float* s_phi = reinterpret_cast<float*>(s_x + kW * kW);        // [a][nu]
  float* s_gam = s_phi + kW * kW;
  const int lane = threadIdx.x;
  const uint32_t job = blockIdx.x;
  if (job >= n_jobs) return;
  int lo = 0, hi = n_tasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (2 * tasks[mid].col_base <= job) lo = mid; else hi = mid - 1;
  }
  const TaskDesc& d = tasks[lo];
  if (!d.fused) return;
  const uint32_t local = job - 2 * d.col_base;
  const int y = (int)(local >> 1), slot = (int)(local & 1);
  const int L = d.L, n = d.n, K = d.K;
  const cf* X = edge + d.edge_off + ((uint64_t)y * 2 + slot) * kW * kW;
  for (int i = lane; i < kW * kW; i += 32) {
    s_x[i] = X[i];
    s_phi[i] = phi32[d.phi_off + i];
  }
  for (int i = lane; i < kW; i += 32) s_gam[i] = (float)gam[d.lead_off + i];
  __syncwarp();
  for (int bb = lane; bb < kW; bb += 32) {
    float sum = 0.f;
    for (int nu = 0; nu < kW; ++nu) {
      float zr = 0.f, zi = 0.f;
      for (int a = 0; a < kW; ++a) {
        const float p = s_phi[a * kW + nu];
        const cf x = s_x[a * kW + bb];
        zr += p * x.x;
        zi += p * x.y;
      }
      sum += s_gam[nu] * (zr * zr + zi * zi);
    }
    const uint64_t row = y < L ? (uint64_t)y * kW + bb : (uint64_t)n + (uint64_t)(y - L) * kW + bb;
    weights[d.wt_off + row * K + n + slot] = sum;
  }
}

}  // namespace

cudaError_t launch_chain_tc(const TaskDesc* d_tasks, int n_tasks, uint32_t n_cols,
                            const TcJob* d_jobs, uint32_t n_jobs, const float* d_eta32,
                            const float* d_phi32, const double* d_gam, const void* d_gL,
                            const void* d_gR, const void* d_start, void* d_weights,
                            uint64_t* d_tab, void* d_edge, int32_t* d_err, cudaStream_t s) {
  if (n_jobs == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(chain_tc_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem);
  if (e != cudaSuccess) return e;
  chain_tc_kernel<<<n_jobs, kThreads, kSmem, s>>>(
      d_tasks, d_jobs, d_eta32, static_cast<const cf*>(d_gL), static_cast<const cf*>(d_gR),
      static_cast<const cf*>(d_start), static_cast<float*>(d_weights),
      static_cast<cf*>(d_edge), d_err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const uint32_t lead_jobs = 2 * n_cols;
  e = cudaFuncSetAttribute(lead_weights_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kLeadSmem);
  if (e != cudaSuccess) return e;
  lead_weights_kernel<<<lead_jobs, 32, kLeadSmem, s>>>(
      d_tasks, n_tasks, lead_jobs, d_phi32, d_gam, static_cast<const cf*>(d_edge),
      static_cast<float*>(d_weights));
  return cudaGetLastError();
}

}  // namespace negf
