// Block-column adjoint of the transmission's gradient: no n x n array anywhere.
//
// The derivative target and the seeds are those of k_backward.cu (score-function seeds wbar of
// every Step 6' weight, ubar of every injection-mode weight): with Gbar the Wirtinger seed of
// every element of G = (E - H - Sigma)^{-1},
//   dT/dV_k = 2 Re (G Gbar G)_kk,   dT/deta_k = Im (G Gbar G)_kk + the explicit gamma_k terms.
// Here (G Gbar G)_kk is accumulated one block column m (the W sites of slice m) at a time:
//   X = G[:, m]     G_mm by one inversion, then the RGF relations of Sec. III.B:
//                   G_{k,m} = -t g^L_k G_{k+1,m} (k < m),  G_{k,m} = -t g^R_k G_{k-1,m} (k > m);
//   U = Gbar[:, m]  each column of Gbar needs only the same column of G (site seeds, the lead
//                   columns of the site rows), and, in the start lead's boundary slice s_p, the
//                   injection rows' psi = G Phi_p = X Phi (column m = s_p alone);
//   Z = G U         by block-tridiagonal elimination with the left-connected blocks
//                   (g^L_{L-1} taken as G_{L-1,L-1}):
//                     y_0 = g^L_0 U_0,  y_k = g^L_k (U_k - t y_{k-1}),
//                     z_{L-1} = y_{L-1},  z_k = y_k - t g^L_k z_{k+1};
//   (G Gbar G)_kk += sum_{j in slice m} Z[k, j] G[j, k] = sum_j Z[k, j] X[k, j]   (G = G^T).
// A column costs about 3 L block products (W x W x W), a task 3 L^2 W^3 complex multiply-adds
// (5 L for the column s_p), against the n^3 of the dense adjoint product; its memory is two
// block columns per CTA in flight.
//
// Checkpoints (ckpt_stride s): adj_sweep_kernel runs both RGF sweeps of every task once and keeps
// only every s-th block (left: g^L_k at k = 0, s, 2s, ...; right: g^R_k at k = L-1, L-1-s, ...).
// Before a group of tasks runs its columns, adj_expand_kernel recomputes the blocks between
// checkpoints, one CTA per segment of s slices (s serial inversions each, the segments in
// parallel), into buffers that live only while that group's columns run.  The kept blocks take
// 1/s of the memory of all tasks' sweeps; the recompute is one more inversion per block.
//
// Thread layout of the block products: 256 threads as 16 x 16; thread (ty, tx) owns rows
// ty + 16 a and columns tx + 16 b (a, b < RT = ceil(W / 16)) of the W x W result, blocks row-major
// with stride W in shared memory.  Every W x W block, the seeds and the per-step arithmetic are
// in the precision of the tables (complex64 or complex128; the FP64 pipe of this GPU is 1/64 of
// the FP32 rate, so an FP32 build keeps FP64 out of the per-step work: the modes, broadenings
// and dephasing rates are staged as FP32 in shared memory); the gradient is accumulated in FP64.
#include <cuda_runtime.h>
#include <math.h>

#include "gj.cuh"
#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr int kAdjThreads = 256;

__device__ __forceinline__ cd conj_(cd a) { return cd{a.x, -a.y}; }
__device__ __forceinline__ cf conj_(cf a) { return cf{a.x, -a.y}; }

// Lead self-energy Sigma_r = Phi diag(sigma) Phi^T, entry (a, b) (FP64; both leads alike)
__device__ __forceinline__ cd lead_sigma(int a, int b, int W, const double* phi, const cd* sg) {
  cd acc = mk(0.0, 0.0);
  for (int m = 0; m < W; ++m) acc = acc + (phi[a * W + m] * phi[b * W + m]) * sg[m];
  return acc;
}

// A <- E - H_kk - Sigma_s(k) - [lead terms] - t^2 P (P = the block in A, in place; P absent when
// !with_prev): the slice matrix of the left (right) sweep at slice k.
template <typename C>
__device__ void form_slice(C* A, int k, int W, const TaskDesc& d, const double* onsite,
                           const double* eta, const double* phi, const cd* sg, bool lead_l,
                           bool lead_r, bool with_prev) {
  using R = typename Real<C>::T;
  const R tt = (R)(d.t * d.t);
  for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
    const int a = idx / W, b = idx - a * W;
    C v = slice_entry<C>(a, b, k, W, d.E, d.t, onsite, eta, slice_block(d, onsite));
    if (lead_l || lead_r) {
      const cd s = lead_sigma(a, b, W, phi, sg);
      const int nl = (lead_l ? 1 : 0) + (lead_r ? 1 : 0);
      v = v - to_c(mk((double)nl * s.x, (double)nl * s.y), C{});
    }
    if (with_prev) v = v - tt * A[idx];
    A[idx] = v;
  }
}

// every site of slice k dephases: inversion without a pivot search (see gj_rows)
__device__ __forceinline__ bool slice_dephased(const double* eta, int k, int W) {
  return __syncthreads_and(threadIdx.x >= W || eta[k * W + threadIdx.x] > 0.0);
}

// ---- checkpointed sweeps: one CTA per (task, direction) --------------------------------------
// Left (dir 0): k = 0 .. L-1, the last block the full G_{L-1,L-1} (right lead included).
// Right (dir 1): k = L-1 .. 1.  Kept: every s-th block of each direction, at ck + task's
// offset + (index along the sweep / s) W^2.
template <typename C>
__global__ void __launch_bounds__(kAdjThreads) adj_sweep_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, const double* __restrict__ wire,
    const double* __restrict__ phig, const cd* __restrict__ sig,
    const uint64_t* __restrict__ ck_off, int s, C* __restrict__ ck, int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int job = blockIdx.x;
  if (job >= 2 * n_tasks) return;
  const int task = job >> 1, dir = job & 1;
  const TaskDesc d = tasks[task];
  const int W = d.W, L = d.L, WW = W * W;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* rowk = A + WW;
  C* fcol = rowk + W;
  int* perm = reinterpret_cast<int*>(fcol + W);
  int* flag = perm + W;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  const double* phi = phig + d.phi_off;
  const cd* sg = sig + d.lead_off;
  const int nck = (L + s - 1) / s;
  C* out = ck + ck_off[task] + (uint64_t)dir * nck * WW;
  const int steps = dir == 0 ? L : L - 1;
  for (int i = 0; i < steps; ++i) {
    const int k = dir == 0 ? i : L - 1 - i;
    form_slice(A, k, W, d, onsite, eta, phi, sg, dir == 0 && k == 0, k == L - 1, i > 0);
    __syncthreads();
    const bool deph = slice_dephased(eta, k, W);
    if (!cta_gj(A, rowk, fcol, perm, flag, W, !deph)) {
      if (threadIdx.x == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
    if (i % s == 0) {
      C* dst = out + (uint64_t)(i / s) * WW;
      for (int idx = threadIdx.x; idx < WW; idx += blockDim.x) dst[idx] = A[idx];
    }
    __syncthreads();
  }
}

// ---- recompute between checkpoints: one CTA per (task of the group, direction, segment) -----
// gl[k] (k = 0 .. L-1) and gr[k] (k = 1 .. L-1) of each task of the group, W^2 each.
template <typename C>
__global__ void __launch_bounds__(kAdjThreads) adj_expand_kernel(
    const TaskDesc* __restrict__ tasks, int task0, int n_group, const double* __restrict__ wire,
    const double* __restrict__ phig, const cd* __restrict__ sig,
    const uint64_t* __restrict__ ck_off, int s, const C* __restrict__ ck, C* __restrict__ gl,
    C* __restrict__ gr, int32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TaskDesc d0 = tasks[task0];
  const int L = d0.L, W = d0.W, WW = W * W;
  const int nck = (L + s - 1) / s;
  const int job = blockIdx.x;
  if (job >= n_group * 2 * nck) return;
  const int tl = job / (2 * nck), rem = job - tl * 2 * nck, dir = rem / nck, c = rem - dir * nck;
  const int task = task0 + tl;
  const TaskDesc d = tasks[task];
  const int steps = dir == 0 ? L : L - 1;
  const int i0 = c * s;
  if (i0 >= steps) return;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* rowk = A + WW;
  C* fcol = rowk + W;
  int* perm = reinterpret_cast<int*>(fcol + W);
  int* flag = perm + W;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  const double* phi = phig + d.phi_off;
  const cd* sg = sig + d.lead_off;
  const C* src = ck + ck_off[task] + ((uint64_t)dir * nck + c) * WW;
  C* out = (dir == 0 ? gl : gr) + (uint64_t)tl * L * WW;
  for (int idx = threadIdx.x; idx < WW; idx += blockDim.x) A[idx] = src[idx];
  const int i_end = min(i0 + s, steps);
  for (int i = i0;; ++i) {
    const int k = dir == 0 ? i : L - 1 - i;
    __syncthreads();
    C* dst = out + (uint64_t)k * WW;
    for (int idx = threadIdx.x; idx < WW; idx += blockDim.x) dst[idx] = A[idx];
    if (i + 1 >= i_end) break;
    const int kn = dir == 0 ? k + 1 : k - 1;
    __syncthreads();
    form_slice(A, kn, W, d, onsite, eta, phi, sg, false, kn == L - 1 && dir == 0, true);
    __syncthreads();
    const bool deph = slice_dephased(eta, kn, W);
    if (!cta_gj(A, rowk, fcol, perm, flag, W, !deph)) {
      if (threadIdx.x == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
  }
}

// ---- block products ------------------------------------------------------------------------
// out = A B with A a W x W block (stride W) and B a W x N panel (stride N, N <= 64): thread
// (ty, tx) owns rows ty + 16 a (a < RT) and columns tx + 16 b (b < RTN).
template <typename C, int RT, int RTN>
__device__ __forceinline__ void cta_prod(const C* __restrict__ A, const C* __restrict__ B, int W,
                                         int N, C (&acc)[RT][RTN]) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < RTN; ++b) acc[a][b] = mkc(0.0, 0.0, C{});
  int ra[RT], cb[RTN];
#pragma unroll
  for (int a = 0; a < RT; ++a) {
    const int r = ty + 16 * a;
    ra[a] = (r < W ? r : W - 1) * W;                // clamped: rows/columns beyond are discarded
  }
#pragma unroll
  for (int b = 0; b < RTN; ++b) {
    const int c = tx + 16 * b;
    cb[b] = c < N ? c : N - 1;
  }
  for (int l = 0; l < W; ++l) {
    C av[RT], bv[RTN];
#pragma unroll
    for (int a = 0; a < RT; ++a) av[a] = A[ra[a] + l];
#pragma unroll
    for (int b = 0; b < RTN; ++b) bv[b] = B[l * N + cb[b]];
#pragma unroll
    for (int a = 0; a < RT; ++a)
#pragma unroll
      for (int b = 0; b < RTN; ++b) {
        acc[a][b].x += av[a].x * bv[b].x - av[a].y * bv[b].y;
        acc[a][b].y += av[a].x * bv[b].y + av[a].y * bv[b].x;
      }
  }
}

// visit this thread's valid entries (i, j) of a W x N product tile
template <int RT, int RTN, typename F>
__device__ __forceinline__ void for_tile(int W, int N, F f) {
  const int ty = threadIdx.x >> 4, tx = threadIdx.x & 15;
#pragma unroll
  for (int a = 0; a < RT; ++a)
#pragma unroll
    for (int b = 0; b < RTN; ++b) {
      const int i = ty + 16 * a, j = tx + 16 * b;
      if (i < W && j < N) f(a, b, i, j);
    }
}

template <typename C>
__device__ __forceinline__ void load_block(C* dst, const C* __restrict__ src, int count) {
  for (int idx = threadIdx.x; idx < count; idx += blockDim.x) dst[idx] = src[idx];
}

// A block of up to 256 RT^2 entries (a W x W block, W <= 16 RT) read into registers one step
// ahead: fetch() issues the loads before a product, put() stores them after it.
template <typename C, int RT>
struct BlockAhead {
  C v[RT * RT];
  __device__ __forceinline__ void fetch(const C* __restrict__ src, int count) {
#pragma unroll
    for (int q = 0; q < RT * RT; ++q) {
      const int idx = threadIdx.x + q * kAdjThreads;
      if (idx < count) v[q] = src[idx];
    }
  }
  __device__ __forceinline__ void put(C* dst, int count) const {
#pragma unroll
    for (int q = 0; q < RT * RT; ++q) {
      const int idx = threadIdx.x + q * kAdjThreads;
      if (idx < count) dst[idx] = v[q];
    }
  }
};

struct AdjArgs {
  const TaskDesc* tasks;
  int task0, n_group, p;
  const double* wire;
  const double* phi;
  const cd* sig;
  const double* gam;
  const void* wbar;          // [rows x K] per task at wt_off, in the precision of the tables
  const double* ubar;        // per task at mode_off
  uint64_t site_off0;        // dT of the group's first task (sites of earlier tasks before it)
  double* dV;
  double* dE;
  int32_t* err;
};

// Block columns per job: NC = 64 / W of them side by side (at most 8), so that each step's
// product is a W x (NC W) panel; the start lead's boundary column, which carries the injection
// work, is a job of its own.
__host__ __device__ inline int adj_ncols(int W) {
  const int nc = 64 / W;
  return nc < 1 ? 1 : (nc > 8 ? 8 : nc);
}

// One job per (task of the group, column set): the boundary column s_p of every task first,
// then the other columns NC at a time in increasing order.  Scratch per CTA: X and Y
// [L][W][NC W]; per task of the group: gl, gr, Psi [L][W][W], Tl [2][W][W].
template <typename C, int RT, int RTN>
__global__ void __launch_bounds__(kAdjThreads, RT >= 2 ? 1 : (sizeof(C) == 8 ? 3 : 2)) adj_column_kernel(AdjArgs g, const C* __restrict__ gl_all,
                                                                 const C* __restrict__ gr_all,
                                                                 C* __restrict__ psi_all,
                                                                 C* __restrict__ tl_all,
                                                                 C* __restrict__ xs_all,
                                                                 C* __restrict__ ys_all) {
  using R = typename Real<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const TaskDesc d0 = g.tasks[g.task0];
  const int W = d0.W, L = d0.L, WW = W * W, n = d0.n, K = d0.K;
  const int NC = adj_ncols(W), NP = NC * W;            // panel width
  const int PA = WW > W * NP ? WW : W * NP;
  C* sA = reinterpret_cast<C*>(smem_raw);              // g block / X_k panel / seeds
  C* sB = sA + PA;                                     // the running panel
  C* sT = sB + W * NP;                                 // Gamma_lead, Phi
  C* rowk = sT + WW;
  C* fcol = rowk + W;
  int* perm = reinterpret_cast<int*>(fcol + W);
  int* flag = perm + W;
  // FP32 builds: Phi, Gamma (per mode) and one slice's eta as R, after the integer words
  R* aux = reinterpret_cast<R*>(
      smem_raw + ((reinterpret_cast<unsigned char*>(flag + 2) - smem_raw + 15) & ~(size_t)15));
  const int p = g.p;
  const int sp = p == 0 ? 0 : L - 1;
  const R t = (R)d0.t;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int other = L - 1;                             // columns besides s_p
  const int per_task = 1 + (other + NC - 1) / NC;
  C* X = xs_all + (uint64_t)blockIdx.x * L * W * NP;
  C* Y = ys_all + (uint64_t)blockIdx.x * L * W * NP;
  const int n_jobs = g.n_group * per_task;
  for (int job = blockIdx.x; job < n_jobs; job += gridDim.x) {
    const int tl = job % g.n_group, jj = job / g.n_group;
    const bool inj = jj == 0;                          // the start lead's boundary column
    const int ncols = inj ? 1 : min(NC, other - (jj - 1) * NC);
    const int first = inj ? sp : (jj - 1) * NC + (p == 0 ? 1 : 0);   // columns first .. + ncols
    const int N = inj ? W : NP;                        // this job's panel stride
    auto col_m = [&](int c) { return first + c; };
    const TaskDesc d = g.tasks[g.task0 + tl];
    const double* onsite = g.wire + d.onsite_off;
    const double* eta = onsite + n;
    const double* phi = g.phi + d.phi_off;
    const cd* sg = g.sig + d.lead_off;
    const double* gam = g.gam + d.lead_off;
    const R* wb = static_cast<const R*>(g.wbar) + d.wt_off;
    const double* ub = g.ubar + d.mode_off + p * W;
    const R* phiR;                                     // Phi [x][m'], Gamma_m', ubar_m' as R
    const R* gamR;
    const R* ubR;
    R* etaS = nullptr;                                 // FP32: eta of the current slice
    if constexpr (sizeof(R) == 4) {
      __syncthreads();
      for (int idx = tid; idx < WW; idx += blockDim.x) aux[idx] = (R)phi[idx];
      for (int m = tid; m < W; m += blockDim.x) {
        aux[WW + m] = (R)gam[m];
        aux[WW + W + m] = (R)ub[m];
      }
      phiR = aux;
      gamR = aux + WW;
      ubR = aux + WW + W;
      etaS = aux + WW + 2 * W;
    } else {
      phiR = phi;
      gamR = gam;
      ubR = ub;
    }
    const C* gl = gl_all + (uint64_t)tl * L * WW;
    const C* gr = gr_all + (uint64_t)tl * L * WW;
    C* Psi = psi_all + (uint64_t)tl * L * WW;
    C* Tl = tl_all + (uint64_t)tl * 2 * WW;
    const uint64_t so = g.site_off0 + (uint64_t)tl * n;
    const uint64_t XS = (uint64_t)W * N;               // one slice of a panel
    C acc[RT][RTN];

    // ---- G_mm of every column: (E - H_mm - Sigma_s - [leads] - t^2 g^L_{m-1} - t^2 g^R_{m+1})^-1
    for (int c = 0; c < ncols; ++c) {
      const int m = col_m(c);
      __syncthreads();
      const R tt = t * t;
      for (int idx = tid; idx < WW; idx += blockDim.x) {
        const int a = idx / W, b = idx - a * W;
        C v = slice_entry<C>(a, b, m, W, d.E, d.t, onsite, eta, slice_block(d, onsite));
        const int nl = (m == 0 ? 1 : 0) + (m == L - 1 ? 1 : 0);
        if (nl) {
          const cd s = lead_sigma(a, b, W, phi, sg);
          v = v - to_c(mk(nl * s.x, nl * s.y), C{});
        }
        if (m > 0) v = v - tt * gl[(uint64_t)(m - 1) * WW + idx];
        if (m < L - 1) v = v - tt * gr[(uint64_t)(m + 1) * WW + idx];
        sA[idx] = v;
      }
      __syncthreads();
      const bool deph = slice_dephased(eta, m, W);
      if (!cta_gj(sA, rowk, fcol, perm, flag, W, !deph)) {
        if (tid == 0) atomicOr(g.err, ERR_SINGULAR);
        return;
      }
      for (int idx = tid; idx < WW; idx += blockDim.x) {
        const int a = idx / W, b = idx - a * W;
        X[(uint64_t)m * XS + a * N + c * W + b] = sA[idx];
      }
    }
    // ---- the block columns X_k = G_{k,m}: towards slice 0 (columns with m > k, each joining
    // at k = m - 1 with G_mm), then towards slice L - 1 (columns with m < k)
    const int m_lo = col_m(0), m_hi = col_m(ncols - 1);
    auto inject = [&](int c, int m) {                  // panel block c <- G_mm
      for (int idx = tid; idx < WW; idx += blockDim.x) {
        const int a = idx / W, b = idx - a * W;
        sB[a * N + c * W + b] = X[(uint64_t)m * XS + a * N + c * W + b];
      }
    };
    // narrow panels (RT = 1): each step's g block, panel entries and seeds are read one step
    // ahead, while the previous product runs
    constexpr bool kAhead = RT == 1;
    BlockAhead<C, RT> ga;
    if (kAhead && m_hi - 1 >= 0) ga.fetch(gl + (uint64_t)(m_hi - 1) * WW, WW);
    for (int k = m_hi - 1; k >= 0; --k) {
      __syncthreads();
      for (int c = 0; c < ncols; ++c)
        if (col_m(c) == k + 1) inject(c, col_m(c));
      if (kAhead) ga.put(sA, WW);
      else load_block(sA, gl + (uint64_t)k * WW, WW);
      __syncthreads();
      if (kAhead && k > 0) ga.fetch(gl + (uint64_t)(k - 1) * WW, WW);
      cta_prod<C, RT, RTN>(sA, sB, W, N, acc);
      __syncthreads();
      for_tile<RT, RTN>(W, N, [&](int a, int b, int i, int j) {
        const C v = (R)(-1) * t * acc[a][b];
        sB[i * N + j] = v;
        if (col_m(j / W) > k) X[(uint64_t)k * XS + i * N + j] = v;
      });
    }
    if (kAhead && m_lo + 1 < L) ga.fetch(gr + (uint64_t)(m_lo + 1) * WW, WW);
    for (int k = m_lo + 1; k < L; ++k) {
      __syncthreads();
      for (int c = 0; c < ncols; ++c)
        if (col_m(c) == k - 1) inject(c, col_m(c));
      if (kAhead) ga.put(sA, WW);
      else load_block(sA, gr + (uint64_t)k * WW, WW);
      __syncthreads();
      if (kAhead && k + 1 < L) ga.fetch(gr + (uint64_t)(k + 1) * WW, WW);
      cta_prod<C, RT, RTN>(sA, sB, W, N, acc);
      __syncthreads();
      for_tile<RT, RTN>(W, N, [&](int a, int b, int i, int j) {
        const C v = (R)(-1) * t * acc[a][b];
        sB[i * N + j] = v;
        if (col_m(j / W) < k) X[(uint64_t)k * XS + i * N + j] = v;
      });
    }
    // ---- column s_p: psi = X Phi (the injection rows' G Phi_p), the lead-column terms Tl_r of
    // the injection rows, and their contribution Cc_k = psibar_k Phi^T to U (kept in Y)
    if (inj) {
      __syncthreads();
      for (int idx = tid; idx < WW; idx += blockDim.x) {
        const int a = idx / W, b = idx - a * W;
        sT[idx] = C{phiR[idx], R(0)};                              // Phi [x][m']
        sB[idx] = C{phiR[b * W + a], R(0)};                        // Phi^T [m'][y]
      }
      for (int k = 0; k < L; ++k) {
        __syncthreads();
        load_block(sA, X + (uint64_t)k * WW, WW);
        __syncthreads();
        cta_prod<C, RT, RTN>(sA, sT, W, W, acc);
        for_tile<RT, RTN>(W, W, [&](int a, int b, int i, int j) { Psi[(uint64_t)k * WW + i * W + j] = acc[a][b]; });
      }
      // Tl_r[x][m'] = sum_nu Gamma_nu phi_nu(x) conj(z_nu^(m')), z = Phi^T psi_{s_r}
      for (int r = 0; r < 2; ++r) {
        const int sr = r == 0 ? 0 : L - 1;
        __syncthreads();
        for (int idx = tid; idx < WW; idx += blockDim.x) {
          const int nu = idx / W, mp = idx - nu * W;
          R zx = 0, zy = 0;
          for (int x = 0; x < W; ++x) {
            const R f = phiR[x * W + nu];
            const C ps = Psi[(uint64_t)sr * WW + x * W + mp];
            zx += f * ps.x;
            zy += f * ps.y;
          }
          sA[idx] = C{zx, zy};
        }
        __syncthreads();
        for (int idx = tid; idx < WW; idx += blockDim.x) {
          const int x = idx / W, mp = idx - x * W;
          R tx = 0, ty = 0;
          for (int nu = 0; nu < W; ++nu) {
            const R f = gamR[nu] * phiR[x * W + nu];
            const C z = sA[nu * W + mp];
            tx += f * z.x;
            ty -= f * z.y;
          }
          Tl[(uint64_t)r * WW + idx] = C{tx, ty};
        }
      }
      __syncthreads();
      for (int k = 0; k < L; ++k) {
        if constexpr (sizeof(R) == 4) {
          if (tid < W) etaS[tid] = (R)eta[k * W + tid];       // readers of the last slice passed a barrier
        }
        __syncthreads();
        for (int idx = tid; idx < WW; idx += blockDim.x) {
          const int mp = idx / W, i = idx - mp * W;              // psibar_k [i][m']
          const R* wrow = wb + (uint64_t)(n + p * W + mp) * K;
          const int b = k * W + i;
          const C ps = Psi[(uint64_t)k * WW + i * W + mp];
          R eb;
          if constexpr (sizeof(R) == 4) eb = etaS[i]; else eb = eta[b];
          const R f = wrow[b] * eb;
          R vx = f * ps.x, vy = -f * ps.y;
          for (int r = 0; r < 2; ++r) {
            const int sr = r == 0 ? 0 : L - 1;
            if (k != sr) continue;
            const R wl = wrow[n + r];
            if (wl == R(0)) continue;
            const C tv = Tl[(uint64_t)r * WW + i * W + mp];
            vx += wl * tv.x;
            vy += wl * tv.y;
          }
          sA[i * W + mp] = C{vx, vy};
        }
        __syncthreads();
        cta_prod<C, RT, RTN>(sA, sB, W, W, acc);
        for_tile<RT, RTN>(W, W, [&](int a, int b, int i, int j) { Y[(uint64_t)k * WW + i * W + j] = acc[a][b]; });
      }
    }
    // the lead broadening of the boundary slices, Gamma_lead = Phi diag(Gamma) Phi^T (real)
    __syncthreads();
    for (int idx = tid; idx < WW; idx += blockDim.x) {
      const int a = idx / W, b = idx - a * W;
      R v = 0;
      for (int nu = 0; nu < W; ++nu) v += gamR[nu] * phiR[a * W + nu] * phiR[b * W + nu];
      sT[idx] = C{v, R(0)};
    }
    // ---- forward elimination: y_k = g^L_k (U_k - t y_{k-1}), U_k = Gbar[k-block, columns]
    // kAhead: this thread's panel entries X[k][i][jj2], seeds wbar_{(m,j),(k,i)} and eta of
    // slice k, read one step ahead
    C xa[RT][RTN];
    R wa[RT][RTN], ea[RT];
    auto fetch_eta = [&](int k) {
#pragma unroll
      for (int a = 0; a < RT; ++a) {
        const int i = (tid >> 4) + 16 * a;
        ea[a] = i < W ? (R)eta[k * W + i] : R(0);
      }
    };
    auto fetch_seeds = [&](int k) {
      fetch_eta(k);
      for_tile<RT, RTN>(W, N, [&](int a, int bb, int i, int jj2) {
        const int c = jj2 / W, j = jj2 - c * W;
        if (c < ncols) {
          xa[a][bb] = X[(uint64_t)k * XS + i * N + jj2];
          wa[a][bb] = wb[(uint64_t)(col_m(c) * W + j) * K + k * W + i];
        }
      });
    };
    if (kAhead) {
      ga.fetch(gl, WW);
      fetch_seeds(0);
    }
    for (int k = 0; k < L; ++k) {
      const bool edge = k == 0 || k == L - 1;
      __syncthreads();
      if (edge) {
        // lead columns of the site rows: U[x][j] += (sum_r wbar_{(m,j), n+r}) conj(Gamma_lead X_k)[x][j]
        load_block(sA, X + (uint64_t)k * XS, W * N);
        __syncthreads();
        cta_prod<C, RT, RTN>(sT, sA, W, N, acc);
        __syncthreads();
        for_tile<RT, RTN>(W, N, [&](int a, int b, int i, int j) { sA[i * N + j] = conj_(acc[a][b]); });
        __syncthreads();
      }
      // in the products' thread layout (row i, panel column jj2 = c W + j): the panel's shared
      // and global accesses stay conflict-free and coalesced; the seeds wbar_{(m,j),(k,i)} are
      // read two rows of 16 per warp
      if (!kAhead) fetch_eta(k);
      for_tile<RT, RTN>(W, N, [&](int a, int bb, int i, int jj2) {
        const int c = jj2 / W, j = jj2 - c * W;
        C u = C{R(0), R(0)};
        if (c < ncols) {
          const int m = col_m(c);
          const R* wrow = wb + (uint64_t)(m * W + j) * K;
          C xv;
          R f;
          if constexpr (RT == 1) {                     // read one step ahead
            xv = xa[a][bb];
            f = wa[a][bb] * ea[a];
          } else {
            xv = X[(uint64_t)k * XS + i * N + jj2];
            f = wrow[k * W + i] * ea[a];
          }
          R ux = f * xv.x, uy = -f * xv.y;
          if (edge) {
            R wl = 0;
            if (k == 0) wl += wrow[n];
            if (k == L - 1) wl += wrow[n + 1];
            if (wl != R(0)) {
              const C tb = sA[i * N + jj2];
              ux += wl * tb.x;
              uy += wl * tb.y;
            }
          }
          if (inj) {
            const C cc = Y[(uint64_t)k * WW + i * W + j];
            ux += cc.x;
            uy += cc.y;
            if (k == sp) {
              // mode weights u_m' = lambda_m' <phi_m'|A|phi_m'>: i sum ubar Gamma phi phi
              R v = 0;
              for (int mp = 0; mp < W; ++mp) v += ubR[mp] * gamR[mp] * phiR[i * W + mp] * phiR[j * W + mp];
              uy += v;
            }
          }
          u = C{ux, uy};
        }
        if (k > 0) u = u - t * sB[i * N + jj2];
        sB[i * N + jj2] = u;
      });
      __syncthreads();
      if (kAhead) ga.put(sA, WW);
      else load_block(sA, gl + (uint64_t)k * WW, WW);
      __syncthreads();
      if (kAhead && k + 1 < L) {
        ga.fetch(gl + (uint64_t)(k + 1) * WW, WW);
        fetch_seeds(k + 1);
      }
      cta_prod<C, RT, RTN>(sA, sB, W, N, acc);
      __syncthreads();
      for_tile<RT, RTN>(W, N, [&](int a, int b, int i, int j) {
        sB[i * N + j] = acc[a][b];
        Y[(uint64_t)k * XS + i * N + j] = acc[a][b];
      });
    }
    // ---- back substitution z_k = y_k - t g^L_k z_{k+1}, and the diagonal of G Gbar G
    // kAhead: g^L_k, this thread's y_k entries (in xa) and its warp's diagonal inputs (rows
    // a = warp + 8 q, panel columns lane + 32 e: X[k] and the seeds) read one step ahead
    C xd[2][2];
    R wd[2][2];
    auto fetch_y = [&](int k) {
      for_tile<RT, RTN>(W, N, [&](int a, int bb, int i, int j) {
        xa[a][bb] = Y[(uint64_t)k * XS + i * N + j];
      });
    };
    auto fetch_diag = [&](int k) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int a = warp + 8 * q, jj2 = lane + 32 * e;
          if (a < W && jj2 < ncols * W) {
            const int c = jj2 / W, j = jj2 - c * W;
            xd[q][e] = X[(uint64_t)k * XS + a * N + jj2];
            wd[q][e] = wb[(uint64_t)(col_m(c) * W + j) * K + k * W + a];
          }
        }
    };
    // the diagonal of row a of slice k from z (sB) and X[k]: sum_j z[a][j] X[a][j] and the
    // explicit gamma terms, added to the gradient by lane 0
    auto diag_row = [&](int k, int a, R zx, R zy, R ex) {
      const int site = k * W + a;
      if (inj) {
        for (int j = lane; j < W; j += 32) {
          const C ps = Psi[(uint64_t)k * WW + a * W + j];
          ex += wb[(uint64_t)(n + p * W + j) * K + site] * (ps.x * ps.x + ps.y * ps.y);
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        zx += __shfl_down_sync(0xffffffffu, zx, o);
        zy += __shfl_down_sync(0xffffffffu, zy, o);
        ex += __shfl_down_sync(0xffffffffu, ex, o);
      }
      if (lane == 0) {
        atomicAdd(g.dV + so + site, 2.0 * (double)zx);
        atomicAdd(g.dE + so + site, (double)zy + (double)ex);
      }
    };
    if (kAhead) {
      if (L >= 2) {
        ga.fetch(gl + (uint64_t)(L - 2) * WW, WW);
        fetch_y(L - 2);
      }
      fetch_diag(L - 1);
    }
    for (int k = L - 1; k >= 0; --k) {
      if (k < L - 1) {
        __syncthreads();
        if (kAhead) ga.put(sA, WW);
        else load_block(sA, gl + (uint64_t)k * WW, WW);
        __syncthreads();
        if (kAhead && k > 0) ga.fetch(gl + (uint64_t)(k - 1) * WW, WW);
        cta_prod<C, RT, RTN>(sA, sB, W, N, acc);
        __syncthreads();
        for_tile<RT, RTN>(W, N, [&](int a, int b, int i, int j) {
          const C y = kAhead ? xa[a][b] : Y[(uint64_t)k * XS + i * N + j];
          sB[i * N + j] = y - t * acc[a][b];
        });
        if (kAhead && k > 0) fetch_y(k - 1);
      }
      __syncthreads();
      if constexpr (RT == 1) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int a = warp + 8 * q;
          if (a >= W) continue;                          // warp-uniform
          R zx = 0, zy = 0, ex = 0;
#pragma unroll
          for (int e = 0; e < 2; ++e) {
            const int jj2 = lane + 32 * e;
            if (jj2 < ncols * W) {
              const C z = sB[a * N + jj2];
              const C x = xd[q][e];
              zx += z.x * x.x - z.y * x.y;
              zy += z.x * x.y + z.y * x.x;
              ex += wd[q][e] * (x.x * x.x + x.y * x.y);
            }
          }
          diag_row(k, a, zx, zy, ex);
        }
        if (k > 0) fetch_diag(k - 1);
      } else {
        for (int a = warp; a < W; a += kAdjThreads / 32) {
          const int site = k * W + a;
          R zx = 0, zy = 0, ex = 0;
          for (int jj2 = lane; jj2 < ncols * W; jj2 += 32) {
            const int c = jj2 / W, j = jj2 - c * W;
            const C z = sB[a * N + jj2];
            const C x = X[(uint64_t)k * XS + a * N + jj2];
            zx += z.x * x.x - z.y * x.y;
            zy += z.x * x.y + z.y * x.x;
            ex += wb[(uint64_t)(col_m(c) * W + j) * K + site] * (x.x * x.x + x.y * x.y);
          }
          diag_row(k, a, zx, zy, ex);
        }
      }
    }
  }
}

template <typename C>
size_t gj_smem(int W) {
  return sizeof(C) * (size_t)(W * W + 2 * W) + sizeof(int) * (size_t)(W + 2);
}
template <typename C>
size_t column_smem(int W) {
  const size_t NP = (size_t)adj_ncols(W) * W;
  const size_t PA = (size_t)W * W > W * NP ? (size_t)W * W : W * NP;
  const size_t base =
      sizeof(C) * (PA + W * NP + (size_t)W * W + 2 * W) + sizeof(int) * (size_t)(W + 2);
  // FP32: Phi, Gamma, ubar and one slice's eta staged as FP32 behind the integer words
  const size_t aux = sizeof(C) == 8 ? sizeof(float) * ((size_t)W * W + 3 * W) : 0;
  return ((base + 15) & ~(size_t)15) + aux;
}

template <typename C, int RT, int RTN>
cudaError_t columns_rt(const AdjArgs& a, int W, const C* gl, const C* gr, C* psi, C* tl, C* xs,
                       C* ys, int slots, cudaStream_t s) {
  const size_t smem = column_smem<C>(W);
  cudaError_t e = cudaFuncSetAttribute(adj_column_kernel<C, RT, RTN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  adj_column_kernel<C, RT, RTN><<<slots, kAdjThreads, smem, s>>>(a, gl, gr, psi, tl, xs, ys);
  return cudaGetLastError();
}

// CTAs of the column kernel for width W that one SM holds (registers and shared memory)
template <typename C, int RT, int RTN>
int occupancy_rt(int W) {
  const size_t smem = column_smem<C>(W);
  if (cudaFuncSetAttribute(adj_column_kernel<C, RT, RTN>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 1;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, adj_column_kernel<C, RT, RTN>,
                                                    kAdjThreads, smem) != cudaSuccess)
    return 1;
  return per_sm < 1 ? 1 : per_sm;
}

template <typename C>
int occupancy_impl(int W) {
  const int rt = (W + 15) / 16, rtn = (adj_ncols(W) * W + 15) / 16;
  if (rt == 1 && rtn <= 1) return occupancy_rt<C, 1, 1>(W);
  if (rt == 1 && rtn <= 2) return occupancy_rt<C, 1, 2>(W);
  if (rt == 1 && rtn <= 3) return occupancy_rt<C, 1, 3>(W);
  if (rt == 1) return occupancy_rt<C, 1, 4>(W);
  if (rt == 2 && rtn <= 3) return occupancy_rt<C, 2, 3>(W);
  if (rt == 2) return occupancy_rt<C, 2, 4>(W);
  if (rt == 3) return occupancy_rt<C, 3, 3>(W);
  return occupancy_rt<C, 4, 4>(W);
}

template <typename C>
cudaError_t columns_impl(const AdjArgs& a, int W, const void* gl, const void* gr, void* psi,
                         void* tl, void* xs, void* ys, int slots, cudaStream_t s) {
  const C* cgl = static_cast<const C*>(gl);
  const C* cgr = static_cast<const C*>(gr);
  C* cpsi = static_cast<C*>(psi);
  C* ctl = static_cast<C*>(tl);
  C* cxs = static_cast<C*>(xs);
  C* cys = static_cast<C*>(ys);
  // RT = ceil(W / 16) row tiles; RTN = ceil(NC W / 16) column tiles of the panel (>= RT, so
  // that the injection column's W x W products fit too)
  const int rt = (W + 15) / 16, rtn = (adj_ncols(W) * W + 15) / 16;
  if (rt == 1 && rtn <= 1) return columns_rt<C, 1, 1>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  if (rt == 1 && rtn <= 2) return columns_rt<C, 1, 2>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  if (rt == 1 && rtn <= 3) return columns_rt<C, 1, 3>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  if (rt == 1) return columns_rt<C, 1, 4>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  if (rt == 2 && rtn <= 3) return columns_rt<C, 2, 3>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  if (rt == 2) return columns_rt<C, 2, 4>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  if (rt == 3) return columns_rt<C, 3, 3>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
  return columns_rt<C, 4, 4>(a, W, cgl, cgr, cpsi, ctl, cxs, cys, slots, s);
}

}  // namespace

size_t adjoint_column_smem(int W, int precision) {
  return precision == NEGF_FP64 ? column_smem<cd>(W) : column_smem<cf>(W);
}

int adjoint_cols_per_job(int W) { return adj_ncols(W); }

int adjoint_column_occupancy(int W, int precision) {
  return precision == NEGF_FP64 ? occupancy_impl<cd>(W) : occupancy_impl<cf>(W);
}

cudaError_t launch_adjoint_sweep(const TaskDesc* d_tasks, int n_tasks, int max_W, int precision,
                                 const double* d_wire, const double* d_phi, const cd* d_sig,
                                 const uint64_t* d_ck_off, int stride, void* d_ck,
                                 int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  if (precision == NEGF_FP64) {
    const size_t smem = gj_smem<cd>(max_W);
    cudaError_t e = cudaFuncSetAttribute(adj_sweep_kernel<cd>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adj_sweep_kernel<cd><<<2 * n_tasks, kAdjThreads, smem, s>>>(
        d_tasks, n_tasks, d_wire, d_phi, d_sig, d_ck_off, stride, static_cast<cd*>(d_ck), d_err);
  } else {
    const size_t smem = gj_smem<cf>(max_W);
    cudaError_t e = cudaFuncSetAttribute(adj_sweep_kernel<cf>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    adj_sweep_kernel<cf><<<2 * n_tasks, kAdjThreads, smem, s>>>(
        d_tasks, n_tasks, d_wire, d_phi, d_sig, d_ck_off, stride, static_cast<cf*>(d_ck), d_err);
  }
  return cudaGetLastError();
}

cudaError_t launch_adjoint_expand(const TaskDesc* d_tasks, int task0, int n_group, int W, int L,
                                  int precision, const double* d_wire, const double* d_phi,
                                  const cd* d_sig, const uint64_t* d_ck_off, int stride,
                                  const void* d_ck, void* d_gl, void* d_gr, int32_t* d_err,
                                  cudaStream_t s) {
  if (n_group == 0) return cudaSuccess;
  const int nck = (L + stride - 1) / stride;
  const unsigned blocks = (unsigned)(n_group * 2 * nck);
  cudaError_t e = precision == NEGF_FP64
                      ? cudaFuncSetAttribute(adj_expand_kernel<cd>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gj_smem<cd>(W))
                      : cudaFuncSetAttribute(adj_expand_kernel<cf>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gj_smem<cf>(W));
  if (e != cudaSuccess) return e;
  if (precision == NEGF_FP64)
    adj_expand_kernel<cd><<<blocks, kAdjThreads, gj_smem<cd>(W), s>>>(
        d_tasks, task0, n_group, d_wire, d_phi, d_sig, d_ck_off, stride,
        static_cast<const cd*>(d_ck), static_cast<cd*>(d_gl), static_cast<cd*>(d_gr), d_err);
  else
    adj_expand_kernel<cf><<<blocks, kAdjThreads, gj_smem<cf>(W), s>>>(
        d_tasks, task0, n_group, d_wire, d_phi, d_sig, d_ck_off, stride,
        static_cast<const cf*>(d_ck), static_cast<cf*>(d_gl), static_cast<cf*>(d_gr), d_err);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_columns(const TaskDesc* d_tasks, int task0, int n_group, int W,
                                   int precision, int start_lead, const double* d_wire,
                                   const double* d_phi, const cd* d_sig, const double* d_gam,
                                   const void* d_wbar, const double* d_ubar, uint64_t site_off0,
                                   double* d_dV, double* d_dE, const void* d_gl, const void* d_gr,
                                   void* d_psi, void* d_tl, void* d_xs, void* d_ys, int slots,
                                   int32_t* d_err, cudaStream_t s) {
  if (n_group == 0 || slots == 0) return cudaSuccess;
  AdjArgs a{d_tasks, task0, n_group, start_lead, d_wire, d_phi, d_sig, d_gam, d_wbar, d_ubar,
            site_off0, d_dV, d_dE, d_err};                  // d_wbar: FP64, or FP32 for FP32 tables
  if (precision == NEGF_FP64)
    return columns_impl<cd>(a, W, d_gl, d_gr, d_psi, d_tl, d_xs, d_ys, slots, s);
  return columns_impl<cf>(a, W, d_gl, d_gr, d_psi, d_tl, d_xs, d_ys, slots, s);
}

}  // namespace negf
