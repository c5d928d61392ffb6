// Lead self-energies, RGF sweeps and the block-column / transition-weight kernels.
//
// Sec. III.B: the paper obtains G^r by the recursive Green's function algorithm (RGF), the
// diagonal once per sample and one column of G^r per walker step.  Here every column a table
// row needs is produced once per (wire, energy) task:
//   * lead_modes_kernel   - eigen self-energies Sigma_m and Gamma_m of the lead strips
//                           (Sec. II.A lead self-energies; Sec. III.A model)
//   * rgf_sweep_kernel    - left- and right-connected blocks g^L_k, g^R_k (one CTA per sweep)
//   * block_column_kernel - per slice m: G_mm by one more inversion, then the block column
//                           G_{k,m} = -t g^L_k G_{k+1,m} (k < m), -t g^R_k G_{k-1,m} (k > m),
//                           emitted directly as Step 6' weights (Eq. draw_i_simult and the lead
//                           probability of Step 6'); two extra CTAs per task propagate G Phi for
//                           the injection rows of Step 4/5 and the mode weights of
//                           Eq. lead_out_probability.
// W x W block inversions are Gauss-Jordan with partial pivoting in FP64 in shared memory.
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ bool finite_cd(cd v) { return isfinite(v.x) && isfinite(v.y); }

// Sine mode phi_m(a) of a W-site cross-section, m, a in [0, W).
__device__ __forceinline__ double phi_mode(int a, int m, int W) {
  return sqrt(2.0 / (W + 1)) * sinpi((double)((m + 1) * (a + 1)) / (double)(W + 1));
}

// Gauss-Jordan inversion of the W x W left half of aug [W][2W] (right half holds I on entry,
// the inverse on exit).  Partial pivoting by |a_ik|^2 (lowest index on ties).  All threads of
// the block must call it.  Returns false (uniformly) on an exactly zero pivot column.
__device__ bool gj_invert(cd* aug, int W, cd* fcol, int* s_piv) {
  const int W2 = 2 * W;
  const int tid = threadIdx.x, bd = blockDim.x, lane = tid & 31;
  for (int k = 0; k < W; ++k) {
    if (tid < 32) {
      double best = -1.0;
      int bi = k;
      for (int i = k + lane; i < W; i += 32) {
        double v = norm2(aug[i * W2 + k]);
        if (v > best) { best = v; bi = i; }
      }
      for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, best, off);
        int oi = __shfl_xor_sync(0xffffffffu, bi, off);
        if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
      }
      if (lane == 0) *s_piv = (best > 0.0 && isfinite(best)) ? bi : -1;
    }
    __syncthreads();
    const int p = *s_piv;
    if (p < 0) return false;
    if (p != k) {
      for (int j = k + tid; j < W2; j += bd) {
        cd tmp = aug[k * W2 + j];
        aug[k * W2 + j] = aug[p * W2 + j];
        aug[p * W2 + j] = tmp;
      }
    }
    __syncthreads();
    const cd inv = cdiv(mk(1.0, 0.0), aug[k * W2 + k]);
    for (int i = tid; i < W; i += bd) fcol[i] = aug[i * W2 + k];
    __syncthreads();
    for (int j = k + tid; j < W2; j += bd) aug[k * W2 + j] = aug[k * W2 + j] * inv;
    __syncthreads();
    const int span = W2 - k;
    for (int idx = tid; idx < W * span; idx += bd) {
      const int i = idx / span, j = k + idx % span;
      if (i != k) aug[i * W2 + j] = aug[i * W2 + j] - fcol[i] * aug[k * W2 + j];
    }
    __syncthreads();
  }
  return true;
}

// Boundary self-energy block Phi diag(sig) Phi^T of one lead into out [W][W] (smem).
__device__ void lead_block(const double* phi, const cd* sig, int W, cd* out) {
  for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
    const int a = idx / W, b = idx % W;
    cd acc = mk(0.0, 0.0);
    for (int m = 0; m < W; ++m) acc = acc + (phi[a * W + m] * phi[b * W + m]) * sig[m];
    out[idx] = acc;
  }
}

// aug <- [E - H_kk - Sigma_s(k) - extra | I] where extra = sum of the given W x W blocks
// scaled by the given factors (lead blocks with factor 1, connected blocks with t^2).
__device__ void build_slice(cd* aug, int W, double E, double t, const double* onsite,
                            const double* eta, int k, const cd* x1, double f1, const cd* x2,
                            double f2) {
  const int W2 = 2 * W;
  for (int idx = threadIdx.x; idx < W * W2; idx += blockDim.x) {
    const int a = idx / W2, j = idx % W2;
    cd v;
    if (j < W) {
      const int b = j;
      v = mk(0.0, 0.0);
      if (a == b) v = mk(E - onsite[k * W + a], 0.5 * eta[k * W + a]);
      if (a - b == 1 || b - a == 1) v.x += t;
      if (x1) v = v - f1 * x1[a * W + b];
      if (x2) v = v - f2 * x2[a * W + b];
    } else {
      v = mk((j - W) == a ? 1.0 : 0.0, 0.0);
    }
    aug[idx] = v;
  }
}

__global__ void lead_modes_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, cd* sig,
                                  double* gam, int32_t* err) {
  const int task = blockIdx.x;
  if (task >= n_tasks) return;
  const TaskDesc d = tasks[task];
  for (int m = threadIdx.x; m < d.W; m += blockDim.x) {
    cd s;
    double g;
    if (d.lead_model == NEGF_LEAD_WIDE_BAND) {
      s = mk(0.0, -0.5 * d.gamma_lead);
      g = d.gamma_lead;
    } else {
      // eps_m = -2t cos((m+1) pi / (W+1)); Sigma_m = t^2 g_s(E - eps_m), retarded branch
      const double eps = -2.0 * d.t * cospi((double)(m + 1) / (double)(d.W + 1));
      const double e = d.E - eps, two_t = 2.0 * d.t;
      if (fabs(fabs(e) - two_t) <= 1e-12 * d.t) atomicOr(err, ERR_INPUT);
      if (fabs(e) < two_t) {
        const double r = sqrt(two_t * two_t - e * e);
        s = mk(0.5 * e, -0.5 * r);
        g = r;
      } else {
        const double r = sqrt(e * e - two_t * two_t);
        s = mk(0.5 * (e - copysign(r, e)), 0.0);
        g = 0.0;
      }
    }
    sig[d.lead_off + m] = s;
    gam[d.lead_off + m] = g;
  }
}

// One CTA per (task, direction): direction 0 = left sweep g^L_0..g^L_{L-2} (Sigma_L at slice
// 0); direction 1 = right sweep g^R_{L-1}..g^R_1 (Sigma_R at slice L-1).
__global__ void __launch_bounds__(kThreads) rgf_sweep_kernel(
    const TaskDesc* __restrict__ tasks, const double* __restrict__ wire, const cd* __restrict__ sig,
    cd* gL, cd* gR, int32_t* err) {
  const TaskDesc d = tasks[blockIdx.x];
  const int dir = blockIdx.y;
  const int W = d.W, L = d.L, W2 = 2 * W;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd* aug = reinterpret_cast<cd*>(smem_raw);           // W x 2W
  cd* prev = aug + W * W2;                              // W x W
  cd* lblk = prev + W * W;                              // W x W
  cd* fcol = lblk + W * W;                              // W
  double* phi = reinterpret_cast<double*>(fcol + W);    // W x W
  int* s_piv = reinterpret_cast<int*>(phi + W * W);
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  const int steps = L - 1;
  if (steps <= 0) return;
  for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x)
    phi[idx] = phi_mode(idx / W, idx % W, W);
  __syncthreads();
  lead_block(phi, sig + d.lead_off, W, lblk);
  __syncthreads();
  cd* out = dir == 0 ? gL : gR;
  for (int s = 0; s < steps; ++s) {
    const int k = dir == 0 ? s : L - 1 - s;
    if (s == 0) build_slice(aug, W, d.E, d.t, onsite, eta, k, lblk, 1.0, nullptr, 0.0);
    else build_slice(aug, W, d.E, d.t, onsite, eta, k, prev, d.t * d.t, nullptr, 0.0);
    __syncthreads();
    if (!gj_invert(aug, W, fcol, s_piv)) {
      if (threadIdx.x == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
    cd* dst = out + d.g_off + (uint64_t)k * W * W;
    bool bad = false;
    for (int idx = threadIdx.x; idx < W * W; idx += blockDim.x) {
      const cd v = aug[(idx / W) * W2 + W + idx % W];
      prev[idx] = v;
      dst[idx] = v;
      bad |= !finite_cd(v);
    }
    if (bad) atomicOr(err, ERR_NONFINITE);
    __syncthreads();
  }
}

template <typename R> struct CT;
template <> struct CT<double> { using T = cd; };
template <> struct CT<float> { using T = cf; };
__device__ __forceinline__ cd to_c(cd v, double) { return v; }
__device__ __forceinline__ cf to_c(cd v, float) { return cf{(float)v.x, (float)v.y}; }

// Shared-memory layout of block_column_kernel for slice width W and propagation type C:
//   region0 : max(W x 2W cd (inversion), 4 W x W C (propagation X0, X1, Gb, Xs))
//   phi, rs, red : W x W double each;  lblk : W x W cd;  fcol : W cd;  arow, lgam : W double
template <typename C>
__host__ __device__ inline size_t column_region0(int W) {
  const size_t a = sizeof(cd) * (size_t)(2 * W * W);
  const size_t b = sizeof(C) * (size_t)(4 * W * W);
  return ((a > b ? a : b) + 15) & ~size_t(15);
}
template <typename C>
__host__ __device__ inline size_t column_smem_bytes(int W) {
  return column_region0<C>(W) + sizeof(double) * (size_t)(3 * W * W) +
         sizeof(cd) * (size_t)(W * W + W) + sizeof(double) * (size_t)(2 * W) + 16;
}

// Per block column: see the file header.  blockIdx.y = m in [0, L) for site column m,
// L for the injection rows of lead L, L+1 for those of lead R.
template <typename R>
__global__ void __launch_bounds__(kThreads) block_column_kernel(
    const TaskDesc* __restrict__ tasks, const double* __restrict__ wire, const cd* __restrict__ sig,
    const double* __restrict__ gam, const cd* __restrict__ gL, const cd* __restrict__ gR,
    R* __restrict__ weights, double* __restrict__ rowsum, double* __restrict__ mode_w,
    double* __restrict__ cvals, int32_t* err) {
  using C = typename CT<R>::T;
  const TaskDesc d = tasks[blockIdx.x];
  const int W = d.W, L = d.L, n = d.n, K = d.K, W2 = 2 * W;
  const int y = blockIdx.y;
  if (y >= L + 2) return;
  const int tid = threadIdx.x, bd = blockDim.x;
  const bool inj = y >= L;
  const int p = y - L;                        // injection lead (valid if inj)
  const int m0 = inj ? (p == 0 ? 0 : L - 1) : y;

  extern __shared__ __align__(16) unsigned char smem_raw[];
  cd* aug = reinterpret_cast<cd*>(smem_raw);                       // W x 2W (inversion)
  C* X0 = reinterpret_cast<C*>(smem_raw);                          // propagation, after it
  C* X1 = X0 + W * W;
  C* Gb = X1 + W * W;
  C* Xs = Gb + W * W;
  double* phi = reinterpret_cast<double*>(smem_raw + column_region0<C>(W));
  double* rs = phi + W * W;                                        // partial row sums [b][a]
  double* red = rs + W * W;                                        // reduction scratch
  cd* lblk = reinterpret_cast<cd*>(red + W * W);                   // lead / start block
  cd* fcol = lblk + W * W;
  double* arow = reinterpret_cast<double*>(fcol + W);              // A_ii per row
  double* lgam = arow + W;                                         // lead Gamma_m
  __shared__ int s_piv;

  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + n;
  const double t = d.t;
  for (int idx = tid; idx < W * W; idx += bd) {
    phi[idx] = phi_mode(idx / W, idx % W, W);
    rs[idx] = 0.0;
  }
  for (int m = tid; m < W; m += bd) lgam[m] = gam[d.lead_off + m];
  __syncthreads();

  // ---- diagonal block G_{m0 m0} in FP64: invert E - H - Sigma_s - left - right
  {
    const cd* left;
    const cd* right;
    double fl, fr;
    const bool lead_here = (m0 == 0) || (m0 == L - 1);
    if (lead_here) lead_block(phi, sig + d.lead_off, W, lblk);
    __syncthreads();
    if (m0 == 0) { left = lblk; fl = 1.0; }
    else { left = gL + d.g_off + (uint64_t)(m0 - 1) * W * W; fl = t * t; }
    if (m0 == L - 1) { right = lblk; fr = 1.0; }
    else { right = gR + d.g_off + (uint64_t)(m0 + 1) * W * W; fr = t * t; }
    build_slice(aug, W, d.E, t, onsite, eta, m0, left, fl, right, fr);
    __syncthreads();
    if (!gj_invert(aug, W, fcol, &s_piv)) {
      if (tid == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
  }
  // start block S = G_mm (site column) or G_mm Phi (injection) in FP64, kept in lblk
  for (int idx = tid; idx < W * W; idx += bd) {
    const int a = idx / W, b = idx % W;
    cd v;
    if (!inj) {
      v = aug[a * W2 + W + b];
    } else {
      v = mk(0.0, 0.0);
      for (int c = 0; c < W; ++c) v = v + phi[c * W + b] * aug[a * W2 + W + c];
    }
    lblk[idx] = v;
  }
  __syncthreads();
  // A of each row: site b: -2 Im G_bb;  mode mu: -2 Im (Phi^T G Phi)_{mu mu}
  if (tid < W) {
    const int b = tid;
    double A;
    if (!inj) {
      A = -2.0 * lblk[b * W + b].y;
    } else {
      double im = 0.0;
      for (int a = 0; a < W; ++a) im += phi[a * W + b] * lblk[a * W + b].y;
      A = -2.0 * im;
      const double mw = lgam[b] * A;
      mode_w[d.mode_off + p * W + b] = mw;
      red[b] = mw;
    }
    arow[b] = A;
  }
  __syncthreads();
  if (inj && tid == 0) {
    double c = 0.0;
    for (int b = 0; b < W; ++b) c += red[b];
    cvals[blockIdx.x * 2 + p] = c;
    rowsum[d.row_base + d.rows + p] = c;
  }
  // the inversion buffer is dead: convert the start block into the propagation precision
  for (int idx = tid; idx < W * W; idx += bd) {
    const C v = to_c(lblk[idx], R(0));
    X0[idx] = v;
    Xs[idx] = v;
  }
  __syncthreads();

  const int row0 = inj ? n + p * W : m0 * W;
  R* wrow = weights + d.wt_off;
  // Emit the weights of block k held in X (X[a][b] = G_{(k,a),(m0,b)}, or (G Phi)_{(k,a),mu}):
  // site columns gamma_(k,a) |X[a][b]|^2, and at the boundary slices the lead columns
  // sum_nu Gamma_nu |(Phi^T X)_{nu b}|^2 = <psi_b|Gamma_lead|psi_b>.  Partial row sums in rs.
  auto emit = [&](const C* X, int k) {
    for (int idx = tid; idx < W * W; idx += bd) {
      const int b = idx / W, a = idx % W;
      const R w = (R)eta[k * W + a] * norm2(X[a * W + b]);
      wrow[(uint64_t)(row0 + b) * K + k * W + a] = w;
      rs[idx] += (double)w;
    }
    if (k == 0 || k == L - 1) {
      for (int idx = tid; idx < W * W; idx += bd) {
        const int nu = idx / W, b = idx % W;
        C acc = C{0, 0};
        for (int a = 0; a < W; ++a) acc = acc + (R)phi[a * W + nu] * X[a * W + b];
        red[idx] = lgam[nu] * (double)norm2(acc);
      }
      __syncthreads();
      if (tid < W) {
        const int b = tid;
        double s = 0.0;
        for (int nu = 0; nu < W; ++nu) s += red[nu * W + b];
        const R wl = (R)s;
        if (k == 0) wrow[(uint64_t)(row0 + b) * K + n + 0] = wl;
        if (k == L - 1) wrow[(uint64_t)(row0 + b) * K + n + 1] = wl;
        rs[b * W] += (double)wl * (double)((k == 0) + (k == L - 1));
      }
    }
    __syncthreads();
  };
  emit(X0, m0);
  C* cur = X0;
  C* nxt = X1;
  // towards slice 0: X_k = -t g^L_k X_{k+1}
  for (int k = m0 - 1; k >= 0; --k) {
    const cd* gk = gL + d.g_off + (uint64_t)k * W * W;
    for (int idx = tid; idx < W * W; idx += bd) Gb[idx] = to_c(gk[idx], R(0));
    __syncthreads();
    for (int idx = tid; idx < W * W; idx += bd) {
      const int a = idx / W, b = idx % W;
      C acc = C{0, 0};
      for (int c = 0; c < W; ++c) acc = acc + Gb[a * W + c] * cur[c * W + b];
      nxt[idx] = (R)(-t) * acc;
    }
    __syncthreads();
    C* tmp = cur; cur = nxt; nxt = tmp;
    emit(cur, k);
  }
  // towards slice L-1 from the saved start: X_k = -t g^R_k X_{k-1}
  for (int idx = tid; idx < W * W; idx += bd) X0[idx] = Xs[idx];
  cur = X0;
  nxt = X1;
  __syncthreads();
  for (int k = m0 + 1; k < L; ++k) {
    const cd* gk = gR + d.g_off + (uint64_t)k * W * W;
    for (int idx = tid; idx < W * W; idx += bd) Gb[idx] = to_c(gk[idx], R(0));
    __syncthreads();
    for (int idx = tid; idx < W * W; idx += bd) {
      const int a = idx / W, b = idx % W;
      C acc = C{0, 0};
      for (int c = 0; c < W; ++c) acc = acc + Gb[a * W + c] * cur[c * W + b];
      nxt[idx] = (R)(-t) * acc;
    }
    __syncthreads();
    C* tmp = cur; cur = nxt; nxt = tmp;
    emit(cur, k);
  }
  // FP64 row sums and the sum-rule check (rows must add up to <i|A|i>, Sec. II.D)
  if (tid < W) {
    const int b = tid;
    double s = 0.0;
    for (int a = 0; a < W; ++a) s += rs[b * W + a];
    rowsum[d.row_base + row0 + b] = s;
    const double A = arow[b];
    const double tol = sizeof(R) == 8 ? 1e-6 : 1e-2;
    if (!isfinite(s) || s < 0.0) atomicOr(err, ERR_NONFINITE);
    else if (A > 1e-300 && fabs(s - A) > tol * A) atomicOr(err, ERR_ROWSUM);
  }
}

}  // namespace

cudaError_t launch_lead_modes(const TaskDesc* d_tasks, int n_tasks, int max_W, cd* d_sig,
                              double* d_gam, int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  lead_modes_kernel<<<n_tasks, 64, 0, s>>>(d_tasks, n_tasks, d_sig, d_gam, d_err);
  return cudaGetLastError();
}

static size_t sweep_smem(int W) {
  return sizeof(cd) * (size_t)(W * 2 * W + W * W + W * W + W) + sizeof(double) * W * W + 16;
}

cudaError_t launch_rgf_sweep(const TaskDesc* d_tasks, int n_tasks, int max_W,
                             const double* d_wire, const cd* d_sig, cd* d_gL, cd* d_gR,
                             int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  const size_t smem = sweep_smem(max_W);
  cudaError_t e = cudaFuncSetAttribute(rgf_sweep_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rgf_sweep_kernel<<<dim3(n_tasks, 2), kThreads, smem, s>>>(d_tasks, d_wire, d_sig, d_gL, d_gR,
                                                            d_err);
  return cudaGetLastError();
}


cudaError_t launch_block_columns(const TaskDesc* d_tasks, int n_tasks, int max_W, int max_L,
                                 int precision, const double* d_wire, const cd* d_sig,
                                 const double* d_gam, const cd* d_gL, const cd* d_gR,
                                 void* d_weights, double* d_rowsum, double* d_mode_w,
                                 double* d_c, int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  dim3 grid(n_tasks, max_L + 2);
  cudaError_t e;
  if (precision == NEGF_FP64) {
    const size_t smem = column_smem_bytes<cd>(max_W);
    e = cudaFuncSetAttribute(block_column_kernel<double>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    block_column_kernel<double><<<grid, kThreads, smem, s>>>(
        d_tasks, d_wire, d_sig, d_gam, d_gL, d_gR, static_cast<double*>(d_weights), d_rowsum,
        d_mode_w, d_c, d_err);
  } else {
    const size_t smem = column_smem_bytes<cf>(max_W);
    e = cudaFuncSetAttribute(block_column_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    block_column_kernel<float><<<grid, kThreads, smem, s>>>(
        d_tasks, d_wire, d_sig, d_gam, d_gL, d_gR, static_cast<float*>(d_weights), d_rowsum,
        d_mode_w, d_c, d_err);
  }
  return cudaGetLastError();
}

}  // namespace negf
