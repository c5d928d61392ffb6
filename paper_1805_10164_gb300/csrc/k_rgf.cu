// Lead self-energies, RGF sweeps and the block-column / transition-weight kernels.
//
// Sec. III.B: the paper obtains G^r by the recursive Green's function algorithm (RGF), the
// diagonal once per sample and one column of G^r per walker step.  Here every column a table
// row needs is produced once per (wire, energy) task:
//   * lead_modes_kernel   - eigen self-energies Sigma_m and Gamma_m of the lead strips
//                           (Sec. II.A lead self-energies; Sec. III.A model)
//   * rgf_sweep_*_kernel  - left- and right-connected blocks g^L_k, g^R_k (one warp per task
//                           and direction in registers for complex64 W <= 16, one CTA
//                           otherwise; the sweep is a serial chain of W x W inversions)
//   * diag_*_kernel       - per slice m: G_mm by one more inversion; for the boundary slices
//                           also G Phi, the A of every row (for the sum-rule check), the mode
//                           weights of Eq. lead_out_probability and c_p = Tr[Gamma_p A]
//                           (Eq. elast_lin_xpq)
//   * chain_*_kernel      - per slice m and direction, the block column
//                           G_{k,m} = -t g^L_k G_{k+1,m} (k < m), -t g^R_k G_{k-1,m} (k > m),
//                           emitted directly as Step 6' weights (Eq. draw_i_simult and the lead
//                           probability of Step 6'); the two injection columns propagate G Phi
//                           for the rows of Steps 4-5.
// W x W block inversions are Gauss-Jordan: in registers by one warp for complex64 W <= 16, in
// shared memory by one CTA otherwise; partial pivoting except on slices where every site
// dephases (see gj_rows).  All of it runs in the precision of the tables: complex128 for
// NEGF_FP64, complex64 for NEGF_FP32; the lead self-energies, whose square roots are singular
// at the sub-band edges, are FP64 in both and rounded once.
#include <cuda_runtime.h>
#include <math.h>

#include "gj.cuh"
#include "negf_internal.cuh"

namespace negf {
namespace {

// Sine mode phi_m(a) of a W-site cross-section, m, a in [0, W).
__device__ __forceinline__ double phi_mode(int a, int m, int W) {
  return sqrt(2.0 / (W + 1)) * sinpi((double)((m + 1) * (a + 1)) / (double)(W + 1));
}

__global__ void lead_modes_kernel(const TaskDesc* __restrict__ tasks, int n_tasks,
                                  const double* __restrict__ wire, double* phi, float* phi32,
                                  float* eta32, cd* sig, double* gam, int32_t* err) {
  const int task = blockIdx.x;
  if (task >= n_tasks) return;
  const TaskDesc d = tasks[task];
  if (d.e_idx == 0) {
    // once per wire: transverse modes (a multi-orbital slice's come from slice_modes_kernel)
    // and the FP32 copy of eta
    if (!d.slice_h)
      for (int idx = threadIdx.x; idx < d.W * d.W; idx += blockDim.x) {
        const double v = phi_mode(idx / d.W, idx % d.W, d.W);
        phi[d.phi_off + idx] = v;
        phi32[d.phi_off + idx] = (float)v;
      }
    const double* eta = wire + d.onsite_off + d.n;
    for (int i = threadIdx.x; i < d.n; i += blockDim.x) eta32[d.onsite_off / 2 + i] = (float)eta[i];
  }
  for (int m = threadIdx.x; m < d.W; m += blockDim.x) {
    cd s;
    double g;
    if (d.lead_model == NEGF_LEAD_WIDE_BAND) {
      s = mk(0.0, -0.5 * d.gamma_lead);
      g = d.gamma_lead;
    } else {
      // eps_m = -2t cos((m+1) pi / (W+1)) (a slice block: its m-th eigenvalue);
      // Sigma_m = t^2 g_s(E - eps_m), retarded branch
      const double eps = d.slice_h
                             ? wire[d.onsite_off + 2 * (uint64_t)d.n + (uint64_t)d.W * d.W + m]
                             : -2.0 * d.t * cospi((double)(m + 1) / (double)(d.W + 1));
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

// ---- CTA-wide inversions (any W <= 64; complex128, and complex64 above W = 16) -------------
// cta_gj: the slice block sits in shared memory and is inverted in place by Gauss-Jordan (no
// augmented identity):
//   pivot k:  a_kk <- 1/a_kk;  a_kj <- a_kj / a_kk;  a_ik <- -a_ik / a_kk;
//             a_ij <- a_ij - (a_ik / a_kk) a_kj            (i, j != k)
// with two barriers per pivot: the pivot row (1/a_kk formed once, in a_kk's slot) and the
// pivot column are copied out, then every thread updates its entries with a_kj / a_kk formed
// once per thread.  Thread t owns column t mod W of rows t / W, t / W + R,
// ... (R = threads / W), so that a warp touches consecutive entries of one row.  On a
// slice where every site dephases no pivot search is needed (see gj_rows); otherwise rows are
// interchanged by partial pivoting and the inverse's columns unscrambled at the end.  The
// diagonal blocks use it, and the sweeps on slices with an undephased site.
//
// The complex64 sweeps above W = 16 (rgf_sweep_cta_kernel) run it on the block in shared
// memory with 1024 threads.  The complex128 sweeps (rgf_sweep_rows_kernel) keep the block in
// registers instead: thread t owns column j = t mod W of rows g, g + RG, g + 2 RG, ...
// (g = t / W, RG = ceil(W / RPT) row groups of at most RPT rows), and a pivot costs one
// barrier: the owners of row k publish it, the owners of column k publish that column, and the
// owner of a_kk publishes 1/a_kk, into one of two buffers (alternating with k, so that the next
// pivot's writes cannot overtake this pivot's reads); then every thread updates its rows.  On
// GB300's FP64 pipe the arithmetic of a pivot dominates, and this form computes the reciprocal
// once per pivot instead of once per thread.  The next slice's matrix E - H - Sigma_s - t^2 g_k
// is formed in the same registers while g_k is stored.
constexpr int kSweepThreads = 256;       // diagonal blocks: many CTAs
constexpr int kSweepCtaThreads = 1024;   // complex64 sweeps: few serial chains, one CTA per SM
constexpr int kSweepRowsThreads = 256;   // complex128 sweeps
constexpr int kSweepRegMaxW = 16;        // complex64 sweeps up to this width: one warp each

template <typename C>
__host__ __device__ inline size_t sweep_rows_bytes(int W) {
  // A W x W | pivot rows 2 x 64 | pivot columns 2 x 64 | 1/pivot 2 (complex) | phi W x W
  // double | perm 64, flag (int)
  return sizeof(C) * (size_t)(W * W + 4 * 64 + 2) + sizeof(double) * (size_t)(W * W) +
         sizeof(int) * (size_t)(64 + 2);
}

// In-place inverse of the register-held block (see above; no pivot search: the caller takes
// it on slices where every site dephases, gj_rows says why that is safe).  i_m = g + RG m are
// this thread's rows, valid while i_m < W; false (uniformly) on a zero or non-finite pivot.
template <typename C, int RPT>
__device__ bool gj_regcols(C (&a)[RPT], int W, int RG, int g, int j, bool own, C* rowk,
                           C* fcol, C* sinv) {
  int kr = 0, km = 0;                       // pivot k = kr + RG km: its row group and slot
  for (int k = 0; k < W; ++k) {
    const int b = k & 1;
    C* rk = rowk + 64 * b;
    C* fc = fcol + 64 * b;
    if (own && g == kr) {
      C v = a[0];
#pragma unroll
      for (int m = 1; m < RPT; ++m)
        if (m == km) v = a[m];
      rk[j] = v;
      if (j == k) sinv[b] = cdiv(mkc(1.0, 0.0, C{}), v);
    }
    if (own && j == k) {
#pragma unroll
      for (int m = 0; m < RPT; ++m)
        if (g + RG * m < W) fc[g + RG * m] = a[m];
    }
    __syncthreads();
    const C inv = sinv[b];
    if (!finite_c(inv)) return false;       // every thread reads the same value
    if (own) {
      if (j != k) {
        const C t = rk[j] * inv;            // a_kj / a_kk
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          const int i = g + RG * m;
          if (i < W) {
            const C v = a[m] - fc[i] * t;
            a[m] = i == k ? t : v;
          }
        }
      } else {
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
          const int i = g + RG * m;
          if (i < W) {
            const C v = mkc(0.0, 0.0, C{}) - fc[i] * inv;
            a[m] = i == k ? inv : v;
          }
        }
      }
    }
    if (++kr == RG) {
      kr = 0;
      ++km;
    }
  }
  return true;
}

template <typename C, int RPT>
__device__ __forceinline__ void sweep_rows_body(const TaskDesc& d, int dir,
                                               const double* __restrict__ wire,
                                               const double* __restrict__ phig,
                                               const cd* __restrict__ sig, C* gL, C* gR,
                                               int32_t* err, unsigned char* smem_raw) {
  using R = typename Real<C>::T;
  const int W = d.W, L = d.L, WW = W * W;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int RG = (W + RPT - 1) / RPT;
  const int j = tid % W, g = tid / W;
  const bool own = g < RG;
  C* A = reinterpret_cast<C*>(smem_raw);   // the block, for the pivoted inversion only
  C* rowk = A + WW;
  C* fcol = rowk + 2 * 64;
  C* sinv = fcol + 2 * 64;
  double* phi = reinterpret_cast<double*>(sinv + 2);
  int* perm = reinterpret_cast<int*>(phi + WW);
  int* flag = perm + 64;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  const cd* sg = sig + d.lead_off;
  for (int idx = tid; idx < WW; idx += nth) phi[idx] = phig[d.phi_off + idx];
  __syncthreads();
  // first slice of the sweep: E - H - Sigma_s - Phi diag(sigma) Phi^T (the lead block in FP64)
  const int kf = dir == 0 ? 0 : L - 1;
  C a[RPT];
#pragma unroll
  for (int m = 0; m < RPT; ++m) {
    const int i = g + RG * m;
    a[m] = mkc(0.0, 0.0, C{});
    if (own && i < W) {
      cd acc = mk(0.0, 0.0);
      for (int q = 0; q < W; ++q) acc = acc + (phi[i * W + q] * phi[j * W + q]) * sg[q];
      a[m] = slice_entry<C>(i, j, kf, W, d.E, d.t, onsite, eta, slice_block(d, onsite)) - to_c(acc, C{});
    }
  }
  C* out = dir == 0 ? gL : gR;
  const R tt = (R)(d.t * d.t);
  for (int s = 0; s < L - 1; ++s) {
    const int k = dir == 0 ? s : L - 1 - s;
    const bool deph = __syncthreads_and(tid >= W || eta[k * W + tid] > 0.0);
    bool ok;
    if (deph) {
      ok = gj_regcols<C, RPT>(a, W, RG, g, j, own, rowk, fcol, sinv);
    } else {
      // an undephased site: partial pivoting on the block in shared memory
#pragma unroll
      for (int m = 0; m < RPT; ++m)
        if (own && g + RG * m < W) A[(g + RG * m) * W + j] = a[m];
      __syncthreads();
      ok = cta_gj(A, rowk, fcol, perm, flag, W, true);
      __syncthreads();
#pragma unroll
      for (int m = 0; m < RPT; ++m)
        if (own && g + RG * m < W) a[m] = A[(g + RG * m) * W + j];
    }
    if (!ok) {
      if (tid == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
    // store g_k; form the next slice: E - H - Sigma_s - t^2 g_k
    C* dst = out + d.g_off + (uint64_t)k * WW;
    const bool more = s + 1 < L - 1;
    const int kn = dir == 0 ? s + 1 : L - 2 - s;
    bool bad = false;
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
      const int i = g + RG * m;
      if (own && i < W) {
        const C v = a[m];
        dst[i * W + j] = v;
        bad |= !finite_c(v);
        if (more) a[m] = slice_entry<C>(i, j, kn, W, d.E, d.t, onsite, eta, slice_block(d, onsite)) - tt * v;
      }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(err, ERR_NONFINITE);
  }
}

__global__ void __launch_bounds__(kSweepRowsThreads) rgf_sweep_rows_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, const double* __restrict__ wire,
    const double* __restrict__ phig, const cd* __restrict__ sig, cd* gL, cd* gR, int32_t* err) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int job = blockIdx.x;
  if (job >= 2 * n_tasks) return;
  const TaskDesc d = tasks[job >> 1];
  const int dir = job & 1;
  if (d.L < 2 || d.W > 64) return;
  // rows per thread: W <= 16 -> 4, W <= 32 -> 8, W <= 64 -> 16 (at most 4 row groups, so that
  // kSweepRowsThreads = 256 threads cover every width)
  if (d.W <= 16)
    sweep_rows_body<cd, 4>(d, dir, wire, phig, sig, gL, gR, err, smem_raw);
  else if (d.W <= 32)
    sweep_rows_body<cd, 8>(d, dir, wire, phig, sig, gL, gR, err, smem_raw);
  else
    sweep_rows_body<cd, 16>(d, dir, wire, phig, sig, gL, gR, err, smem_raw);
}

template <typename C>
__host__ __device__ inline size_t sweep_smem_bytes(int W) {
  // A W x W | pivot row W | multipliers W (complex) | phi W x W double | perm W, flag (int)
  return sizeof(C) * (size_t)(W * W + 2 * W) + sizeof(double) * (size_t)(W * W) +
         sizeof(int) * (size_t)(W + 2);
}

// complex64 sweeps of width min_W .. 64 with the block in shared memory (cta_gj)
__global__ void __launch_bounds__(kSweepCtaThreads) rgf_sweep_cta_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, const double* __restrict__ wire,
    const double* __restrict__ phig, const cd* __restrict__ sig, cf* gL, cf* gR, int32_t* err,
    int min_W) {
  using C = cf;
  using R = float;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int job = blockIdx.x;
  if (job >= 2 * n_tasks) return;
  const TaskDesc d = tasks[job >> 1];
  const int dir = job & 1;
  const int W = d.W, L = d.L, WW = W * W;
  const int tid = threadIdx.x, nth = blockDim.x;
  if (L < 2 || W > 64 || W < min_W) return;       // narrower tasks: rgf_sweep_reg_kernel
  C* A = reinterpret_cast<C*>(smem_raw);
  C* rowk = A + WW;
  C* fcol = rowk + W;
  double* phi = reinterpret_cast<double*>(fcol + W);
  int* perm = reinterpret_cast<int*>(phi + WW);
  int* flag = perm + W;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  const cd* sg = sig + d.lead_off;
  for (int idx = tid; idx < WW; idx += nth) phi[idx] = phig[d.phi_off + idx];
  __syncthreads();
  // first slice of the sweep: E - H - Sigma_s - Phi diag(sigma) Phi^T (the lead block in FP64)
  const int kf = dir == 0 ? 0 : L - 1;
  for (int idx = tid; idx < WW; idx += nth) {
    const int a = idx / W, b = idx - a * W;
    cd acc = mk(0.0, 0.0);
    for (int m = 0; m < W; ++m) acc = acc + (phi[a * W + m] * phi[b * W + m]) * sg[m];
    A[idx] = slice_entry<C>(a, b, kf, W, d.E, d.t, onsite, eta, slice_block(d, onsite)) - to_c(acc, C{});
  }
  C* out = dir == 0 ? gL : gR;
  const R tt = (R)(d.t * d.t);
  for (int s = 0; s < L - 1; ++s) {
    const int k = dir == 0 ? s : L - 1 - s;
    const bool deph = __syncthreads_and(tid >= W || eta[k * W + tid] > 0.0);
    if (!cta_gj(A, rowk, fcol, perm, flag, W, !deph)) {
      if (tid == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
    // store g_k; build the next slice in place: E - H - Sigma_s - t^2 g_k
    C* dst = out + d.g_off + (uint64_t)k * WW;
    const bool more = s + 1 < L - 1;
    const int kn = dir == 0 ? s + 1 : L - 2 - s;
    bool bad = false;
    for (int idx = tid; idx < WW; idx += nth) {
      const C v = A[idx];
      dst[idx] = v;
      bad |= !finite_c(v);
      if (more) {
        const int a = idx / W, b = idx - a * W;
        A[idx] = slice_entry<C>(a, b, kn, W, d.E, d.t, onsite, eta, slice_block(d, onsite)) - tt * v;
      }
    }
    if (__syncthreads_or(bad) && tid == 0) atomicOr(err, ERR_NONFINITE);
  }
}

// ---- register-resident variants for complex64 blocks with W <= 16 ------------------------
// Lane i < W holds row i of the augmented matrix [M | I] in registers: a[0, MAXW) the slice
// matrix, a[MAXW, 2 MAXW) the identity (then the inverse).  Gauss-Jordan pivots without moving
// rows: at step k the pivot is the unused row with the largest |a_ik|^2 (one warp max-reduction
// of a 32-bit key), the pivot lane publishes its row in shared memory (broadcast loads cost far
// less than two shuffles per element), and every other row eliminates column k.  Row i of the inverse then sits in the lane that pivoted column i.  The kernels call
// these with MAXW equal to the block width, so that every column index is a constant.

// Gauss-Jordan on the register-held rows; on return lane i < W holds row i of the inverse in
// a[MAXW, MAXW + W).  Returns false uniformly on a zero or non-finite pivot.
//
// At step k the pivot lane computes 1 / a_pk itself and publishes it with its row as it stands;
// every other row subtracts (a_ik / a_pk) times that row.  Pivot rows are not rescaled during
// the elimination (a pivot row only ever changes by multiples of later pivot rows, so it stays
// a_pk times its normalised form); each is divided by its own pivot at the end.  This keeps the
// reciprocal off the other lanes' dependency chain.
//
// pivot == false eliminates in row order without a pivot search.  The caller takes it only when
// every site of the slice dephases (eta_i > 0): the slice matrix E - H - Sigma is then complex
// symmetric with imaginary part >= diag(eta / 2) > 0 (the lead and connected-block terms add
// positive semidefinite imaginary parts, since Im G^r <= 0), its Schur complements keep that
// property, so no pivot vanishes and elimination without pivoting is stable for this class.
// The row goes through shared memory as 16-byte pairs of entries: on a lone warp each shared
// memory (or shuffle) instruction costs about as much as a dozen arithmetic ones, so the
// broadcast is made of as few, and as wide, accesses as possible.
// srow: 2 W + 2 complex64 of this warp's shared memory, 16-byte aligned.
template <int W>
__device__ bool gj_rows(cf (&a)[2 * W], bool pivot, cf* srow) {
  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  float4* row = reinterpret_cast<float4*>(srow);   // row[q]: entries 2q, 2q + 1; row[W]: 1/pivot
  bool used = lane >= W;                           // lanes without a row never pivot
  int src = lane;
  cf own_inv{1.f, 0.f};                            // 1 / pivot of the step this lane pivoted
#pragma unroll
  for (int k = 0; k < W; ++k) {
    int p = k;
    if (pivot) {
      // key: |a_ik|^2 (non-negative, so its bits order like the value) with its low 5 mantissa
      // bits replaced by 31 - lane: the largest candidate wins, lower lanes on near-ties
      const float v = used ? 0.f : norm2(a[k]);
      const unsigned key = (__float_as_uint(v) & ~31u) | (unsigned)(31 - lane);
      const unsigned best = __reduce_max_sync(FULL, key);
      const unsigned mag = best & ~31u;
      if (mag == 0u || mag >= 0x7f800000u) return false;   // zero, inf or NaN pivot
      p = 31 - (int)(best & 31u);
      if (lane == k) src = p;
    }
    const bool me = lane == p;
    __syncwarp();                                  // the previous step's row has been read
    if (me) {
      const float rr = __frcp_rn(norm2(a[k]));      // inf for a zero pivot: caught below
      own_inv = cf{a[k].x * rr, -a[k].y * rr};
      row[W] = make_float4(own_inv.x, own_inv.y, 0.f, 0.f);
#pragma unroll
      for (int q = (k + 1) / 2; q < W; ++q)
        row[q] = make_float4(a[2 * q].x, a[2 * q].y, a[2 * q + 1].x, a[2 * q + 1].y);
    }
    __syncwarp();
    const float4 iv = row[W];
    if (!pivot && !(isfinite(iv.x) && isfinite(iv.y) && (iv.x != 0.f || iv.y != 0.f)))
      return false;
    const cf f = me ? cf{0.f, 0.f} : a[k] * cf{iv.x, iv.y};
#pragma unroll
    for (int q = (k + 1) / 2; q < W; ++q) {
      const float4 r = row[q];
      if (2 * q > k) a[2 * q] = a[2 * q] - f * cf{r.x, r.y};
      a[2 * q + 1] = a[2 * q + 1] - f * cf{r.z, r.w};
    }
    used |= me;
  }
#pragma unroll
  for (int j = W; j < 2 * W; ++j) {
    a[j] = a[j] * own_inv;
    if (pivot) {
      a[j].x = __shfl_sync(FULL, a[j].x, src);
      a[j].y = __shfl_sync(FULL, a[j].y, src);
    }
  }
  return true;
}

// In-place Gauss-Jordan inversion without pivoting: lane j < W holds column j of the matrix in
// a[0, W) on entry and column j of its inverse on return.  At step k the pivot column is
// broadcast through shared memory and every lane updates its own column from registers:
//   lane j != k:  a_kj <- a_kj / a_kk,  a_ij <- a_ij - a_ik a_kj / a_kk  (i != k)
//   lane k:       a_kk <- 1 / a_kk,     a_ik <- -a_ik / a_kk             (i != k)
// (both written as a_ij - c_i piv with piv = a_kj / a_kk, or 1 + 1 / a_kk on lane k).  Only for
// matrices whose imaginary part is positive definite (see gj_rows).  Returns false uniformly on
// a zero or non-finite pivot.  scol: W + 1 complex64 of shared memory, 16-byte aligned.
template <int W>
__device__ bool gj_cols(cf (&a)[W], cf* scol) {
  const int lane = threadIdx.x & 31;
  float4* col = reinterpret_cast<float4*>(scol);
  constexpr int W2 = (W + 1) / 2;
#pragma unroll
  for (int k = 0; k < W; ++k) {
    __syncwarp();                                  // the previous column has been read
    if (lane == k) {
#pragma unroll
      for (int q = 0; q < W2; ++q)
        col[q] = make_float4(a[2 * q].x, a[2 * q].y, 2 * q + 1 < W ? a[2 * q + 1].x : 0.f,
                             2 * q + 1 < W ? a[2 * q + 1].y : 0.f);
    }
    __syncwarp();
    cf c[2 * W2];
#pragma unroll
    for (int q = 0; q < W2; ++q) {
      const float4 v = col[q];
      c[2 * q] = cf{v.x, v.y};
      c[2 * q + 1] = cf{v.z, v.w};
    }
    const float m = norm2(c[k]);
    if (!(m > 0.f) || !isfinite(m)) return false;
    const float rr = __frcp_rn(m);
    const cf inv{c[k].x * rr, -c[k].y * rr};
    const bool me = lane == k;
    const cf piv = me ? cf{1.f + inv.x, inv.y} : a[k] * inv;
#pragma unroll
    for (int i = 0; i < W; ++i)
      if (i != k) a[i] = a[i] - c[i] * piv;
    a[k] = me ? inv : piv;
  }
  return true;
}

// Inverse of the W x W slice matrix A held by columns (lane j < W: column j in a).  Slices where
// every site dephases take gj_cols; the others the pivoted row routine applied to A^T (lane j's
// column of A is row j of A^T, and row j of (A^T)^-1 is column j of A^-1).  Lanes >= W must hold
// zeros.  buf: 2 W + 2 complex64 of shared memory, 16-byte aligned.
template <int W>
__device__ bool invert_slice(cf (&a)[W], bool all_dephase, cf* buf) {
  if (all_dephase) return gj_cols<W>(a, buf);
  const int lane = threadIdx.x & 31;
  cf ar[2 * W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    ar[j] = a[j];
    ar[W + j] = cf{(lane < W && lane == j) ? 1.f : 0.f, 0.f};
  }
  if (!gj_rows<W>(ar, true, buf)) return false;
#pragma unroll
  for (int j = 0; j < W; ++j) a[j] = ar[W + j];
  return true;
}

// Column j (lane j < W) of E - H_kk - Sigma_s(k) - x, where x is this lane's column; other lanes
// get zero columns.
template <int W>
__device__ void build_col(cf (&a)[W], double E, double t, double onsite_j, double eta_j,
                          const cf (&x)[W], const double* h = nullptr) {
  const int j = threadIdx.x & 31;
  if (h) {
    // multi-orbital slice block: column j of E - h - diag(onsite) + i eta / 2 - x
#pragma unroll
    for (int i = 0; i < W; ++i) {
      cf v{0.f, 0.f};
      if (j < W)
        v = cf{(float)((i == j ? E - onsite_j : 0.0) - h[i * W + j]),
               i == j ? (float)(0.5 * eta_j) : 0.f} - x[i];
      a[i] = v;
    }
    return;
  }
  const cf diag{(float)(E - onsite_j), (float)(0.5 * eta_j)};
  const float tf = (float)t;
#pragma unroll
  for (int i = 0; i < W; ++i) {
    cf v{0.f, 0.f};
    if (j < W) {
      if (i == j) v = diag;
      if (i - j == 1 || j - i == 1) v.x += tf;
      v = v - x[i];
    }
    a[i] = v;
  }
}

// row (= column, the block is symmetric) j of the lead block Phi diag(sig) Phi^T (lanes j < W)
template <int MAXW>
__device__ void lead_col(const double* phi, const cd* sig, int W, cf (&x)[MAXW]) {
  const int j = threadIdx.x & 31;
#pragma unroll
  for (int i = 0; i < MAXW; ++i) {
    cd acc = mk(0.0, 0.0);
    if (i < W && j < W)
      for (int m = 0; m < W; ++m) acc = acc + (phi[i * W + m] * phi[j * W + m]) * sig[m];
    x[i] = cf{(float)acc.x, (float)acc.y};
  }
}

// One sweep (task d, direction dir) with W == MAXW known at compile time.
template <int MAXW>
__device__ __forceinline__ void sweep_reg_body(const TaskDesc& d, int dir,
                                               const double* __restrict__ wire,
                                               const double* __restrict__ phig,
                                               const cd* __restrict__ sig, cf* gL, cf* gR,
                                               int32_t* err, cf* srow) {
  constexpr int W = MAXW;
  const int L = d.L;
  const int lane = threadIdx.x & 31;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  const float ttf = (float)(d.t * d.t);     // FP32 on the serial path (FP64 is slow here)
  cf x[MAXW], a[MAXW];
  lead_col<MAXW>(phig + d.phi_off, sig + d.lead_off, W, x);   // column j of the lead block
  cf* out = dir == 0 ? gL : gR;
  const int jc = lane < W ? lane : 0;
  // the next slice's onsite energy and dephasing are fetched one step ahead
  int k = dir == 0 ? 0 : L - 1;
  double on_j = onsite[k * W + jc], eta_j = eta[k * W + jc];
  for (int s = 0; s < L - 1; ++s) {
    k = dir == 0 ? s : L - 1 - s;
    const double on_cur = on_j, eta_cur = eta_j;
    if (s + 1 < L - 1) {
      const int kn = dir == 0 ? s + 1 : L - 2 - s;
      on_j = onsite[kn * W + jc];
      eta_j = eta[kn * W + jc];
    }
    build_col<W>(a, d.E, d.t, on_cur, eta_cur, x, slice_block(d, onsite));
    const bool deph = __all_sync(0xffffffffu, lane >= W || eta_cur > 0.0);
    if (!invert_slice<W>(a, deph, srow)) {
      if (lane == 0) atomicOr(err, ERR_SINGULAR);
      return;
    }
    // lane j holds column j of g_k: store it (rows i at i W + j, coalesced over the lanes) and
    // keep t^2 times it as the next slice's column j of x
    cf* dst = out + d.g_off + (uint64_t)k * W * W + jc;
    bool bad = false;
#pragma unroll
    for (int i = 0; i < W; ++i) {
      if (lane < W) {
        dst[(uint64_t)i * W] = a[i];
        bad |= !finite_c(a[i]);
      }
      x[i] = cf{ttf * a[i].x, ttf * a[i].y};
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
  }
}

// Calls Body<W>::run(args...) for the compile-time W equal to w (1 <= w <= 16).
template <template <int> class Body, typename... Args>
__device__ __forceinline__ void by_width(int w, Args&&... args) {
  switch (w) {
    case 1: Body<1>::run(args...); break;
    case 2: Body<2>::run(args...); break;
    case 3: Body<3>::run(args...); break;
    case 4: Body<4>::run(args...); break;
    case 5: Body<5>::run(args...); break;
    case 6: Body<6>::run(args...); break;
    case 7: Body<7>::run(args...); break;
    case 8: Body<8>::run(args...); break;
    case 9: Body<9>::run(args...); break;
    case 10: Body<10>::run(args...); break;
    case 11: Body<11>::run(args...); break;
    case 12: Body<12>::run(args...); break;
    case 13: Body<13>::run(args...); break;
    case 14: Body<14>::run(args...); break;
    case 15: Body<15>::run(args...); break;
    case 16: Body<16>::run(args...); break;
    default: break;
  }
}

template <int W>
struct SweepReg {
  template <typename... A>
  __device__ __forceinline__ static void run(A... a) { sweep_reg_body<W>(a...); }
};

// One warp per (task, direction), tasks of width W <= kSweepRegMaxW.
__global__ void rgf_sweep_reg_kernel(const TaskDesc* __restrict__ tasks, int n_tasks,
                                     const double* __restrict__ wire,
                                     const double* __restrict__ phig, const cd* __restrict__ sig,
                                     cf* gL, cf* gR, int32_t* err) {
  const int job = blockIdx.x;
  if (job >= 2 * n_tasks) return;
  __shared__ __align__(16) cf s_row[34];
  const TaskDesc d = tasks[job >> 1];
  if (d.L < 2) return;
  by_width<SweepReg>(d.W, d, job & 1, wire, phig, sig, gL, gR, err, s_row);
}

// last task whose first job index (`first(t)`) is <= job
template <typename F>
__device__ __forceinline__ int find_task(int n_tasks, uint32_t job, F first) {
  int lo = 0, hi = n_tasks - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first(mid) <= job) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// CTA-wide diagonal blocks (any W <= 64): one CTA of kSweepThreads threads per (task, y); same
// outputs as diag_kernel, with the inversion of cta_gj.
template <typename C>
__host__ __device__ inline size_t diag_cta_bytes(int W) {
  // A, S (lead block, then start block) W x W | pivot row, multipliers W (complex) | phi W x W
  // double | mode weights W double | perm W, flag (int)
  return sizeof(C) * (size_t)(2 * W * W + 2 * W) + sizeof(double) * (size_t)(W * W + W) +
         sizeof(int) * (size_t)(W + 2);
}

template <typename C>
__global__ void __launch_bounds__(kSweepThreads) diag_cta_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs,
    const double* __restrict__ wire, const double* __restrict__ phig, const cd* __restrict__ sig,
    const double* __restrict__ gam, const C* __restrict__ gL, const C* __restrict__ gR,
    C* __restrict__ start, double* __restrict__ rowsum, double* __restrict__ mode_w,
    double* __restrict__ cvals, int32_t* err, int min_W) {
  using R = typename Real<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const uint32_t job = blockIdx.x;
  if (job >= n_jobs) return;
  const int task = find_task(n_tasks, job, [&](int t) { return tasks[t].col_base; });
  const TaskDesc d = tasks[task];
  const int W = d.W, L = d.L, n = d.n, WW = W * W;
  if (W > 64 || W < min_W) return;                // narrower tasks: diag_reg_kernel
  const int tid = threadIdx.x, nth = blockDim.x;
  const int y = (int)(job - d.col_base);
  const bool inj = y >= L;
  const int p = y - L;
  const int m0 = inj ? (p == 0 ? 0 : L - 1) : y;
  C* A = reinterpret_cast<C*>(smem_raw);
  C* S = A + WW;
  C* rowk = S + WW;
  C* fcol = rowk + W;
  double* phi = reinterpret_cast<double*>(fcol + W);
  double* mw_s = phi + WW;
  int* perm = reinterpret_cast<int*>(mw_s + W);
  int* flag = perm + W;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + n;
  const R tt = (R)(d.t * d.t);
  const bool lead_l = m0 == 0, lead_r = m0 == L - 1;
  for (int idx = tid; idx < WW; idx += nth) phi[idx] = phig[d.phi_off + idx];
  __syncthreads();
  if (lead_l || lead_r) {
    const cd* sg = sig + d.lead_off;
    for (int idx = tid; idx < WW; idx += nth) {
      const int a = idx / W, b = idx - a * W;
      cd acc = mk(0.0, 0.0);
      for (int m = 0; m < W; ++m) acc = acc + (phi[a * W + m] * phi[b * W + m]) * sg[m];
      S[idx] = to_c(acc, C{});
    }
  }
  __syncthreads();
  // A = E - H - Sigma_s - (lead block or t^2 g^L_{m-1}) - (lead block or t^2 g^R_{m+1})
  const C* gl = lead_l ? nullptr : gL + d.g_off + (uint64_t)(m0 - 1) * WW;
  const C* gr = lead_r ? nullptr : gR + d.g_off + (uint64_t)(m0 + 1) * WW;
  for (int idx = tid; idx < WW; idx += nth) {
    const int a = idx / W, b = idx - a * W;
    C v = slice_entry<C>(a, b, m0, W, d.E, d.t, onsite, eta, slice_block(d, onsite));
    v = v - (gl ? tt * gl[idx] : S[idx]);
    v = v - (gr ? tt * gr[idx] : S[idx]);
    A[idx] = v;
  }
  const bool deph = __syncthreads_and(tid >= W || eta[m0 * W + tid] > 0.0);
  if (!cta_gj(A, rowk, fcol, perm, flag, W, !deph)) {
    if (tid == 0) atomicOr(err, ERR_SINGULAR);
    return;
  }
  // start block: G_mm, or G_mm Phi for the injection columns
  C* dst = start + d.start_off + (uint64_t)y * WW;
  bool bad = false;
  for (int idx = tid; idx < WW; idx += nth) {
    C v;
    if (!inj) {
      v = A[idx];
    } else {
      const int a = idx / W, b = idx - a * W;
      v = mkc(0.0, 0.0, C{});
      for (int c = 0; c < W; ++c) v = v + (R)phi[c * W + b] * A[a * W + c];
    }
    S[idx] = v;
    dst[idx] = v;
    bad |= !finite_c(v);
  }
  if (__syncthreads_or(bad) && tid == 0) atomicOr(err, ERR_NONFINITE);
  // A per row: site b: -2 Im G_bb;  mode mu: -2 Im (Phi^T G Phi)_{mu mu}
  for (int b = tid; b < W; b += nth) {
    if (!inj) {
      rowsum[d.row_base + m0 * W + b] = -2.0 * (double)S[b * W + b].y;
    } else {
      double im = 0.0;
      for (int a = 0; a < W; ++a) im += phi[a * W + b] * (double)S[a * W + b].y;
      const double Ab = -2.0 * im;
      rowsum[d.row_base + n + p * W + b] = Ab;
      const double mw = gam[d.lead_off + b] * Ab;
      mode_w[d.mode_off + p * W + b] = mw;
      mw_s[b] = mw;
    }
  }
  __syncthreads();
  if (inj && tid == 0) {
    double c = 0.0;
    for (int b = 0; b < W; ++b) c += mw_s[b];      // fixed order
    cvals[task * 2 + p] = c;
    rowsum[d.row_base + d.rows + p] = c;
  }
}

// Register-resident diagonal-block kernel (complex64, W <= MAXW <= 16); same outputs as
// diag_kernel.  Shared memory per warp: G (W x W complex64) and phi (W x W double).
template <int MAXW>
__device__ __forceinline__ void diag_reg_body(const TaskDesc& d, int task, uint32_t job,
                                              const double* __restrict__ wire,
                                              const double* __restrict__ phig,
                                              const cd* __restrict__ sig,
                                              const double* __restrict__ gam,
                                              const cf* __restrict__ gL,
                                              const cf* __restrict__ gR, cf* __restrict__ start,
                                              double* __restrict__ rowsum,
                                              double* __restrict__ mode_w,
                                              double* __restrict__ cvals, int32_t* err, cf* sG,
                                              double* phi, double* s_mw, cf* srow) {
  constexpr int W = MAXW;
  const int lane = threadIdx.x & 31;
  const int L = d.L, n = d.n;
  const int y = (int)(job - d.col_base);
  const bool inj = y >= L;
  const int p = y - L;
  const int m0 = inj ? (p == 0 ? 0 : L - 1) : y;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + n;
  const double tt = d.t * d.t;
  for (int idx = lane; idx < W * W; idx += 32) phi[idx] = phig[d.phi_off + idx];
  // this lane's column of left + right (lead block or t^2 g)
  cf x[MAXW], a[MAXW];
  const bool lead_l = m0 == 0, lead_r = m0 == L - 1;
  if (lead_l || lead_r) {
    lead_col<MAXW>(phig + d.phi_off, sig + d.lead_off, W, x);
    if (lead_l && lead_r) {
#pragma unroll
      for (int i = 0; i < MAXW; ++i) x[i] = 2.f * x[i];
    }
  } else {
#pragma unroll
    for (int i = 0; i < MAXW; ++i) x[i] = cf{0.f, 0.f};
  }
  const int jc = lane < W ? lane : 0;
  const cf* gl = lead_l ? nullptr : gL + d.g_off + (uint64_t)(m0 - 1) * W * W;
  const cf* gr = lead_r ? nullptr : gR + d.g_off + (uint64_t)(m0 + 1) * W * W;
#pragma unroll
  for (int i = 0; i < MAXW; ++i) {
    if (lane < W) {
      if (gl) x[i] = x[i] + (float)tt * gl[i * W + jc];
      if (gr) x[i] = x[i] + (float)tt * gr[i * W + jc];
    }
  }
  const double eta_j = eta[m0 * W + jc];
  build_col<W>(a, d.E, d.t, onsite[m0 * W + jc], eta_j, x, slice_block(d, onsite));
  const bool deph = __all_sync(0xffffffffu, lane >= W || eta_j > 0.0);
  if (!invert_slice<W>(a, deph, srow)) {
    if (lane == 0) atomicOr(err, ERR_SINGULAR);
    return;
  }
  bool bad = false;
#pragma unroll
  for (int i = 0; i < MAXW; ++i) {
    if (lane < W) {
      sG[i * W + lane] = a[i];
      bad |= !finite_c(a[i]);
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) atomicOr(err, ERR_NONFINITE);
  __syncwarp();
  // start block: G_mm, or G_mm Phi for the injection columns
  cf* dst = start + d.start_off + (uint64_t)y * W * W;
  for (int idx = lane; idx < W * W; idx += 32) {
    cf v;
    if (!inj) {
      v = sG[idx];
    } else {
      const int r = idx / W, b = idx % W;
      v = cf{0.f, 0.f};
      for (int c = 0; c < W; ++c) v = v + (float)phi[c * W + b] * sG[r * W + c];
    }
    dst[idx] = v;
  }
  // A per row: site b: -2 Im G_bb;  mode mu: -2 sum_{a,c} phi_mu(a) phi_mu(c) Im G_ac
  for (int b = lane; b < W; b += 32) {
    if (!inj) {
      rowsum[d.row_base + m0 * W + b] = -2.0 * (double)sG[b * W + b].y;
    } else {
      double im = 0.0;
      for (int r = 0; r < W; ++r) {
        double row_im = 0.0;
        for (int c = 0; c < W; ++c) row_im += phi[c * W + b] * (double)sG[r * W + c].y;
        im += phi[r * W + b] * row_im;
      }
      const double A = -2.0 * im;
      rowsum[d.row_base + n + p * W + b] = A;
      const double mw = gam[d.lead_off + b] * A;
      mode_w[d.mode_off + p * W + b] = mw;
      s_mw[b] = mw;
    }
  }
  __syncwarp();
  if (inj && lane == 0) {
    double c = 0.0;
    for (int b = 0; b < W; ++b) c += s_mw[b];            // fixed order
    cvals[task * 2 + p] = c;
    rowsum[d.row_base + d.rows + p] = c;
  }
}

template <int W>
struct DiagReg {
  template <typename... A>
  __device__ __forceinline__ static void run(A... a) { diag_reg_body<W>(a...); }
};

// Register-resident diagonal blocks (complex64, W <= 16), one warp per column job; same outputs
// as diag_kernel.  Shared memory per warp: G (W x W complex64), phi (W x W double), the mode
// weights.
__global__ void diag_reg_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs,
                                const double* __restrict__ wire, const double* __restrict__ phig,
                                const cd* __restrict__ sig, const double* __restrict__ gam,
                                const cf* __restrict__ gL, const cf* __restrict__ gR,
                                cf* __restrict__ start, double* __restrict__ rowsum,
                                double* __restrict__ mode_w, double* __restrict__ cvals,
                                int32_t* err) {
  __shared__ cf s_G[8][16 * 16];
  __shared__ double s_phi[8][16 * 16];
  __shared__ double s_mw[8][16];
  __shared__ __align__(16) cf s_row[8][34];
  const int warp = threadIdx.x >> 5;
  const uint32_t job = blockIdx.x * (blockDim.x >> 5) + warp;
  if (job >= n_jobs) return;
  const int task = find_task(n_tasks, job, [&](int t) { return tasks[t].col_base; });
  const TaskDesc d = tasks[task];
  by_width<DiagReg>(d.W, d, task, job, wire, phig, sig, gam, gL, gR, start, rowsum, mode_w,
                    cvals, err, s_G[warp], s_phi[warp], s_mw[warp], s_row[warp]);
}

template <typename C>
__host__ __device__ inline size_t chain_warp_bytes(int W) {
  // X0, X1, Gb : W x W complex | phi : W x W real | lgam : W real
  return sizeof(C) * (size_t)(3 * W * W) + sizeof(typename Real<C>::T) * (size_t)(W * W + W);
}

// One warp per (task, y, direction): the block column of start slice m0 propagated towards
// slice 0 (direction 0, which also emits the start block) or towards slice L-1 (direction 1),
// each block emitted as Step 6' weights of the column's W rows.
template <typename C>
__global__ void chain_kernel(const TaskDesc* __restrict__ tasks, int n_tasks, uint32_t n_jobs,
                             int max_W, const typename Real<C>::T* __restrict__ eta_all,
                             const typename Real<C>::T* __restrict__ phig,
                             const double* __restrict__ gam, const C* __restrict__ gL,
                             const C* __restrict__ gR, const C* __restrict__ start,
                             typename Real<C>::T* __restrict__ weights, C* __restrict__ green,
                             C* __restrict__ gphi) {
  using R = typename Real<C>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t job = blockIdx.x * (blockDim.x >> 5) + warp;
  if (job >= n_jobs) return;
  const int task = find_task(n_tasks, job, [&](int t) { return 2 * tasks[t].col_base; });
  const TaskDesc d = tasks[task];
  if (d.fused || d.cta_chain) return;            // emitted by the tensor-core / CTA chains
  const int W = d.W, L = d.L, n = d.n, K = d.K;
  const uint32_t local = job - 2 * d.col_base;
  const int y = (int)(local >> 1), dir = (int)(local & 1);
  const bool inj = y >= L;
  const int p = y - L;
  const int m0 = inj ? (p == 0 ? 0 : L - 1) : y;
  if (dir == 1 && m0 == L - 1) return;           // nothing towards slice L-1
  unsigned char* base = smem_raw + (size_t)warp * chain_warp_bytes<C>(max_W);
  C* X0 = reinterpret_cast<C*>(base);
  C* X1 = X0 + W * W;
  C* Gb = X1 + W * W;
  R* phi = reinterpret_cast<R*>(Gb + W * W);
  R* lgam = phi + W * W;
  // eta in the table precision: the FP64 wire array (+ n past onsite) or its FP32 copy
  const R* eta = eta_all + (sizeof(R) == 8 ? d.onsite_off + n : d.onsite_off / 2);
  const R mt = (R)(-d.t);
  for (int idx = lane; idx < W * W; idx += 32) {
    phi[idx] = phig[d.phi_off + idx];
    X0[idx] = start[d.start_off + (uint64_t)y * W * W + idx];
  }
  for (int m = lane; m < W; m += 32) lgam[m] = (R)gam[d.lead_off + m];
  __syncwarp();
  const int row0 = inj ? n + p * W : m0 * W;
  R* wrow = weights + d.wt_off;
  // weights of block k held in X (X[a][b] = G_{(k,a),(m0,b)} or (G Phi)_{(k,a),mu})
  // idx / W without an integer division: (idx + 1/2) / W is at least 1/(2W) away from an
  // integer, far above the float error for idx < W^2 <= 4096
  const float rW = 1.0f / (float)W;
  auto emit = [&](const C* X, int k) {
    for (int idx = lane; idx < W * W; idx += 32) {
      const int b = (int)(((float)idx + 0.5f) * rW), a = idx - b * W;
      wrow[(uint64_t)(row0 + b) * K + k * W + a] = eta[k * W + a] * norm2(X[a * W + b]);
      if (green) {
        // keep G (site columns) or G Phi (injection columns) for the gradient
        if (!inj) green[d.green_off + (uint64_t)(k * W + a) * n + m0 * W + b] = X[a * W + b];
        else gphi[d.gphi_off + (uint64_t)(k * W + a) * 2 * W + p * W + b] = X[a * W + b];
      }
    }
    if (k == 0 || k == L - 1) {
      // lead weight of row b: sum_nu Gamma_nu |(Phi^T X)_{nu b}|^2 = <psi_b|Gamma_lead|psi_b>
      for (int b = lane; b < W; b += 32) {
        R sum = 0;
        for (int nu = 0; nu < W; ++nu) {
          C acc = C{0, 0};
          for (int a = 0; a < W; ++a) acc = acc + phi[a * W + nu] * X[a * W + b];
          sum += lgam[nu] * norm2(acc);
        }
        if (k == 0) wrow[(uint64_t)(row0 + b) * K + n + 0] = sum;
        if (k == L - 1) wrow[(uint64_t)(row0 + b) * K + n + 1] = sum;
      }
    }
  };
  C* cur = X0;
  C* nxt = X1;
  if (dir == 0) emit(cur, m0);
  const int k_end = dir == 0 ? -1 : L;
  const int step = dir == 0 ? -1 : 1;
  const C* gsrc = dir == 0 ? gL : gR;
  // the next block g_k is loaded into registers one step ahead (lane's entries idx = lane + 32 i)
  constexpr int kPre = 4;                        // covers W * W <= 128 entries
  const bool pre = W * W <= 32 * kPre;
  C gpre[kPre];
  auto fetch = [&](int k) {
    const C* gk = gsrc + d.g_off + (uint64_t)k * W * W;
#pragma unroll
    for (int i = 0; i < kPre; ++i) {
      const int idx = lane + 32 * i;
      if (idx < W * W) gpre[i] = gk[idx];
    }
  };
  if (pre && m0 + step != k_end) fetch(m0 + step);
  for (int k = m0 + step; k != k_end; k += step) {
    if (pre) {
#pragma unroll
      for (int i = 0; i < kPre; ++i) {
        const int idx = lane + 32 * i;
        if (idx < W * W) Gb[idx] = gpre[i];
      }
      if (k + step != k_end) fetch(k + step);
    } else {
      const C* gk = gsrc + d.g_off + (uint64_t)k * W * W;
      for (int idx = lane; idx < W * W; idx += 32) Gb[idx] = gk[idx];
    }
    __syncwarp();
    for (int idx = lane; idx < W * W; idx += 32) {
      const int a = (int)(((float)idx + 0.5f) * rW), b = idx - a * W;
      C acc = C{0, 0};
      for (int c = 0; c < W; ++c) acc = acc + Gb[a * W + c] * cur[c * W + b];
      nxt[idx] = mt * acc;
    }
    __syncwarp();
    C* tmp = cur; cur = nxt; nxt = tmp;
    emit(cur, k);
    __syncwarp();
  }
}

int warps_for(size_t per_warp, int max_warps) {
  int w = max_warps;
  while (w > 1 && per_warp * w > 96 * 1024) --w;
  return w;
}

// Most warps per chain CTA that fit the opt-in shared memory (and 16 warps).
template <typename C>
int chain_max(int max_W) {
  const size_t per = chain_warp_bytes<C>(max_W);
  int w = 16;
  while (w > 1 && per * w > 200 * 1024) --w;
  return w;
}

template <typename C>
cudaError_t sweep_impl(const TaskDesc* d_tasks, int n_tasks, int max_W, const double* d_wire,
                       const double* d_phi, const cd* d_sig, C* d_gL, C* d_gR, int32_t* d_err,
                       cudaStream_t s);

template <>
cudaError_t sweep_impl<cf>(const TaskDesc* d_tasks, int n_tasks, int max_W,
                           const double* d_wire, const double* d_phi, const cd* d_sig, cf* d_gL,
                           cf* d_gR, int32_t* d_err, cudaStream_t s);

template <>
cudaError_t sweep_impl<cd>(const TaskDesc* d_tasks, int n_tasks, int max_W,
                           const double* d_wire, const double* d_phi, const cd* d_sig, cd* d_gL,
                           cd* d_gR, int32_t* d_err, cudaStream_t s) {
  // one CTA per sweep: each sweep is a serial chain of W x W inversions, spread one per SM
  const size_t smem = sweep_rows_bytes<cd>(max_W);
  cudaError_t e = cudaFuncSetAttribute(rgf_sweep_rows_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rgf_sweep_rows_kernel<<<2 * n_tasks, kSweepRowsThreads, smem, s>>>(
      d_tasks, n_tasks, d_wire, d_phi, d_sig, d_gL, d_gR, d_err);
  return cudaGetLastError();
}

template <>
cudaError_t sweep_impl<cf>(const TaskDesc* d_tasks, int n_tasks, int max_W,
                           const double* d_wire, const double* d_phi, const cd* d_sig, cf* d_gL,
                           cf* d_gR, int32_t* d_err, cudaStream_t s) {
  // one warp per sweep for the tasks of width <= 32 (it skips wider ones), a CTA per sweep for
  // the rest
  rgf_sweep_reg_kernel<<<2 * n_tasks, 32, 0, s>>>(d_tasks, n_tasks, d_wire, d_phi, d_sig, d_gL,
                                                  d_gR, d_err);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || max_W <= kSweepRegMaxW) return e;
  const size_t smem = sweep_smem_bytes<cf>(max_W);
  e = cudaFuncSetAttribute(rgf_sweep_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)smem);
  if (e != cudaSuccess) return e;
  rgf_sweep_cta_kernel<<<2 * n_tasks, kSweepCtaThreads, smem, s>>>(
      d_tasks, n_tasks, d_wire, d_phi, d_sig, d_gL, d_gR, d_err, kSweepRegMaxW + 1);
  return cudaGetLastError();
}

template <typename C>
cudaError_t columns_impl(const TaskDesc* d_tasks, int n_tasks, uint32_t n_cols, int max_W,
                         const double* d_wire, const typename Real<C>::T* d_eta,
                         const double* d_phi, const typename Real<C>::T* d_phiR, const cd* d_sig,
                         const double* d_gam, const C* d_gL, const C* d_gR, C* d_start,
                         typename Real<C>::T* d_w, double* d_rowsum, double* d_mode_w,
                         double* d_c, int32_t* d_err, C* d_green, C* d_gphi, cudaStream_t s,
                         int chain_warps, int cols_max_W) {
  if (sizeof(C) == sizeof(cf)) {
    // register-resident diagonal blocks for the tasks of width <= 16, 4 warps per block (the
    // kernel skips wider tasks)
    const int warps = 4;
    const unsigned blocks = (n_cols + warps - 1) / warps;
    const cf* gl = reinterpret_cast<const cf*>(d_gL);
    const cf* gr = reinterpret_cast<const cf*>(d_gR);
    cf* st = reinterpret_cast<cf*>(d_start);
    diag_reg_kernel<<<blocks, 32 * warps, 0, s>>>(d_tasks, n_tasks, n_cols, d_wire, d_phi, d_sig,
                                                  d_gam, gl, gr, st, d_rowsum, d_mode_w, d_c,
                                                  d_err);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (sizeof(C) != sizeof(cf) || max_W > 16) {
    const size_t smem = diag_cta_bytes<C>(max_W);
    cudaError_t e = cudaFuncSetAttribute(diag_cta_kernel<C>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    diag_cta_kernel<C><<<n_cols, kSweepThreads, smem, s>>>(
        d_tasks, n_tasks, n_cols, d_wire, d_phi, d_sig, d_gam, d_gL, d_gR, d_start, d_rowsum,
        d_mode_w, d_c, d_err, sizeof(C) == sizeof(cf) ? 17 : 1);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  const uint32_t jobs = 2 * n_cols;
  if (cols_max_W == 0) return cudaSuccess;      // every task's columns come from another kernel
  if (sizeof(C) == sizeof(cf) && cols_max_W <= 32 && d_green == nullptr)
    return launch_chain_cols(d_tasks, n_tasks, jobs, cols_max_W,
                             reinterpret_cast<const float*>(d_eta),
                             reinterpret_cast<const float*>(d_phiR), d_gam,
                             reinterpret_cast<const cf*>(d_gL), reinterpret_cast<const cf*>(d_gR),
                             reinterpret_cast<const cf*>(d_start), reinterpret_cast<float*>(d_w),
                             s);
  const size_t per = chain_warp_bytes<C>(max_W);
  int warps = warps_for(per, 8);
  if (chain_warps > 0) warps = chain_warps < chain_max<C>(max_W) ? chain_warps : chain_max<C>(max_W);
  const size_t smem = per * warps;
  cudaError_t e = cudaFuncSetAttribute(chain_kernel<C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  chain_kernel<C><<<(jobs + warps - 1) / warps, 32 * warps, smem, s>>>(
      d_tasks, n_tasks, jobs, max_W, d_eta, d_phiR, d_gam, d_gL, d_gR, d_start, d_w, d_green,
      d_gphi);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_lead_modes(const TaskDesc* d_tasks, int n_tasks, int max_W,
                              const double* d_wire, double* d_phi, float* d_phi32,
                              float* d_eta32, cd* d_sig, double* d_gam, int32_t* d_err,
                              cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  lead_modes_kernel<<<n_tasks, 128, 0, s>>>(d_tasks, n_tasks, d_wire, d_phi, d_phi32, d_eta32,
                                            d_sig, d_gam, d_err);
  return cudaGetLastError();
}

cudaError_t launch_rgf_sweep(const TaskDesc* d_tasks, int n_tasks, int max_W, int precision,
                             const double* d_wire, const double* d_phi, const cd* d_sig,
                             void* d_gL, void* d_gR, int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  if (precision == NEGF_FP64)
    return sweep_impl<cd>(d_tasks, n_tasks, max_W, d_wire, d_phi, d_sig,
                          static_cast<cd*>(d_gL), static_cast<cd*>(d_gR), d_err, s);
  return sweep_impl<cf>(d_tasks, n_tasks, max_W, d_wire, d_phi, d_sig, static_cast<cf*>(d_gL),
                        static_cast<cf*>(d_gR), d_err, s);
}

cudaError_t launch_block_columns(const TaskDesc* d_tasks, int n_tasks, uint32_t n_cols,
                                 int max_W, int precision, const double* d_wire,
                                 const float* d_eta32, const double* d_phi, const float* d_phi32,
                                 const cd* d_sig, const double* d_gam, const void* d_gL,
                                 const void* d_gR, void* d_start, void* d_weights,
                                 double* d_rowsum, double* d_mode_w, double* d_c, int32_t* d_err,
                                 void* d_green, void* d_gphi, cudaStream_t s, int chain_warps,
                                 int cols_max_W) {
  if (n_tasks == 0 || n_cols == 0) return cudaSuccess;
  if (cols_max_W < 0) cols_max_W = max_W;
  if (precision == NEGF_FP64)
    return columns_impl<cd>(d_tasks, n_tasks, n_cols, max_W, d_wire, d_wire, d_phi, d_phi,
                            d_sig, d_gam, static_cast<const cd*>(d_gL),
                            static_cast<const cd*>(d_gR), static_cast<cd*>(d_start),
                            static_cast<double*>(d_weights), d_rowsum, d_mode_w, d_c, d_err,
                            static_cast<cd*>(d_green), static_cast<cd*>(d_gphi), s,
                            chain_warps, cols_max_W);
  return columns_impl<cf>(d_tasks, n_tasks, n_cols, max_W, d_wire, d_eta32, d_phi, d_phi32,
                          d_sig, d_gam, static_cast<const cf*>(d_gL),
                          static_cast<const cf*>(d_gR), static_cast<cf*>(d_start),
                          static_cast<float*>(d_weights), d_rowsum, d_mode_w, d_c, d_err,
                          static_cast<cf*>(d_green), static_cast<cf*>(d_gphi), s,
                          chain_warps, cols_max_W);
}

int chain_warps_max(int max_W, int precision) {
  return precision == NEGF_FP64 ? chain_max<cd>(max_W) : chain_max<cf>(max_W);
}

}  // namespace negf
