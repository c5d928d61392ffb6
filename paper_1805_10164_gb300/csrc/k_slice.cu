// Modes of a multi-orbital slice block (the exact strip lead of a wire with a slice block h).
//
// The lead of such a wire is the clean strip of h with the orbital-diagonal coupling -t between
// slices; it separates into the eigenvectors phi_m of h, each a chain with onsite eps_m (the
// eigenvalue) and hopping -t, whose surface self-energy is t^2 g_s(E - eps_m) (the lead
// self-energies of Sec. II.A for this lead).  slice_modes_kernel diagonalises h once per wire:
// cyclic Jacobi rotations in FP64 (Jacobi's method; the rotation angle of the 2 x 2 symmetric
// Schur decomposition, t = sign(theta) / (|theta| + sqrt(theta^2 + 1)),
// theta = (a_qq - a_pp) / (2 a_pq)), the W (W - 1) / 2 index pairs of a sweep visited in W - 1
// rounds of disjoint pairs (round-robin order), so that one round's rotations commute and are
// applied together: rows, then columns, then the accumulated eigenvectors.  Sweeps stop when
// the off-diagonal sum of squares falls below 1e-30 of the matrix's; the eigenpairs are written
// in ascending order of eigenvalue (phi [a][m] in FP64 and FP32, eps after h in the wire data).
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

constexpr int kJacobiThreads = 256;
constexpr int kJacobiMaxSweeps = 40;

__global__ void __launch_bounds__(kJacobiThreads) slice_modes_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, double* __restrict__ wire,
    double* __restrict__ phi, float* __restrict__ phi32, int32_t* __restrict__ err) {
  extern __shared__ __align__(16) double jac_smem[];
  const TaskDesc d = tasks[blockIdx.x];
  if (!d.slice_h || d.e_idx != 0) return;            // once per wire
  const int W = d.W, WW = W * W, Wp = W + (W & 1), np = Wp / 2;
  const int tid = threadIdx.x;
  double* A = jac_smem;
  double* V = A + WW;
  double* cs = V + WW;                                // (c, s) per pair
  double* red = cs + 2 * np;                          // 2 * blockDim partial sums
  int* pq = reinterpret_cast<int*>(red + 2 * blockDim.x);   // (p, q) per pair
  int* perm = pq + 2 * np;
  const double* h = wire + d.onsite_off + 2 * (uint64_t)d.n;
  double* eps = wire + d.onsite_off + 2 * (uint64_t)d.n + WW;
  for (int i = tid; i < WW; i += blockDim.x) {
    A[i] = h[i];
    V[i] = (i / W == i % W) ? 1.0 : 0.0;
  }
  __syncthreads();
  bool converged = false;
  for (int sweep = 0; sweep < kJacobiMaxSweeps; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = tid; i < WW; i += blockDim.x) {
      const double v = A[i] * A[i];
      tot += v;
      if (i / W != i % W) off += v;
    }
    red[tid] = off;
    red[blockDim.x + tid] = tot;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
      if (tid < k) {
        red[tid] += red[tid + k];
        red[blockDim.x + tid] += red[blockDim.x + tid + k];
      }
      __syncthreads();
    }
    off = red[0];
    tot = red[blockDim.x];
    __syncthreads();
    if (!(off > 1e-30 * tot)) {                       // (also ends on a zero matrix)
      converged = isfinite(tot);
      break;
    }
    for (int r = 0; r < Wp - 1; ++r) {
      if (tid < np) {
        int p, q;
        if (tid == 0) {
          p = r;
          q = Wp - 1;
        } else {
          p = (r + tid) % (Wp - 1);
          q = (r - tid + Wp - 1) % (Wp - 1);
        }
        if (p > q) { const int x = p; p = q; q = x; }
        double c = 1.0, s = 0.0;
        if (q < W) {
          const double apq = A[p * W + q];
          if (apq != 0.0) {
            const double theta = (A[q * W + q] - A[p * W + p]) / (2.0 * apq);
            const double t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
          }
        } else {
          p = q = -1;                                 // the padding index of an odd W
        }
        pq[2 * tid] = p;
        pq[2 * tid + 1] = q;
        cs[2 * tid] = c;
        cs[2 * tid + 1] = s;
      }
      __syncthreads();
      // rows p, q of every pair: A <- J^T A
      for (int idx = tid; idx < np * W; idx += blockDim.x) {
        const int k = idx / W, j = idx - k * W;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        if (p < 0) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double ap = A[p * W + j], aq = A[q * W + j];
        A[p * W + j] = c * ap - s * aq;
        A[q * W + j] = s * ap + c * aq;
      }
      __syncthreads();
      // columns p, q: A <- A J, V <- V J
      for (int idx = tid; idx < np * W; idx += blockDim.x) {
        const int k = idx / W, i = idx - k * W;
        const int p = pq[2 * k], q = pq[2 * k + 1];
        if (p < 0) continue;
        const double c = cs[2 * k], s = cs[2 * k + 1];
        const double ap = A[i * W + p], aq = A[i * W + q];
        A[i * W + p] = c * ap - s * aq;
        A[i * W + q] = s * ap + c * aq;
        const double vp = V[i * W + p], vq = V[i * W + q];
        V[i * W + p] = c * vp - s * vq;
        V[i * W + q] = s * vp + c * vq;
      }
      __syncthreads();
    }
  }
  if (!converged) {
    if (tid == 0) atomicOr(err, ERR_NONFINITE);
    return;
  }
  // ascending order of the eigenvalues (one thread: W <= 64)
  if (tid == 0) {
    for (int m = 0; m < W; ++m) perm[m] = m;
    for (int m = 1; m < W; ++m) {
      const int x = perm[m];
      const double v = A[x * W + x];
      int j = m - 1;
      while (j >= 0 && A[perm[j] * W + perm[j]] > v) {
        perm[j + 1] = perm[j];
        --j;
      }
      perm[j + 1] = x;
    }
  }
  __syncthreads();
  for (int idx = tid; idx < WW; idx += blockDim.x) {
    const int a = idx / W, m = idx - a * W;
    const double v = V[a * W + perm[m]];
    phi[d.phi_off + idx] = v;
    phi32[d.phi_off + idx] = (float)v;
  }
  for (int m = tid; m < W; m += blockDim.x) eps[m] = A[perm[m] * W + perm[m]];
}

size_t jacobi_smem(int W) {
  const int np = (W + (W & 1)) / 2;
  return sizeof(double) * (2 * (size_t)W * W + 2 * np + 2 * kJacobiThreads) +
         sizeof(int) * (2 * (size_t)np + W);
}

}  // namespace

cudaError_t launch_slice_modes(const TaskDesc* d_tasks, int n_tasks, int max_W, double* d_wire,
                               double* d_phi, float* d_phi32, int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  const size_t smem = jacobi_smem(max_W);
  cudaError_t e = cudaFuncSetAttribute(slice_modes_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  slice_modes_kernel<<<n_tasks, kJacobiThreads, smem, s>>>(d_tasks, n_tasks, d_wire, d_phi,
                                                           d_phi32, d_err);
  return cudaGetLastError();
}

}  // namespace negf
