// CTA-wide W x W complex inversion (Gauss-Jordan) and the slice matrices of the RGF sweeps,
// shared by the table build and the block-column adjoint of the gradient.
#pragma once

#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

template <typename C> struct Real;
template <> struct Real<cd> { using T = double; };
template <> struct Real<cf> { using T = float; };

__device__ __forceinline__ cd to_c(cd v, cd) { return v; }
__device__ __forceinline__ cf to_c(cd v, cf) { return cf{(float)v.x, (float)v.y}; }
__device__ __forceinline__ cd mkc(double a, double b, cd) { return cd{a, b}; }
__device__ __forceinline__ cf mkc(double a, double b, cf) { return cf{(float)a, (float)b}; }
__device__ __forceinline__ bool finite_c(cd v) { return isfinite(v.x) && isfinite(v.y); }
__device__ __forceinline__ bool finite_c(cf v) { return isfinite(v.x) && isfinite(v.y); }

// The task's multi-orbital slice block h [W][W] (it follows eta in the wire data), or nullptr
// for the square-lattice cross-section.
__device__ __forceinline__ const double* slice_block(const TaskDesc& d, const double* onsite) {
  return d.slice_h ? onsite + 2 * (uint64_t)d.n : nullptr;
}

// E - H_kk - Sigma_s(k) entry (a, b) of slice k, in the precision of C; H_kk = h + diag(onsite)
// for a multi-orbital slice block h, else diag(onsite) with -t between neighbours
template <typename C>
__device__ __forceinline__ C slice_entry(int a, int b, int k, int W, double E, double t,
                                         const double* onsite, const double* eta,
                                         const double* h = nullptr) {
  using R = typename Real<C>::T;
  if (h)
    return mkc((a == b ? E - onsite[k * W + a] : 0.0) - h[a * W + b],
               a == b ? 0.5 * eta[k * W + a] : 0.0, C{});
  C v = mkc(a == b ? E - onsite[k * W + a] : 0.0, a == b ? 0.5 * eta[k * W + a] : 0.0, C{});
  if (a - b == 1 || b - a == 1) v.x += (R)t;
  return v;
}

// In-place inverse of A (W x W, shared memory) by the whole CTA; false (uniformly) on a zero or
// non-finite pivot.
template <typename C>
__device__ bool cta_gj(C* A, C* rowk, C* fcol, int* perm, int* flag, int W, bool pivot) {
  using R = typename Real<C>::T;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int R_ = nth / W;                          // row groups
  const int j = tid % W, rg = tid / W;             // this thread's column and row group
  const bool own = rg < R_;
  for (int k = 0; k < W; ++k) {
    if (pivot) {
      if (tid < 32) {
        R best = -1;
        int bi = k;
        for (int i = k + tid; i < W; i += 32) {
          const R v = norm2(A[i * W + k]);
          if (v > best) { best = v; bi = i; }
        }
        for (int off = 16; off > 0; off >>= 1) {
          const R ov = __shfl_xor_sync(0xffffffffu, best, off);
          const int oi = __shfl_xor_sync(0xffffffffu, bi, off);
          if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
        }
        if (tid == 0) {
          flag[0] = (best > 0 && isfinite(best)) ? bi : -1;
          perm[k] = bi;
        }
      }
      __syncthreads();
      const int p = flag[0];
      if (p < 0) return false;
      if (p != k) {
        for (int c = tid; c < W; c += nth) {
          const C tmp = A[k * W + c];
          A[k * W + c] = A[p * W + c];
          A[p * W + c] = tmp;
        }
      }
      __syncthreads();
    }
    // the pivot row (with 1/a_kk in place of a_kk, formed once) and the pivot column
    for (int c = tid; c < 2 * W; c += nth) {
      if (c < W) rowk[c] = c == k ? cdiv(mkc(1.0, 0.0, C{}), A[k * W + k]) : A[k * W + c];
      else fcol[c - W] = A[(c - W) * W + k];
    }
    __syncthreads();
    const C inv = rowk[k];
    if (!finite_c(inv)) return false;              // every thread reads the same value
    if (own) {
      const C t = j == k ? inv : rowk[j] * inv;    // a_kj / a_kk
      for (int i = rg; i < W; i += R_) {
        C v;
        if (i == k) v = t;
        else if (j == k) v = mkc(0.0, 0.0, C{}) - fcol[i] * inv;
        else v = A[i * W + j] - fcol[i] * t;
        A[i * W + j] = v;
      }
    }
    __syncthreads();
  }
  if (pivot) {
    for (int k = W - 1; k >= 0; --k) {
      const int p = perm[k];
      if (p != k) {
        for (int i = tid; i < W; i += nth) {
          const C tmp = A[i * W + k];
          A[i * W + k] = A[i * W + p];
          A[i * W + p] = tmp;
        }
      }
      __syncthreads();
    }
  }
  return true;
}

}  // namespace
}  // namespace negf
