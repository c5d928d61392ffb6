// Current assembly from walk tallies (Eq. iqof_t_el_db with the Monte Carlo estimator of
// Eq. elast_lin_xpq and the binomial standard error of Sec. IV.B.2), and the device-side input
// check used when the wire arrays live on the device.
#include <cuda_runtime.h>
#include <math.h>

#include "negf_internal.cuh"

namespace negf {
namespace {

__device__ __forceinline__ double fermi(double E, double mu, double kT) {
  return 0.5 * (1.0 - tanh(0.5 * (E - mu) / kT));   // 1 / (1 + exp((E - mu) / kT))
}

// out layout: I[n_wires] | se[n_wires] | T[n_tasks] | T_se[n_tasks] | truncated (as double)
// One block per wire; its energies are summed in a fixed order (thread-strided partial sums,
// then a shared-memory tree), so the result does not depend on timing.
constexpr int kCurThreads = 128;

__global__ void __launch_bounds__(kCurThreads) current_kernel(
    const TaskDesc* __restrict__ tasks, int n_tasks, int n_wires,
    const int32_t* __restrict__ wire_task0, const double* __restrict__ cvals,
    const unsigned long long* __restrict__ tally, int p, double mu_p, double mu_q, double kT,
    double* __restrict__ out) {
  __shared__ double s_acc[kCurThreads], s_var[kCurThreads], s_tr[kCurThreads];
  const int q = 1 - p;
  double* I = out;
  double* se = out + n_wires;
  double* T = se + n_wires;
  double* Tse = T + n_tasks;
  double* trunc = Tse + n_tasks;
  const int w = blockIdx.x;
  double acc = 0.0, var = 0.0, tr = 0.0;
  for (int k = wire_task0[w] + threadIdx.x; k < wire_task0[w + 1]; k += blockDim.x) {
    const TaskDesc& d = tasks[k];
    const unsigned long long* c = tally + (size_t)k * NEGF_TALLY_FIELDS;
    const double N = (double)c[0];
    const double nq = (double)c[1 + q];
    const double cp = cvals[2 * k + p];
    double Tk = 0.0, sk = 0.0;
    if (N > 0.0) {
      const double P = nq / N;
      Tk = cp * P;
      sk = cp * sqrt(P * (1.0 - P) / N);
    }
    T[k] = Tk;
    Tse[k] = sk;
    const double wd = d.w_E * (fermi(d.E, mu_p, kT) - fermi(d.E, mu_q, kT));
    acc += wd * Tk;
    var += wd * wd * sk * sk;
    tr += (double)c[3];
  }
  s_acc[threadIdx.x] = acc;
  s_var[threadIdx.x] = var;
  s_tr[threadIdx.x] = tr;
  __syncthreads();
  for (int h = kCurThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      s_acc[threadIdx.x] += s_acc[threadIdx.x + h];
      s_var[threadIdx.x] += s_var[threadIdx.x + h];
      s_tr[threadIdx.x] += s_tr[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    I[w] = s_acc[0];
    se[w] = sqrt(s_var[0]);
    if (s_tr[0] > 0.0) atomicAdd(trunc, s_tr[0]);
  }
}

__global__ void validate_kernel(const TaskDesc* __restrict__ tasks, int n_tasks,
                                const double* __restrict__ wire, int32_t* err) {
  const TaskDesc d = tasks[blockIdx.x];
  // only the first task of each wire checks that wire's arrays
  if (d.e_idx != 0) return;
  const double* onsite = wire + d.onsite_off;
  const double* eta = onsite + d.n;
  bool bad = false;
  for (int i = threadIdx.x; i < d.n; i += blockDim.x)
    bad |= !isfinite(onsite[i]) || !isfinite(eta[i]) || !(eta[i] >= 0.0);
  if (d.slice_h) {
    // a multi-orbital slice block must be finite and exactly symmetric
    const double* h = eta + d.n;
    for (int i = threadIdx.x; i < d.W * d.W; i += blockDim.x) {
      const int a = i / d.W, b = i - a * d.W;
      bad |= !isfinite(h[i]) || h[i] != h[b * d.W + a];
    }
  }
  if (bad) atomicOr(err, ERR_INPUT);
  if (threadIdx.x == 0 && !(isfinite(d.E) && isfinite(d.w_E))) atomicOr(err, ERR_INPUT);
}

__global__ void validate_energy_kernel(const TaskDesc* __restrict__ tasks, int n_tasks,
                                       int32_t* err) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_tasks && !(isfinite(tasks[k].E) && isfinite(tasks[k].w_E))) atomicOr(err, ERR_INPUT);
}

}  // namespace

cudaError_t launch_current(const TaskDesc* d_tasks, int n_tasks, int n_wires,
                           const int32_t* d_wire_task0, const double* d_c,
                           const uint64_t* d_tally, int start_lead, double mu_p, double mu_q,
                           double kT, double* d_out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(d_out + 2 * (size_t)n_wires + 2 * (size_t)n_tasks, 0,
                                  sizeof(double), s);
  if (e != cudaSuccess) return e;
  if (n_wires == 0) return cudaSuccess;
  current_kernel<<<n_wires, kCurThreads, 0, s>>>(
      d_tasks, n_tasks, n_wires, d_wire_task0, d_c,
      reinterpret_cast<const unsigned long long*>(d_tally), start_lead, mu_p, mu_q, kT, d_out);
  return cudaGetLastError();
}

cudaError_t launch_validate(const TaskDesc* d_tasks, int n_tasks, const double* d_wire,
                            int32_t* d_err, cudaStream_t s) {
  if (n_tasks == 0) return cudaSuccess;
  validate_kernel<<<n_tasks, 128, 0, s>>>(d_tasks, n_tasks, d_wire, d_err);
  validate_energy_kernel<<<(n_tasks + 127) / 128, 128, 0, s>>>(d_tasks, n_tasks, d_err);
  return cudaGetLastError();
}

}  // namespace negf
