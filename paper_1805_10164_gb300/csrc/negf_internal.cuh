// Internal declarations shared by the CUDA translation units of libnegf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/negf.h"

namespace negf {

// Device error word bits (OR-ed by kernels, read at synchronising calls).
enum : int32_t {
  ERR_NONFINITE = 1,      // a Green's function block or weight is not finite
  ERR_ROWSUM = 2,         // a table row sums to <= 0 where the site is coupled
  ERR_INPUT = 4,          // device-resident input failed validation
  ERR_SINGULAR = 8,       // zero pivot in a block inversion
  ERR_ALIAS = 16          // alias construction inconsistent (no heavy item)
};

// One (wire, energy) task.  Offsets are in elements of the array they index.
struct TaskDesc {
  int32_t wire, e_idx;
  int32_t W, L, n, K, rows, lead_model;
  double E, t, w_E, gamma_lead;
  uint64_t tab_off;      // alias entries [rows][K]
  uint64_t wt_off;       // weights [rows][K] (float or double)
  uint64_t g_off;        // RGF blocks [L][W][W] complex (FP64) for gL and gR
  uint32_t mode_off;     // mode alias / weights [2][W]
  uint32_t lead_off;     // lead eigen self-energies [W] complex and Gamma [W] double
  uint32_t onsite_off;   // into the wire data array: onsite [L*W], eta follows at +n
  uint32_t row_base;     // first global row-job index of this task (alias build)
};

struct cd { double x, y; };
struct cf { float x, y; };

__host__ __device__ inline cd mk(double a, double b) { return cd{a, b}; }
__host__ __device__ inline cd operator+(cd a, cd b) { return cd{a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cd operator-(cd a, cd b) { return cd{a.x - b.x, a.y - b.y}; }
__host__ __device__ inline cd operator*(cd a, cd b) {
  return cd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ inline cd operator*(double s, cd a) { return cd{s * a.x, s * a.y}; }
__host__ __device__ inline cf operator+(cf a, cf b) { return cf{a.x + b.x, a.y + b.y}; }
__host__ __device__ inline cf operator*(cf a, cf b) {
  return cf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
__host__ __device__ inline cf operator*(float s, cf a) { return cf{s * a.x, s * a.y}; }
__host__ __device__ inline double norm2(cd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline float norm2(cf a) { return a.x * a.x + a.y * a.y; }
// complex division a / b by multiplication with conj(b) / |b|^2
__host__ __device__ inline cd cdiv(cd a, cd b) {
  double d = b.x * b.x + b.y * b.y;
  return cd{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// Launchers (each returns the cudaError_t of its launch).
cudaError_t launch_lead_modes(const TaskDesc* d_tasks, int n_tasks, int max_W, cd* d_sig,
                              double* d_gam, int32_t* d_err, cudaStream_t s);
cudaError_t launch_rgf_sweep(const TaskDesc* d_tasks, int n_tasks, int max_W,
                             const double* d_wire, const cd* d_sig, cd* d_gL, cd* d_gR,
                             int32_t* d_err, cudaStream_t s);
cudaError_t launch_block_columns(const TaskDesc* d_tasks, int n_tasks, int max_W, int max_L,
                                 int precision, const double* d_wire, const cd* d_sig,
                                 const double* d_gam, const cd* d_gL, const cd* d_gR,
                                 void* d_weights, double* d_rowsum, double* d_mode_w,
                                 double* d_c, int32_t* d_err, cudaStream_t s);
cudaError_t launch_alias_build(const TaskDesc* d_tasks, int n_tasks, uint32_t total_jobs,
                               int max_K, int precision, const void* d_weights,
                               const double* d_rowsum, const double* d_mode_w,
                               uint64_t* d_tab, uint64_t* d_mode_tab, int32_t* d_err,
                               cudaStream_t s);
// d_tally holds the counters of tasks task0 .. task0 + n_tasks - 1 (index 0 = task0).
cudaError_t launch_walk(const TaskDesc* d_tasks, int task0, int n_tasks, const uint64_t* d_tab,
                        const uint64_t* d_mode_tab, const double* d_c, int start_lead,
                        uint64_t seed, uint64_t walkers_per_task, uint64_t id_offset,
                        uint32_t max_steps, unsigned long long* d_counter, uint64_t* d_tally,
                        int32_t* d_trace_lead, uint32_t* d_trace_steps, int sm_count,
                        cudaStream_t s);
cudaError_t launch_current(const TaskDesc* d_tasks, int n_tasks, int n_wires,
                           const int32_t* d_wire_task0, const double* d_c,
                           const uint64_t* d_tally, int start_lead, double mu_p, double mu_q,
                           double kT, double* d_out, cudaStream_t s);
cudaError_t launch_validate(const TaskDesc* d_tasks, int n_tasks, const double* d_wire,
                            int32_t* d_err, cudaStream_t s);

}  // namespace negf
