// Internal declarations shared by the CUDA translation units of libnegf.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/negf.h"

namespace negf {

// Device error word bits (OR-ed by kernels, read at synchronising calls).
enum : int32_t {
  ERR_NONFINITE = 1,      // a Green's function block or weight is not finite
  ERR_ROWSUM = 2,         // a table row sums to <= 0 where the site is coupled
  ERR_INPUT = 4,          // device-resident input failed validation
  ERR_SINGULAR = 8,       // zero pivot in a block inversion
  ERR_TIMEOUT = 16        // a bounded device wait gave up
};

// One (wire, energy) task.  Offsets are in elements of the array they index.
struct TaskDesc {
  int32_t wire, e_idx;
  int32_t W, L, n, K, rows, lead_model;
  double E, t, w_E, gamma_lead;
  uint64_t tab_off;      // alias entries [rows][K]
  uint64_t wt_off;       // weights [rows][K] (float or double)
  uint64_t g_off;        // RGF blocks [L][W][W] complex for gL and gR
  uint32_t mode_off;     // mode alias / weights [2][W]
  uint32_t lead_off;     // lead eigen self-energies [W] complex and Gamma [W] double
  uint32_t onsite_off;   // into the wire data array: onsite [L*W], eta follows at +n
  uint32_t row_base;     // first global row-job index of this task (alias build)
  uint32_t col_base;     // first block-column job of this task (L + 2 per task)
  uint32_t phi_off;      // transverse modes phi[a][m] of this wire's width (W x W)
  uint64_t start_off;    // start blocks [L + 2][W][W] complex
  uint64_t green_off;    // dense G [n][n] (kept for the gradient)
  uint64_t gphi_off;     // G Phi of both leads [n][2W] (kept for the gradient)
  int32_t layout;        // NEGF_LAYOUT_ONE_LEVEL or NEGF_LAYOUT_TWO_LEVEL
  int32_t fused;         // two-level tables emitted by the tensor-core chain (W = 64)
  uint64_t l1_off;       // two-level: level-1 entries [rows][L + 2] (level 2 is at tab_off)
  uint64_t l1w_off;      // two-level: level-1 weights [rows][L + 2] in the weights array
  uint64_t edge_off;     // fused: slice-0 and slice-(L-1) blocks [L + 2][2][W][W] complex64
  int32_t cta_chain;     // block columns by a CTA-wide FP32 kernel (W = 64 or 16 < W <= 32)
  int32_t slice_h;       // multi-orbital slice block: h [W][W] at onsite + 2n, then the
                         // eigenvalues of h [W] (written on the device) at onsite + 2n + W^2
  int32_t l2_fused;      // two-level, W = 64 CTA chain: the chain writes the level-2 blocks and
                         // level-1 weights itself (no rows x K weights are stored)
  int32_t pad_;
};

// u32 words of one level-2 block of a two-level table (slice of W sites): one octet of 31-bit
// cumulative thresholds for W <= 8, else an 8-word guide and ceil(W / 8) octets.
__host__ __device__ inline int level2_words(int W) {
  const int G = (W + 7) >> 3;
  return G == 1 ? 8 : 8 + 8 * G;
}

// One job of the tensor-core chain: block columns y0 and y1 (y1 = -1: none) of task `task`
// (index into the descriptor array of the launch) propagated in direction dir (0: towards
// slice 0 with g^L, which also emits the start slices; 1: towards slice L - 1 with g^R).
struct TcJob {
  int32_t task, dir, y0, y1;
};

// Host side: append the chain jobs of task k (L slices) to `jobs` (every block column in
// direction 0 in pairs, the columns with slices beyond their start in direction 1), and order
// a job list longest chain first (desc: the descriptors the jobs' task indices refer to).
void add_tc_jobs(std::vector<TcJob>& jobs, int k, int L);
// The jobs of the W = 64 CTA-wide chain, which uses G = G^T (see k_chain_cta.cu): every block
// column towards slice 0, and towards slice L - 1 only the injection column of lead L.
void add_sym_jobs(std::vector<TcJob>& jobs, int k, int L);
void sort_jobs_longest_first(std::vector<TcJob>& jobs, const TaskDesc* desc);

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
__host__ __device__ inline cf operator-(cf a, cf b) { return cf{a.x - b.x, a.y - b.y}; }
__host__ __device__ inline double norm2(cd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ inline float norm2(cf a) { return a.x * a.x + a.y * a.y; }
// complex division a / b by multiplication with conj(b) / |b|^2
__host__ __device__ inline cd cdiv(cd a, cd b) {
  double d = b.x * b.x + b.y * b.y;
  return cd{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}
__host__ __device__ inline cf cdiv(cf a, cf b) {
  float d = b.x * b.x + b.y * b.y;
  return cf{(a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d};
}

// Launchers (each returns the cudaError_t of its launch).
// Per wire: transverse modes phi (FP64 and FP32 copies, [W][W] at phi_off) and an FP32 copy of
// eta ([n] at onsite_off / 2); per task: lead eigen self-energies.
// Eigenvectors and eigenvalues of the multi-orbital slice blocks (k_slice.cu): phi (FP64 and
// FP32) and eps after each block in the wire data; before launch_lead_modes.
cudaError_t launch_slice_modes(const TaskDesc* d_tasks, int n_tasks, int max_W, double* d_wire,
                               double* d_phi, float* d_phi32, int32_t* d_err, cudaStream_t s);
cudaError_t launch_lead_modes(const TaskDesc* d_tasks, int n_tasks, int max_W,
                              const double* d_wire, double* d_phi, float* d_phi32,
                              float* d_eta32, cd* d_sig, double* d_gam, int32_t* d_err,
                              cudaStream_t s);
// RGF blocks, start blocks: complex128 [..] for NEGF_FP64, complex64 for NEGF_FP32 (the lead
// self-energies stay FP64 in both).  block_bytes() gives the element size.
inline size_t block_bytes(int precision) { return precision == NEGF_FP64 ? 16 : 8; }
cudaError_t launch_rgf_sweep(const TaskDesc* d_tasks, int n_tasks, int max_W, int precision,
                             const double* d_wire, const double* d_phi, const cd* d_sig,
                             void* d_gL, void* d_gR, int32_t* d_err, cudaStream_t s);
// Diagonal blocks (start blocks, A per row, mode weights, c_p) then the block-column chains
// emitting the weights.  n_cols = sum over tasks of L + 2.  On return rowsum holds A of every
// table row and c_p in the two mode-row slots; the alias build replaces them by the row sums.
// cols_max_W: the largest W among the tasks the warp-per-column chains take (neither fused nor
// cta_chain; -1 = max_W), so that a chain instantiation with nothing to do is not launched.
// Block columns with one column per lane (complex64, W <= 32, no gradient outputs; see
// k_chain_cols.cu): jobs = 2 * sum over tasks of (L + 2).
cudaError_t launch_chain_cols(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs, int max_W,
                              const float* d_eta32, const float* d_phi32, const double* d_gam,
                              const cf* d_gL, const cf* d_gR, const cf* d_start, float* d_w,
                              cudaStream_t s);
cudaError_t launch_block_columns(const TaskDesc* d_tasks, int n_tasks, uint32_t n_cols,
                                 int max_W, int precision, const double* d_wire,
                                 const float* d_eta32, const double* d_phi, const float* d_phi32,
                                 const cd* d_sig, const double* d_gam, const void* d_gL,
                                 const void* d_gR, void* d_start, void* d_weights,
                                 double* d_rowsum, double* d_mode_w, double* d_c, int32_t* d_err,
                                 void* d_green, void* d_gphi, cudaStream_t s,
                                 int chain_warps = 0, int cols_max_W = -1);
// Warps per CTA the chain kernel can use for max_W (shared memory bound), and its default.
int chain_warps_max(int max_W, int precision);
// Inelastic Buttiker probes (Step 7'): per task, its wire's first task t0, number of grid
// energies nE and the offset of its energy rows [n][nE] in the energy table.
struct EnergyDesc {
  uint64_t eoff;
  int32_t nE, t0;
};
// Step 7' energy alias rows of every (task, site): job_base[k] = first job of task k (its n
// sites follow); d_rowsum after the alias build (A_ii of every site row).
cudaError_t launch_energy_tables(const TaskDesc* d_tasks, int n_tasks, const EnergyDesc* d_edesc,
                                 const uint32_t* d_job_base, uint32_t total_jobs, int max_nE,
                                 double sigma, const double* d_rowsum, uint64_t* d_etab,
                                 int32_t* d_err, cudaStream_t s);
// Inelastic walks of every task (injection at the task's energy; Step 6' rows of the walker's
// current energy, Step 7' energy rows after every site), tallied per injection task as the
// elastic walk's tally.
cudaError_t launch_inelastic_walk(const TaskDesc* d_tasks, int n_tasks, const EnergyDesc* d_edesc,
                                  const uint64_t* d_tab, const uint64_t* d_mode_tab,
                                  const double* d_c, const uint64_t* d_etab, int start_lead,
                                  uint64_t seed, uint64_t walkers_per_task, uint64_t id_offset,
                                  uint32_t max_steps, uint64_t* d_tally, int sm_count,
                                  cudaStream_t s);
// Alias tables of every row (and mode row); replaces the A values in rowsum by the FP64 row
// sums after checking them.
cudaError_t launch_alias_build(const TaskDesc* d_tasks, int n_tasks, uint32_t total_jobs,
                               int max_K, int precision, const void* d_weights,
                               double* d_rowsum, const double* d_mode_w, uint64_t* d_tab,
                               uint64_t* d_mode_tab, int32_t* d_err, cudaStream_t s,
                               int warps = 0);
// Tensor-core block columns of fused tasks (W = 64, FP32 blocks as 3xTF32): level-2 alias
// rows and level-1 site weights of every slice, then the level-1 lead weights from the edge
// blocks (scratch [L + 2][2][W][W] complex64 at edge_off).  n_cols = sum over tasks of L + 2.
cudaError_t launch_chain_tc(const TaskDesc* d_tasks, int n_tasks, uint32_t n_cols,
                            const TcJob* d_jobs, uint32_t n_jobs, const float* d_eta32,
                            const float* d_phi32, const double* d_gam, const void* d_gL,
                            const void* d_gR, const void* d_start, void* d_weights,
                            uint64_t* d_tab, void* d_edge, int32_t* d_err, cudaStream_t s);
// CTA-wide FP32 block columns of cta_chain tasks: the Step 6' weights of every row, lead
// weights included, as chain_kernel writes them.  Jobs as for launch_chain_tc: the n_wide jobs
// of W = 64 tasks, then the n_narrow jobs of 16 < W <= 32 tasks.
// d_tab, d_err: the tables and error word, for the tasks with l2_fused (W = 64 two-level),
// whose level-2 blocks and level-1 weights the wide kernel writes itself.
cudaError_t launch_chain_cta(const TaskDesc* d_tasks, const TcJob* d_jobs, uint32_t n_wide,
                             uint32_t n_narrow, const float* d_eta32, const float* d_phi32,
                             const double* d_gam, const void* d_gL, const void* d_gR,
                             const void* d_start, void* d_weights, uint64_t* d_tab,
                             int32_t* d_err, cudaStream_t s);
// Warps per CTA the alias kernel can use for rows of max_K slots (shared memory bound).
int alias_warps_max(int max_K);
// Two-level tasks: from the weights [rows][K] of every table row, the level-1 weights (slice
// totals, then the two lead weights; at l1w_off of the same weights array) and the level-2
// alias rows (one per row and slice, W slots, at tab_off).  One-level tasks are skipped.
// n_jobs = sum over tasks of rows + 2 (the row_base numbering).
// max_W: the widest slice among the launch's tasks (sizes the FP32 kernel's registers).
cudaError_t launch_two_level_split(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs,
                                   int precision, void* d_weights, uint64_t* d_tab,
                                   int32_t* d_err, cudaStream_t s, int max_W);
// Walks of tasks d_tasks[task0 .. task0 + n_tasks); d_c is indexed like d_tasks, d_tally holds
// the counters of those tasks (index 0 = task0).  The Philox task number of d_tasks[k] is
// id_base + k.  max_blocks_per_sm > 0 caps the persistent grid (leaving room for concurrent
// kernels).  With d_score non-null every absorbed walk also adds its transitions to
// d_score[lead][tab_off + a K + b] and its injection mode to d_mode_score[lead][mode_off + m]:
// d_mode_score holds kModeReplicas zeroed copies [replica][lead][mode_stride] (every walker of a
// task adds to the same W counters; each block adds to copy blockIdx % kModeReplicas), summed
// into copy 0 before the call returns.
// With d_run non-null the seed and id_offset arguments are ignored and read on the device from
// d_run[0] (seed) and d_run[1] (walker id offset), so a captured graph can be relaunched with
// new values.  two_level: some task of the launch has two-level tables (false: every task is
// one-level, and the launch takes a kernel compiled without the two-level draw).
constexpr int kModeReplicas = 64;
cudaError_t launch_walk(const TaskDesc* d_tasks, int task0, int n_tasks, uint32_t id_base,
                        const uint64_t* d_tab, const uint64_t* d_mode_tab, const double* d_c,
                        int start_lead, uint64_t seed, uint64_t walkers_per_task,
                        uint64_t id_offset, uint32_t max_steps, unsigned long long* d_counter,
                        uint64_t* d_tally, int32_t* d_trace_lead, uint32_t* d_trace_steps,
                        uint64_t* d_score, uint64_t score_stride, uint64_t* d_mode_score,
                        uint32_t mode_stride, int sm_count, int max_blocks_per_sm,
                        cudaStream_t s, const uint64_t* d_run = nullptr, int slots = 1,
                        bool two_level = true);
// Timed random 8-byte gathers over a table of table_bytes (see k_walk.cu); synchronises s.
cudaError_t probe_gather(uint64_t table_bytes, int ilp, int chain, int sm_count,
                         uint64_t* gathers, float* ms, cudaStream_t s);
cudaError_t launch_current(const TaskDesc* d_tasks, int n_tasks, int n_wires,
                           const int32_t* d_wire_task0, const double* d_c,
                           const uint64_t* d_tally, int start_lead, double mu_p, double mu_q,
                           double kT, double* d_out, cudaStream_t s);
// Thermal-window walks over the interpolated chain of one wire's energy grid (k_thermal.cu):
// tasks task0 .. task0 + M - 1 (ascending energies; all one-level, or all two-level with
// two_level set); d_thr [M - 1]: the
// least 53-bit energy word v whose CDF value reaches grid point e + 1 (non-decreasing); tally
// [3 (M - 1) + 5] u64: per interval (absorbed at q, sum a, sum (a >> 16)^2), then absorbed L,
// R, closed, truncated, steps.  Trace arrays optional (nullptr).
cudaError_t launch_thermal_walk(const TaskDesc* d_tasks, int task0, int M, int wire,
                                const uint64_t* d_tab, const uint64_t* d_mode_tab,
                                const double* d_c, int start_lead, uint64_t seed,
                                uint64_t walkers, uint64_t id_offset, uint32_t max_steps,
                                double mu, double kT, double F0, double window,
                                const unsigned long long* d_thr, unsigned long long* d_tally,
                                int32_t* d_lead, uint32_t* d_steps, int32_t* d_interval,
                                uint32_t* d_a, int sm_count, cudaStream_t s,
                                bool two_level = false);
// Distances between the Step 6' probabilities of consecutive grid energies task0 .. task0 + M - 1
// of one wire (k_thermal.cu): d_out[e] for energies e, e + 1 (M - 1 doubles); rows = the tasks'
// table rows; needs the FP weights.
cudaError_t launch_interval_distance(const TaskDesc* d_tasks, int task0, int M, int rows,
                                     int precision, const void* d_weights,
                                     const double* d_rowsum, const double* d_mode_w,
                                     const double* d_c, int start_lead, double* d_out,
                                     cudaStream_t s);
// Backward (score-function gradient, see k_backward.cu).
cudaError_t launch_backward_seeds(const TaskDesc* d_tasks, int n_tasks, uint32_t n_jobs,
                                  int precision, const void* d_weights, const double* d_rowsum,
                                  const double* d_mode_w, const double* d_c,
                                  const uint64_t* d_counts, const uint64_t* d_score,
                                  uint64_t stride, const uint64_t* d_mode_score,
                                  uint32_t mode_stride, int start_lead, void* d_wbar,
                                  int wbar_fp32, double* d_ubar, cudaStream_t s);
cudaError_t launch_backward_task(const TaskDesc& d, int precision, const void* G,
                                 const void* gphi, const double* wbar, const double* ubar,
                                 const double* eta, const double* phi, const double* gam,
                                 int start_lead, void* Gbar, void* Y, double* dV, double* dE,
                                 int sm_count, int32_t* d_err, cudaStream_t s);
// Y = A B for dense complex64 n x n matrices (row-major) on the tensor cores, 3xTF32 with FP32
// accumulation (k_cgemm_tc.cu); a timed-out device wait sets ERR_TIMEOUT in err.
cudaError_t launch_cgemm_tc(const cf* A, const cf* B, cf* Y, int n, int32_t* err,
                            cudaStream_t s);
// Block-column adjoint (k_adjoint.cu): checkpointed sweeps of every task, the recompute of the
// blocks between checkpoints for a group of tasks of one wire, and the column jobs of the group.
size_t adjoint_column_smem(int W, int precision);
int adjoint_cols_per_job(int W);                 // block columns side by side in one job
int adjoint_column_occupancy(int W, int precision);   // column-kernel CTAs one SM holds
cudaError_t launch_adjoint_sweep(const TaskDesc* d_tasks, int n_tasks, int max_W, int precision,
                                 const double* d_wire, const double* d_phi, const cd* d_sig,
                                 const uint64_t* d_ck_off, int stride, void* d_ck,
                                 int32_t* d_err, cudaStream_t s);
cudaError_t launch_adjoint_expand(const TaskDesc* d_tasks, int task0, int n_group, int W, int L,
                                  int precision, const double* d_wire, const double* d_phi,
                                  const cd* d_sig, const uint64_t* d_ck_off, int stride,
                                  const void* d_ck, void* d_gl, void* d_gr, int32_t* d_err,
                                  cudaStream_t s);
cudaError_t launch_adjoint_columns(const TaskDesc* d_tasks, int task0, int n_group, int W,
                                   int precision, int start_lead, const double* d_wire,
                                   const double* d_phi, const cd* d_sig, const double* d_gam,
                                   const void* d_wbar, const double* d_ubar, uint64_t site_off0,
                                   double* d_dV, double* d_dE, const void* d_gl, const void* d_gr,
                                   void* d_psi, void* d_tl, void* d_xs, void* d_ys, int slots,
                                   int32_t* d_err, cudaStream_t s);
cudaError_t launch_grad_sum(const TaskDesc* d_tasks, int n_wires, const int32_t* d_wire_task0,
                            const uint64_t* d_task_site_off, const uint64_t* d_wire_site_off,
                            const double* dT_V, const double* dT_E, const double* d_seed,
                            double mu_p, double mu_q, double kT, double* out_V, double* out_E,
                            cudaStream_t s);
cudaError_t launch_validate(const TaskDesc* d_tasks, int n_tasks, const double* d_wire,
                            int32_t* d_err, cudaStream_t s);

}  // namespace negf
