// negf_build_tables_noalloc: the table build for callers that cannot allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: code running inside a host framework
// that owns all device memory through its own pool (and forbids foreign allocations), or a
// process that must not grow its device footprint after start-up, or a caller that enqueues
// work from a context where an allocation would synchronise the device.  For them this entry
// point runs the kernels negf_build_tables runs for the same wire and precision (one-level
// tables) but takes every scratch buffer from one file-scope device array of fixed size, and
// writes the tables into buffers the caller passes.
// The array exists once per device that loads the library and stays allocated until the
// process exits.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "negf_internal.cuh"

namespace {

constexpr size_t kScratchBytes = NEGF_NOALLOC_SCRATCH_BYTES;

// The scratch array.  In host code its name is only a stand-in for the symbol, not a device
// address: kernels must be given the address returned by cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

bool band_edge(double E, int W, double t) {
  for (int m = 1; m <= W; ++m) {
    const double eps = -2.0 * t * cos(m * M_PI / (W + 1));
    if (fabs(fabs(E - eps) - 2.0 * t) <= 1e-12 * t) return true;
  }
  return false;
}

}  // namespace

extern "C" negf_status negf_build_tables_noalloc(const negf_wire* wire, int32_t precision,
                                                 void* stream, uint64_t* d_alias,
                                                 uint64_t* d_mode_alias, double* d_c) {
  using negf::cd;
  using negf::TaskDesc;
  if (!wire || !d_alias || !d_mode_alias || !d_c) return NEGF_E_INVALID;
  if (precision != NEGF_FP64 && precision != NEGF_FP32 && precision != NEGF_SPLIT_TF32)
    return NEGF_E_INVALID;
  const int prec = precision == NEGF_FP64 ? NEGF_FP64 : NEGF_FP32;
  const negf_wire& wr = *wire;
  if (wr.W < 1 || wr.W > NEGF_MAX_W || wr.L < 1 || !(wr.t > 0.0) || !isfinite(wr.t) ||
      wr.n_energy < 1 || wr.n_energy > NEGF_NOALLOC_MAX_TASKS || !wr.onsite || !wr.eta ||
      !wr.energy)
    return NEGF_E_INVALID;
  if (wr.lead_model != NEGF_LEAD_STRIP && wr.lead_model != NEGF_LEAD_WIDE_BAND) return NEGF_E_INVALID;
  if (wr.lead_model == NEGF_LEAD_WIDE_BAND && !(wr.gamma_lead > 0.0 && isfinite(wr.gamma_lead)))
    return NEGF_E_INVALID;
  const int64_t n = (int64_t)wr.W * wr.L, K = n + 2, rows = n + 2 * wr.W;
  if (n > NEGF_MAX_SITES) return NEGF_E_INVALID;
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(wr.onsite[i]) || !isfinite(wr.eta[i]) || !(wr.eta[i] >= 0.0)) return NEGF_E_INVALID;
  if (wr.slice_h)
    for (int a = 0; a < wr.W; ++a)
      for (int b = 0; b < wr.W; ++b)
        if (!isfinite(wr.slice_h[a * wr.W + b]) ||
            wr.slice_h[a * wr.W + b] != wr.slice_h[b * wr.W + a])
          return NEGF_E_INVALID;
  const int64_t hw = wr.slice_h ? (int64_t)wr.W * (wr.W + 1) : 0;   // block, then eigenvalues
  const int nt = wr.n_energy;
  for (int k = 0; k < nt; ++k) {
    if (!isfinite(wr.energy[k])) return NEGF_E_INVALID;
    if (wr.lead_model == NEGF_LEAD_STRIP && !wr.slice_h && band_edge(wr.energy[k], wr.W, wr.t))
      return NEGF_E_INVALID;
  }
  // block columns as negf_build_tables takes them: FP32 wires of W = 64 or 16 < W <= 32 on the
  // CTA-wide chains (jobs listed here), every other wire on the warp-per-column chains
  const bool cta = prec == NEGF_FP32 && (wr.W == 64 || (wr.W > 16 && wr.W <= 32));

  // ---- carve the scratch array; reject problems that do not fit
  const size_t wsz = prec == NEGF_FP64 ? sizeof(double) : sizeof(float);
  const size_t per_task_tab = (size_t)rows * K;
  size_t off = 0;
  const size_t o_tasks = off;  off += align256(sizeof(TaskDesc) * nt);
  const size_t o_wire = off;   off += align256(sizeof(double) * (2 * n + hw));
  const size_t o_sig = off;    off += align256(sizeof(cd) * nt * wr.W);
  const size_t o_gam = off;    off += align256(sizeof(double) * nt * wr.W);
  const size_t cb = negf::block_bytes(prec);      // bytes per complex block element
  const size_t o_gL = off;     off += align256(cb * nt * (size_t)wr.L * wr.W * wr.W);
  const size_t o_gR = off;     off += align256(cb * nt * (size_t)wr.L * wr.W * wr.W);
  const size_t o_st = off;     off += align256(cb * nt * (size_t)(wr.L + 2) * wr.W * wr.W);
  const size_t o_phi = off;    off += align256(sizeof(double) * wr.W * wr.W);
  const size_t o_phi32 = off;  off += align256(sizeof(float) * wr.W * wr.W);
  const size_t o_eta32 = off;  off += align256(sizeof(float) * n);
  const size_t o_w = off;      off += align256(wsz * nt * per_task_tab);
  const size_t o_rs = off;     off += align256(sizeof(double) * nt * (rows + 2));
  const size_t o_mw = off;     off += align256(sizeof(double) * nt * 2 * wr.W);
  const size_t o_err = off;    off += align256(sizeof(int32_t));
  // CTA-chain jobs: at most L + 2 per task (pairs of the L + 2 block columns in direction 0,
  // pairs of at most L of them in direction 1)
  const size_t o_jobs = off;   off += cta ? align256(sizeof(negf::TcJob) * nt * (size_t)(wr.L + 2)) : 0;
  if (off > kScratchBytes) return NEGF_E_NOMEM;   // the problem needs more than the fixed scratch

  // The array's device address on the current device, looked up on every call (a host-side
  // lookup; it stays right if the device's context was reset and the module reloaded).
  void* scratch = nullptr;
  if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch)
    return NEGF_E_CUDA;
  unsigned char* base = static_cast<unsigned char*>(scratch);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  TaskDesc h_tasks[NEGF_NOALLOC_MAX_TASKS];
  memset(h_tasks, 0, sizeof(TaskDesc) * nt);
  for (int k = 0; k < nt; ++k) {
    TaskDesc& d = h_tasks[k];
    d.wire = 0;
    d.e_idx = k;
    d.layout = NEGF_LAYOUT_ONE_LEVEL;
    d.W = wr.W;
    d.L = wr.L;
    d.n = (int)n;
    d.K = (int)K;
    d.rows = (int)rows;
    d.lead_model = wr.lead_model;
    d.E = wr.energy[k];
    d.t = wr.t;
    d.w_E = 1.0;                 // quadrature weights play no part in the tables
    d.cta_chain = cta ? 1 : 0;
    d.slice_h = wr.slice_h ? 1 : 0;
    d.gamma_lead = wr.gamma_lead;
    d.tab_off = (uint64_t)k * per_task_tab;
    d.wt_off = d.tab_off;
    d.g_off = (uint64_t)k * wr.L * wr.W * wr.W;
    d.mode_off = (uint32_t)(2 * wr.W * k);
    d.lead_off = (uint32_t)(wr.W * k);
    d.onsite_off = 0;
    d.row_base = (uint32_t)(k * (rows + 2));
    d.col_base = (uint32_t)(k * (wr.L + 2));
    d.phi_off = 0;
    d.start_off = (uint64_t)k * (wr.L + 2) * wr.W * wr.W;
  }
  TaskDesc* d_tasks = reinterpret_cast<TaskDesc*>(base + o_tasks);
  double* d_wire = reinterpret_cast<double*>(base + o_wire);
  cd* d_sig = reinterpret_cast<cd*>(base + o_sig);
  double* d_gam = reinterpret_cast<double*>(base + o_gam);
  void* d_gL = base + o_gL;
  void* d_gR = base + o_gR;
  void* d_st = base + o_st;
  double* d_phi = reinterpret_cast<double*>(base + o_phi);
  float* d_phi32 = reinterpret_cast<float*>(base + o_phi32);
  float* d_eta32 = reinterpret_cast<float*>(base + o_eta32);
  void* d_w = base + o_w;
  double* d_rs = reinterpret_cast<double*>(base + o_rs);
  double* d_mw = reinterpret_cast<double*>(base + o_mw);
  int32_t* d_err = reinterpret_cast<int32_t*>(base + o_err);
  negf::TcJob* d_jobs = reinterpret_cast<negf::TcJob*>(base + o_jobs);
  std::vector<negf::TcJob> jobs;                     // host memory only
  if (cta) {
    for (int k = 0; k < nt; ++k) {
      if (wr.W == 64) negf::add_sym_jobs(jobs, k, wr.L);
      else negf::add_tc_jobs(jobs, k, wr.L);
    }
    negf::sort_jobs_longest_first(jobs, h_tasks);
  }

  // the array keeps the previous call's contents: the error word must start at zero (every
  // other scratch value is written before it is read)
  cudaError_t e = cudaMemsetAsync(d_err, 0, sizeof(int32_t), s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tasks, h_tasks, sizeof(TaskDesc) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !jobs.empty())
    e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(negf::TcJob) * jobs.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_wire, wr.onsite, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_wire + n, wr.eta, sizeof(double) * n, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && wr.slice_h)
    e = cudaMemcpyAsync(d_wire + 2 * n, wr.slice_h, sizeof(double) * wr.W * wr.W,
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && wr.slice_h)
    e = negf::launch_slice_modes(d_tasks, nt, wr.W, d_wire, d_phi, d_phi32, d_err, s);
  if (e == cudaSuccess)
    e = negf::launch_lead_modes(d_tasks, nt, wr.W, d_wire, d_phi, d_phi32, d_eta32, d_sig, d_gam,
                                d_err, s);
  if (e == cudaSuccess)
    e = negf::launch_rgf_sweep(d_tasks, nt, wr.W, prec, d_wire, d_phi, d_sig, d_gL, d_gR, d_err,
                               s);
  if (e == cudaSuccess)
    e = negf::launch_block_columns(d_tasks, nt, (uint32_t)(nt * (wr.L + 2)), wr.W, prec, d_wire,
                                   d_eta32, d_phi, d_phi32, d_sig, d_gam, d_gL, d_gR, d_st, d_w,
                                   d_rs, d_mw, d_c, d_err, nullptr, nullptr, s, 0,
                                   cta ? 0 : wr.W);
  if (e == cudaSuccess && cta)
    e = negf::launch_chain_cta(d_tasks, d_jobs, wr.W == 64 ? (uint32_t)jobs.size() : 0u,
                               wr.W == 64 ? 0u : (uint32_t)jobs.size(), d_eta32, d_phi32, d_gam,
                               d_gL, d_gR, d_st, d_w, d_alias, d_err, s);
  if (e == cudaSuccess)
    e = negf::launch_alias_build(d_tasks, nt, (uint32_t)(nt * (rows + 2)), (int)K, prec, d_w,
                                 d_rs, d_mw, d_alias, d_mode_alias, d_err, s);
  int32_t h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, d_err, sizeof h_err, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return NEGF_E_CUDA;
  if (h_err & negf::ERR_INPUT) return NEGF_E_INVALID;
  if (h_err & negf::ERR_TIMEOUT) return NEGF_E_TIMEOUT;
  if (h_err) return NEGF_E_NUMERIC;
  return NEGF_OK;
}
