// Host side of the C ABI declared in include/negf.h: argument checks, memory layout of the
// task batch, stream-ordered allocation and the kernel sequence of each call.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "negf_internal.cuh"

using negf::cd;
using negf::TaskDesc;

// Per-kernel device-time accounting (CUDA events on the context stream around each launch).
struct ProfEntry {
  std::string name;
  uint64_t launches = 0;
  double ms = 0.0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
};

struct negf_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  int sm_count = 1;
  std::string err;
  unsigned long long* d_counter = nullptr;   // work counter of the walk kernel
  bool prof = false;
  std::vector<ProfEntry> prof_entries;
  std::vector<cudaEvent_t> event_pool;
};

struct negf_tables_s {
  negf_ctx ctx = nullptr;
  int n_wires = 0, n_tasks = 0, precision = 0, max_W = 1, max_L = 1, max_K = 3;
  uint32_t total_jobs = 0;
  std::vector<TaskDesc> h_tasks;
  std::vector<int32_t> h_wire_task0;
  TaskDesc* d_tasks = nullptr;
  int32_t* d_wire_task0 = nullptr;
  double* d_wire = nullptr;
  cd* d_sig = nullptr;
  double* d_gam = nullptr;
  uint64_t* d_tab = nullptr;
  uint64_t* d_mode_tab = nullptr;
  double* d_mode_w = nullptr;
  double* d_c = nullptr;
  double* d_rowsum = nullptr;
  void* d_weights = nullptr;     // kept only with keep_weights
  int32_t* d_err = nullptr;
  uint64_t bytes = 0;
};

struct negf_tally_s {
  negf_ctx ctx = nullptr;
  int n_tasks = 0;
  int start_lead = 0;
  uint64_t* d_counts = nullptr;
};

namespace {

negf_status fail(negf_ctx ctx, negf_status st, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return st;
}

#define CUDA_TRY(ctx, call)                                                                 \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail((ctx), e_ == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,      \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
  } while (0)

// Make the context's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

template <typename T>
cudaError_t dalloc(T** p, size_t count, cudaStream_t s, uint64_t* bytes) {
  *p = nullptr;
  if (count == 0) count = 1;
  if (bytes) *bytes += count * sizeof(T);
  return cudaMallocAsync(reinterpret_cast<void**>(p), count * sizeof(T), s);
}

template <typename T>
void dfree(T*& p, cudaStream_t s) {
  if (p) cudaFreeAsync(p, s);
  p = nullptr;
}

void release_tables(negf_tables t) {
  if (!t) return;
  cudaStream_t s = t->ctx ? t->ctx->stream : nullptr;
  dfree(t->d_tasks, s);
  dfree(t->d_wire_task0, s);
  dfree(t->d_wire, s);
  dfree(t->d_sig, s);
  dfree(t->d_gam, s);
  dfree(t->d_tab, s);
  dfree(t->d_mode_tab, s);
  dfree(t->d_mode_w, s);
  dfree(t->d_c, s);
  dfree(t->d_rowsum, s);
  dfree(t->d_weights, s);
  dfree(t->d_err, s);
  delete t;
}

cudaEvent_t take_event(negf_ctx ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

// Records an event pair around the launches of one named kernel when profiling is on.
struct ProfScope {
  negf_ctx ctx;
  int idx = -1;
  uint64_t kernels = 1;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(negf_ctx c, const char* name, uint64_t n_kernels = 1) : ctx(c), kernels(n_kernels) {
    if (!ctx || !ctx->prof) return;
    for (size_t i = 0; i < ctx->prof_entries.size(); ++i)
      if (ctx->prof_entries[i].name == name) idx = (int)i;
    if (idx < 0) {
      ctx->prof_entries.push_back(ProfEntry{});
      ctx->prof_entries.back().name = name;
      idx = (int)ctx->prof_entries.size() - 1;
    }
    a = take_event(ctx);
    b = take_event(ctx);
    if (a && b) cudaEventRecord(a, ctx->stream);
  }
  ~ProfScope() {
    if (idx < 0 || !a || !b) return;
    cudaEventRecord(b, ctx->stream);
    ctx->prof_entries[idx].pending.emplace_back(a, b);
    ctx->prof_entries[idx].launches += kernels;
  }
};

void prof_resolve(negf_ctx ctx) {
  for (auto& e : ctx->prof_entries) {
    for (auto& pr : e.pending) {
      float ms = 0.f;
      if (cudaEventSynchronize(pr.second) == cudaSuccess &&
          cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
        e.ms += ms;
      ctx->event_pool.push_back(pr.first);
      ctx->event_pool.push_back(pr.second);
    }
    e.pending.clear();
  }
}

std::string err_bits(int32_t e) {
  std::string s;
  if (e & negf::ERR_NONFINITE) s += " non-finite Green's function or weight;";
  if (e & negf::ERR_ROWSUM) s += " table row does not sum to <i|A|i>;";
  if (e & negf::ERR_INPUT) s += " input value outside the domain (non-finite, eta < 0 or energy on a lead band edge);";
  if (e & negf::ERR_SINGULAR) s += " singular slice block;";
  return s;
}

// Synchronise and report any device-side error recorded for the tables.
negf_status check_device(negf_ctx ctx, negf_tables t) {
  int32_t e = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&e, t->d_err, sizeof e, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (e & negf::ERR_INPUT) return fail(ctx, NEGF_E_INVALID, "device check:%s", err_bits(e).c_str());
  if (e) return fail(ctx, NEGF_E_NUMERIC, "device check:%s", err_bits(e).c_str());
  return NEGF_OK;
}

bool band_edge(double E, int W, double t) {
  for (int m = 1; m <= W; ++m) {
    const double eps = -2.0 * t * cos(m * M_PI / (W + 1));
    if (fabs(fabs(E - eps) - 2.0 * t) <= 1e-12 * t) return true;
  }
  return false;
}

}  // namespace

extern "C" {

int negf_abi_version(void) { return NEGF_ABI_VERSION; }

negf_status negf_create(negf_ctx* out, int device, void* stream) {
  if (!out) return NEGF_E_INVALID;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return NEGF_E_CUDA;
  negf_ctx ctx = new (std::nothrow) negf_ctx_s;
  if (!ctx) return NEGF_E_NOMEM;
  ctx->device = device;
  ctx->stream = static_cast<cudaStream_t>(stream);
  DeviceGuard g(device);
  // Tables and scratch come from the device's default stream-ordered pool.  Keep freed blocks
  // in the pool across synchronisations instead of unmapping them at every sync (the default
  // release threshold of 0 makes each build re-map hundreds of MB).
  cudaMemPool_t pool = nullptr;
  if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess && pool) {
    uint64_t keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
  }
  if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) !=
          cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->d_counter), sizeof(unsigned long long)) !=
          cudaSuccess) {
    delete ctx;
    return NEGF_E_CUDA;
  }
  *out = ctx;
  return NEGF_OK;
}

void negf_destroy(negf_ctx ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  prof_resolve(ctx);
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  cudaFree(ctx->d_counter);
  delete ctx;
}

negf_status negf_profile_enable(negf_ctx ctx, int32_t on) {
  if (!ctx) return NEGF_E_INVALID;
  DeviceGuard g(ctx->device);
  prof_resolve(ctx);
  ctx->prof_entries.clear();
  ctx->prof = on != 0;
  return NEGF_OK;
}

negf_status negf_profile_read(negf_ctx ctx, int32_t cap, char* names, uint64_t* launches,
                              double* total_ms, int32_t* n_out) {
  if (!ctx || !n_out || cap < 0 || (cap > 0 && (!names || !launches || !total_ms)))
    return fail(ctx, NEGF_E_INVALID, "negf_profile_read: bad argument");
  DeviceGuard g(ctx->device);
  prof_resolve(ctx);
  const int n = (int)ctx->prof_entries.size();
  for (int i = 0; i < n && i < cap; ++i) {
    const ProfEntry& e = ctx->prof_entries[i];
    memset(names + 32 * i, 0, 32);
    strncpy(names + 32 * i, e.name.c_str(), 31);
    launches[i] = e.launches;
    total_ms[i] = e.ms;
  }
  *n_out = n;
  return NEGF_OK;
}

const char* negf_last_error(negf_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }

negf_status negf_build_tables(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                              const negf_build_opts* opts, negf_tables* out) {
  if (!ctx) return NEGF_E_INVALID;
  if (!out) return fail(ctx, NEGF_E_INVALID, "negf_build_tables: out is NULL");
  *out = nullptr;
  if (n_wires < 0 || (n_wires > 0 && !wires))
    return fail(ctx, NEGF_E_INVALID, "negf_build_tables: bad wire list");
  negf_build_opts o{NEGF_FP64, NEGF_MEM_HOST, 0, 0};
  if (opts) o = *opts;
  if (o.precision < NEGF_FP64 || o.precision > NEGF_SPLIT_TF32)
    return fail(ctx, NEGF_E_INVALID, "negf_build_tables: unknown precision %d", o.precision);
  if (o.memspace != NEGF_MEM_HOST && o.memspace != NEGF_MEM_DEVICE)
    return fail(ctx, NEGF_E_INVALID, "negf_build_tables: unknown memspace %d", o.memspace);
  if (o.reserved != 0) return fail(ctx, NEGF_E_INVALID, "negf_build_tables: reserved != 0");
  const bool dev_in = o.memspace == NEGF_MEM_DEVICE;
  const int prec = o.precision == NEGF_FP64 ? NEGF_FP64 : NEGF_FP32;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;

  negf_tables t = new (std::nothrow) negf_tables_s;
  if (!t) return fail(ctx, NEGF_E_NOMEM, "negf_build_tables: host allocation");
  t->ctx = ctx;
  t->n_wires = n_wires;
  t->precision = prec;
  // ---- validate and lay out the batch
  uint64_t tab_off = 0, g_off = 0, wire_off = 0, start_off = 0;
  uint32_t mode_off = 0, lead_off = 0, row_base = 0, col_base = 0, phi_off = 0;
  t->h_wire_task0.push_back(0);
  for (int w = 0; w < n_wires; ++w) {
    const negf_wire& wr = wires[w];
    if (wr.W < 1 || wr.W > NEGF_MAX_W || wr.L < 1 || !(wr.t > 0.0) || !isfinite(wr.t) ||
        wr.n_energy < 0) {
      release_tables(t);
      return fail(ctx, NEGF_E_INVALID, "wire %d: need 1 <= W <= %d, L >= 1, t > 0, n_energy >= 0",
                  w, NEGF_MAX_W);
    }
    if (wr.lead_model != NEGF_LEAD_STRIP && wr.lead_model != NEGF_LEAD_WIDE_BAND) {
      release_tables(t);
      return fail(ctx, NEGF_E_INVALID, "wire %d: unknown lead model %d", w, wr.lead_model);
    }
    if (wr.lead_model == NEGF_LEAD_WIDE_BAND && !(wr.gamma_lead > 0.0 && isfinite(wr.gamma_lead))) {
      release_tables(t);
      return fail(ctx, NEGF_E_INVALID, "wire %d: wide-band lead needs gamma_lead > 0", w);
    }
    const int64_t n = (int64_t)wr.W * wr.L;
    const int64_t K = n + 2, rows = n + 2 * wr.W;
    if (n > NEGF_MAX_SITES) {
      release_tables(t);
      return fail(ctx, NEGF_E_INVALID, "wire %d: W*L = %lld exceeds the supported %d sites",
                  w, (long long)n, NEGF_MAX_SITES);
    }
    if (!wr.onsite || !wr.eta || (wr.n_energy > 0 && !wr.energy)) {
      release_tables(t);
      return fail(ctx, NEGF_E_INVALID, "wire %d: NULL array", w);
    }
    if (!dev_in) {
      for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(wr.onsite[i]) || !isfinite(wr.eta[i]) || !(wr.eta[i] >= 0.0)) {
          release_tables(t);
          return fail(ctx, NEGF_E_INVALID, "wire %d: site %lld: onsite/eta not finite or eta < 0",
                      w, (long long)i);
        }
      }
    }
    // energies and weights are always brought to the host (they become task scalars)
    std::vector<double> E(wr.n_energy), wE(wr.n_energy, 1.0);
    if (wr.n_energy > 0) {
      if (dev_in) {
        CUDA_TRY(ctx, cudaMemcpy(E.data(), wr.energy, sizeof(double) * wr.n_energy,
                                 cudaMemcpyDeviceToHost));
        if (wr.energy_weight)
          CUDA_TRY(ctx, cudaMemcpy(wE.data(), wr.energy_weight, sizeof(double) * wr.n_energy,
                                   cudaMemcpyDeviceToHost));
      } else {
        memcpy(E.data(), wr.energy, sizeof(double) * wr.n_energy);
        if (wr.energy_weight) memcpy(wE.data(), wr.energy_weight, sizeof(double) * wr.n_energy);
      }
    }
    for (int k = 0; k < wr.n_energy; ++k) {
      if (!isfinite(E[k]) || !isfinite(wE[k])) {
        release_tables(t);
        return fail(ctx, NEGF_E_INVALID, "wire %d: energy %d not finite", w, k);
      }
      if (wr.lead_model == NEGF_LEAD_STRIP && band_edge(E[k], wr.W, wr.t)) {
        release_tables(t);
        return fail(ctx, NEGF_E_INVALID, "wire %d: energy %.17g lies on a lead band edge", w, E[k]);
      }
      TaskDesc d{};
      d.wire = w;
      d.e_idx = k;
      d.W = wr.W;
      d.L = wr.L;
      d.n = (int)n;
      d.K = (int)K;
      d.rows = (int)rows;
      d.lead_model = wr.lead_model;
      d.E = E[k];
      d.t = wr.t;
      d.w_E = wE[k];
      d.gamma_lead = wr.gamma_lead;
      d.tab_off = tab_off;
      d.wt_off = tab_off;
      d.g_off = g_off;
      d.mode_off = mode_off;
      d.lead_off = lead_off;
      d.onsite_off = (uint32_t)wire_off;
      d.row_base = row_base;
      d.col_base = col_base;
      d.phi_off = phi_off;
      d.start_off = start_off;
      t->h_tasks.push_back(d);
      tab_off += (uint64_t)rows * K;
      g_off += (uint64_t)wr.L * wr.W * wr.W;
      mode_off += 2 * wr.W;
      lead_off += wr.W;
      row_base += (uint32_t)(rows + 2);
      col_base += (uint32_t)(wr.L + 2);
      start_off += (uint64_t)(wr.L + 2) * wr.W * wr.W;
      t->max_W = std::max(t->max_W, wr.W);
      t->max_L = std::max(t->max_L, wr.L);
      t->max_K = std::max(t->max_K, (int)K);
    }
    wire_off += 2 * (uint64_t)n;
    phi_off += (uint32_t)(wr.W * wr.W);
    t->h_wire_task0.push_back((int32_t)t->h_tasks.size());
  }
  t->n_tasks = (int)t->h_tasks.size();
  t->total_jobs = row_base;
  const int nt = t->n_tasks;
  // ---- device buffers
  // RGF and start blocks in the table precision: complex128 (FP64) or complex64 (FP32)
  double* d_gL = nullptr;
  double* d_gR = nullptr;
  double* d_start = nullptr;
  double* d_phi = nullptr;       // per wire: transverse modes (FP64), then the FP32 copy
  float* d_eta32 = nullptr;      // per wire: eta in FP32
  void* d_weights = nullptr;
  const uint64_t cw = negf::block_bytes(prec) / sizeof(double);   // doubles per complex
  const size_t wsz = prec == NEGF_FP64 ? sizeof(double) : sizeof(float);
#define ALLOC(ptr, count)                                                  \
  do {                                                                     \
    cudaError_t e_ = dalloc(&(ptr), (count), s, &t->bytes);                \
    if (e_ != cudaSuccess) {                                               \
      release_tables(t);                                                   \
      dfree(d_gL, s);                                                      \
      dfree(d_gR, s);                                                      \
      dfree(d_start, s);                                                   \
      dfree(d_phi, s);                                                     \
      dfree(d_eta32, s);                                                   \
      if (d_weights) cudaFreeAsync(d_weights, s);                          \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA, \
                  "allocation of %s (%zu elements): %s", #ptr, (size_t)(count), \
                  cudaGetErrorString(e_));                                 \
    }                                                                      \
  } while (0)
  ALLOC(t->d_tasks, nt);
  ALLOC(t->d_wire_task0, n_wires + 1);
  ALLOC(t->d_wire, wire_off);
  ALLOC(t->d_sig, lead_off);
  ALLOC(t->d_gam, lead_off);
  ALLOC(t->d_tab, tab_off);
  ALLOC(t->d_mode_tab, mode_off);
  ALLOC(t->d_mode_w, mode_off);
  ALLOC(t->d_c, 2 * (size_t)nt);
  ALLOC(t->d_rowsum, row_base);
  ALLOC(t->d_err, 1);
  ALLOC(d_gL, g_off * cw);
  ALLOC(d_gR, g_off * cw);
  ALLOC(d_start, start_off * cw);
  ALLOC(d_phi, (uint64_t)phi_off + (phi_off + 1) / 2);
  ALLOC(d_eta32, wire_off / 2);
  {
    cudaError_t e_ = cudaMallocAsync(&d_weights, std::max<uint64_t>(tab_off, 1) * wsz, s);
    if (e_ != cudaSuccess) {
      release_tables(t);
      dfree(d_gL, s);
      dfree(d_gR, s);
      dfree(d_start, s);
      dfree(d_phi, s);
      dfree(d_eta32, s);
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                  "allocation of the weight scratch: %s", cudaGetErrorString(e_));
    }
  }
#undef ALLOC
  // ---- inputs
  auto bail = [&](negf_status st) {
    release_tables(t);
    dfree(d_gL, s);
    dfree(d_gR, s);
    dfree(d_start, s);
    dfree(d_phi, s);
    dfree(d_eta32, s);
    if (d_weights) cudaFreeAsync(d_weights, s);
    return st;
  };
#define STEP(call)                                                                        \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      return bail(fail(ctx, NEGF_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)));      \
  } while (0)
  STEP(cudaMemsetAsync(t->d_err, 0, sizeof(int32_t), s));
  if (nt > 0) {
    STEP(cudaMemcpyAsync(t->d_tasks, t->h_tasks.data(), sizeof(TaskDesc) * nt,
                         cudaMemcpyHostToDevice, s));
  }
  STEP(cudaMemcpyAsync(t->d_wire_task0, t->h_wire_task0.data(), sizeof(int32_t) * (n_wires + 1),
                       cudaMemcpyHostToDevice, s));
  {
    std::vector<double> stage;
    if (!dev_in) stage.reserve(wire_off);
    uint64_t off = 0;
    for (int w = 0; w < n_wires; ++w) {
      const int64_t n = (int64_t)wires[w].W * wires[w].L;
      if (dev_in) {
        STEP(cudaMemcpyAsync(t->d_wire + off, wires[w].onsite, sizeof(double) * n,
                             cudaMemcpyDeviceToDevice, s));
        STEP(cudaMemcpyAsync(t->d_wire + off + n, wires[w].eta, sizeof(double) * n,
                             cudaMemcpyDeviceToDevice, s));
      } else {
        stage.insert(stage.end(), wires[w].onsite, wires[w].onsite + n);
        stage.insert(stage.end(), wires[w].eta, wires[w].eta + n);
      }
      off += 2 * n;
    }
    if (!dev_in && off > 0)
      STEP(cudaMemcpyAsync(t->d_wire, stage.data(), sizeof(double) * off, cudaMemcpyHostToDevice,
                           s));
    if (!dev_in) STEP(cudaStreamSynchronize(s));   // the staging vector dies here
  }
  // ---- kernels: validation, lead modes, sweeps, block columns + weights, alias tables
  if (nt > 0) {
    if (dev_in) {
      ProfScope ps(ctx, "validate_kernel", 2);
      STEP(negf::launch_validate(t->d_tasks, nt, t->d_wire, t->d_err, s));
    }
    {
      ProfScope ps(ctx, "lead_modes_kernel");
      STEP(negf::launch_lead_modes(t->d_tasks, nt, t->max_W, t->d_wire, d_phi,
                                   reinterpret_cast<float*>(d_phi + phi_off), d_eta32, t->d_sig,
                                   t->d_gam, t->d_err, s));
    }
    {
      ProfScope ps(ctx, "rgf_sweep_kernel");
      STEP(negf::launch_rgf_sweep(t->d_tasks, nt, t->max_W, prec, t->d_wire, d_phi, t->d_sig,
                                  d_gL, d_gR, t->d_err, s));
    }
    {
      ProfScope ps(ctx, "diag_chain_kernels", 2);
      STEP(negf::launch_block_columns(t->d_tasks, nt, col_base, t->max_W, prec, t->d_wire,
                                      d_eta32, d_phi, reinterpret_cast<float*>(d_phi + phi_off),
                                      t->d_sig, t->d_gam, d_gL, d_gR, d_start, d_weights,
                                      t->d_rowsum, t->d_mode_w, t->d_c, t->d_err, s));
    }
    {
      ProfScope ps(ctx, "alias_kernel");
      STEP(negf::launch_alias_build(t->d_tasks, nt, t->total_jobs, t->max_K, prec, d_weights,
                                    t->d_rowsum, t->d_mode_w, t->d_tab, t->d_mode_tab,
                                    t->d_err, s));
    }
  }
#undef STEP
  dfree(d_gL, s);
  dfree(d_gR, s);
  dfree(d_start, s);
  dfree(d_phi, s);
  dfree(d_eta32, s);
  t->bytes -= (2 * std::max<uint64_t>(g_off * cw, 1) + std::max<uint64_t>(start_off * cw, 1) +
               std::max<uint64_t>((uint64_t)phi_off + (phi_off + 1) / 2, 1)) * sizeof(double) +
              std::max<uint64_t>(wire_off / 2, 1) * sizeof(float);
  if (o.keep_weights) {
    t->d_weights = d_weights;
    t->bytes += std::max<uint64_t>(tab_off, 1) * wsz;
  } else {
    cudaFreeAsync(d_weights, s);
  }
  *out = t;
  return NEGF_OK;
}

int32_t negf_tables_num_tasks(negf_tables t) { return t ? t->n_tasks : 0; }
int32_t negf_tables_num_wires(negf_tables t) { return t ? t->n_wires : 0; }
uint64_t negf_tables_device_bytes(negf_tables t) { return t ? t->bytes : 0; }

void negf_tables_free(negf_tables t) {
  if (!t) return;
  DeviceGuard g(t->ctx->device);
  release_tables(t);
}

negf_status negf_get_task_info(negf_ctx ctx, negf_tables t, int32_t task, negf_task_info* out) {
  if (!ctx || !t || !out || t->ctx != ctx) return fail(ctx, NEGF_E_INVALID, "negf_get_task_info: bad handle");
  if (task < 0 || task >= t->n_tasks) return fail(ctx, NEGF_E_INVALID, "task %d out of range", task);
  DeviceGuard g(ctx->device);
  double c[2];
  CUDA_TRY(ctx, cudaMemcpyAsync(c, t->d_c + 2 * task, sizeof c, cudaMemcpyDeviceToHost, ctx->stream));
  negf_status st = check_device(ctx, t);
  if (st != NEGF_OK) return st;
  const TaskDesc& d = t->h_tasks[task];
  out->wire = d.wire;
  out->energy_index = d.e_idx;
  out->W = d.W;
  out->L = d.L;
  out->n = d.n;
  out->K = d.K;
  out->rows = d.rows;
  out->reserved = 0;
  out->energy = d.E;
  out->energy_weight = d.w_E;
  out->c[0] = c[0];
  out->c[1] = c[1];
  return NEGF_OK;
}

negf_status negf_export_tables(negf_ctx ctx, negf_tables t, int32_t task, int32_t what,
                               void* host_buf, size_t* bytes) {
  if (!ctx || !t || !bytes || t->ctx != ctx) return fail(ctx, NEGF_E_INVALID, "negf_export_tables: bad argument");
  if (task < 0 || task >= t->n_tasks) return fail(ctx, NEGF_E_INVALID, "task %d out of range", task);
  const TaskDesc& d = t->h_tasks[task];
  size_t need = 0;
  switch (what) {
    case NEGF_EXPORT_ALIAS: need = sizeof(uint64_t) * (size_t)d.rows * d.K; break;
    case NEGF_EXPORT_MODE_ALIAS: need = sizeof(uint64_t) * 2 * (size_t)d.W; break;
    case NEGF_EXPORT_WEIGHTS:
      if (!t->d_weights) return fail(ctx, NEGF_E_INVALID, "weights were not kept (keep_weights = 0)");
      need = sizeof(double) * (size_t)d.rows * d.K;
      break;
    case NEGF_EXPORT_MODE_WEIGHTS: need = sizeof(double) * 2 * (size_t)d.W; break;
    case NEGF_EXPORT_ROWSUM: need = sizeof(double) * (size_t)d.rows; break;
    default: return fail(ctx, NEGF_E_INVALID, "unknown export kind %d", what);
  }
  if (!host_buf) { *bytes = need; return NEGF_OK; }
  if (*bytes < need) return fail(ctx, NEGF_E_INVALID, "export buffer too small (%zu < %zu)", *bytes, need);
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  switch (what) {
    case NEGF_EXPORT_ALIAS:
      CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, t->d_tab + d.tab_off, need, cudaMemcpyDeviceToHost, s));
      break;
    case NEGF_EXPORT_MODE_ALIAS:
      CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, t->d_mode_tab + d.mode_off, need, cudaMemcpyDeviceToHost, s));
      break;
    case NEGF_EXPORT_WEIGHTS:
      if (t->precision == NEGF_FP64) {
        CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, static_cast<double*>(t->d_weights) + d.wt_off, need,
                                      cudaMemcpyDeviceToHost, s));
      } else {
        std::vector<float> tmp((size_t)d.rows * d.K);
        CUDA_TRY(ctx, cudaMemcpyAsync(tmp.data(), static_cast<float*>(t->d_weights) + d.wt_off,
                                      tmp.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
        CUDA_TRY(ctx, cudaStreamSynchronize(s));
        double* o = static_cast<double*>(host_buf);
        for (size_t i = 0; i < tmp.size(); ++i) o[i] = tmp[i];
      }
      break;
    case NEGF_EXPORT_MODE_WEIGHTS:
      CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, t->d_mode_w + d.mode_off, need, cudaMemcpyDeviceToHost, s));
      break;
    case NEGF_EXPORT_ROWSUM:
      CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, t->d_rowsum + d.row_base, need, cudaMemcpyDeviceToHost, s));
      break;
  }
  negf_status st = check_device(ctx, t);
  if (st != NEGF_OK) return st;
  *bytes = need;
  return NEGF_OK;
}

static negf_status walk_common(negf_ctx ctx, negf_tables t, int32_t start_lead, uint32_t max_steps,
                               const char* who) {
  if (!ctx || !t || t->ctx != ctx) return fail(ctx, NEGF_E_INVALID, "%s: bad handle", who);
  if (start_lead != 0 && start_lead != 1) return fail(ctx, NEGF_E_INVALID, "%s: start_lead must be 0 or 1", who);
  if (max_steps < 1 || max_steps > NEGF_MAX_STEPS)
    return fail(ctx, NEGF_E_INVALID, "%s: max_steps must be in [1, %u]", who, NEGF_MAX_STEPS);
  return NEGF_OK;
}

negf_status negf_walk(negf_ctx ctx, negf_tables t, int32_t start_lead, uint64_t seed,
                      uint64_t walkers_per_task, uint64_t walker_id_offset, uint32_t max_steps,
                      negf_tally* out) {
  negf_status st = walk_common(ctx, t, start_lead, max_steps, "negf_walk");
  if (st != NEGF_OK) return st;
  if (!out) return fail(ctx, NEGF_E_INVALID, "negf_walk: out is NULL");
  *out = nullptr;
  if (walkers_per_task > (1ull << 40))
    return fail(ctx, NEGF_E_INVALID, "negf_walk: walkers_per_task above 2^40");
  DeviceGuard g(ctx->device);
  negf_tally tl = new (std::nothrow) negf_tally_s;
  if (!tl) return fail(ctx, NEGF_E_NOMEM, "negf_walk: host allocation");
  tl->ctx = ctx;
  tl->n_tasks = t->n_tasks;
  tl->start_lead = start_lead;
  cudaError_t e = dalloc(&tl->d_counts, (size_t)t->n_tasks * NEGF_TALLY_FIELDS, ctx->stream, nullptr);
  if (e != cudaSuccess) {
    delete tl;
    return fail(ctx, NEGF_E_NOMEM, "negf_walk: tally allocation: %s", cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(tl->d_counts, 0, sizeof(uint64_t) * std::max(1, t->n_tasks) * NEGF_TALLY_FIELDS,
                      ctx->stream);
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "walk_kernel", (t->n_tasks + 1023) / 1024);
    e = negf::launch_walk(t->d_tasks, 0, t->n_tasks, t->d_tab, t->d_mode_tab, t->d_c, start_lead,
                          seed, walkers_per_task, walker_id_offset, max_steps, ctx->d_counter,
                          tl->d_counts, nullptr, nullptr, ctx->sm_count, ctx->stream);
  }
  if (e != cudaSuccess) {
    cudaFreeAsync(tl->d_counts, ctx->stream);
    delete tl;
    return fail(ctx, NEGF_E_CUDA, "negf_walk: %s", cudaGetErrorString(e));
  }
  *out = tl;
  return NEGF_OK;
}

negf_status negf_walk_trace(negf_ctx ctx, negf_tables t, int32_t task, int32_t start_lead,
                            uint64_t seed, uint64_t walker_id_offset, uint64_t n_walkers,
                            uint32_t max_steps, int32_t* d_lead, uint32_t* d_steps) {
  negf_status st = walk_common(ctx, t, start_lead, max_steps, "negf_walk_trace");
  if (st != NEGF_OK) return st;
  if (task < 0 || task >= t->n_tasks) return fail(ctx, NEGF_E_INVALID, "task %d out of range", task);
  if (n_walkers > 0 && (!d_lead || !d_steps)) return fail(ctx, NEGF_E_INVALID, "negf_walk_trace: NULL output");
  if (n_walkers > (1ull << 40)) return fail(ctx, NEGF_E_INVALID, "negf_walk_trace: too many walkers");
  DeviceGuard g(ctx->device);
  uint64_t* tmp = nullptr;
  CUDA_TRY(ctx, dalloc(&tmp, NEGF_TALLY_FIELDS, ctx->stream, nullptr));
  cudaError_t e = cudaMemsetAsync(tmp, 0, sizeof(uint64_t) * NEGF_TALLY_FIELDS, ctx->stream);
  if (e == cudaSuccess)
    e = negf::launch_walk(t->d_tasks, task, 1, t->d_tab, t->d_mode_tab, t->d_c, start_lead, seed,
                          n_walkers, walker_id_offset, max_steps, ctx->d_counter, tmp, d_lead,
                          d_steps, ctx->sm_count, ctx->stream);
  cudaFreeAsync(tmp, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "negf_walk_trace: %s", cudaGetErrorString(e));
  return NEGF_OK;
}

negf_status negf_tally_counts(negf_ctx ctx, negf_tally tl, uint64_t* host_counts) {
  if (!ctx || !tl || tl->ctx != ctx || (!host_counts && tl->n_tasks > 0))
    return fail(ctx, NEGF_E_INVALID, "negf_tally_counts: bad argument");
  DeviceGuard g(ctx->device);
  if (tl->n_tasks > 0)
    CUDA_TRY(ctx, cudaMemcpyAsync(host_counts, tl->d_counts,
                                  sizeof(uint64_t) * tl->n_tasks * NEGF_TALLY_FIELDS,
                                  cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return NEGF_OK;
}

negf_status negf_tally_accumulate(negf_ctx ctx, negf_tally tl, const uint64_t* host_counts) {
  if (!ctx || !tl || tl->ctx != ctx || (!host_counts && tl->n_tasks > 0))
    return fail(ctx, NEGF_E_INVALID, "negf_tally_accumulate: bad argument");
  const size_t m = (size_t)tl->n_tasks * NEGF_TALLY_FIELDS;
  std::vector<uint64_t> cur(m);
  negf_status st = negf_tally_counts(ctx, tl, cur.data());
  if (st != NEGF_OK) return st;
  for (size_t i = 0; i < m; ++i) cur[i] += host_counts[i];
  DeviceGuard g(ctx->device);
  if (m) {
    CUDA_TRY(ctx, cudaMemcpyAsync(tl->d_counts, cur.data(), sizeof(uint64_t) * m,
                                  cudaMemcpyHostToDevice, ctx->stream));
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return NEGF_OK;
}

int32_t negf_tally_start_lead(negf_tally tl) { return tl ? tl->start_lead : -1; }

void negf_tally_free(negf_tally tl) {
  if (!tl) return;
  DeviceGuard g(tl->ctx->device);
  if (tl->d_counts) cudaFreeAsync(tl->d_counts, tl->ctx->stream);
  delete tl;
}

negf_status negf_current(negf_ctx ctx, negf_tables t, negf_tally tl, double mu_p, double mu_q,
                         double kT, double* I, double* se, double* T, double* T_se) {
  if (!ctx || !t || !tl || t->ctx != ctx || tl->ctx != ctx || tl->n_tasks != t->n_tasks)
    return fail(ctx, NEGF_E_INVALID, "negf_current: bad or mismatched handles");
  if (!(kT > 0.0) || !isfinite(mu_p) || !isfinite(mu_q) || !isfinite(kT))
    return fail(ctx, NEGF_E_INVALID, "negf_current: need finite mu and kT > 0");
  if (t->n_wires > 0 && (!I || !se)) return fail(ctx, NEGF_E_INVALID, "negf_current: NULL I/se");
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  const size_t nw = t->n_wires, nt = t->n_tasks, m = 2 * nw + 2 * nt + 1;
  double* d_out = nullptr;
  CUDA_TRY(ctx, dalloc(&d_out, m, s, nullptr));
  cudaError_t e;
  {
    ProfScope ps(ctx, "current_kernel");
    e = negf::launch_current(t->d_tasks, (int)nt, (int)nw, t->d_wire_task0, t->d_c,
                             tl->d_counts, tl->start_lead, mu_p, mu_q, kT, d_out, s);
  }
  std::vector<double> h(m);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * m, cudaMemcpyDeviceToHost, s);
  cudaFreeAsync(d_out, s);
  if (e != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "negf_current: %s", cudaGetErrorString(e));
  negf_status st = check_device(ctx, t);
  if (st != NEGF_OK) return st;
  for (size_t w = 0; w < nw; ++w) { I[w] = h[w]; se[w] = h[nw + w]; }
  if (T) for (size_t k = 0; k < nt; ++k) T[k] = h[2 * nw + k];
  if (T_se) for (size_t k = 0; k < nt; ++k) T_se[k] = h[2 * nw + nt + k];
  if (h[m - 1] > 0.0)
    return fail(ctx, NEGF_E_STEPCAP, "negf_current: %.0f walks reached max_steps", h[m - 1]);
  return NEGF_OK;
}

}  // extern "C"
