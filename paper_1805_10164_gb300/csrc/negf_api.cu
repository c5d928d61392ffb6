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
using negf::TcJob;

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
  cudaStream_t walk_stream = nullptr;        // second stream of negf_run (created on first use)
  cudaStream_t capture_stream = nullptr;     // plans are captured here (the context stream may
                                             // be the legacy default stream, which cannot be)
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
  bool tables_released = false;  // negf_run: alias tables freed wave by wave
  bool any_two = false;          // some task has two-level tables
  int n_waves = 1;
  void* d_green = nullptr;       // keep_green: dense G per task, then G Phi per task
  void* d_gphi = nullptr;
  double* d_phi = nullptr;       // keep_green / keep_weights: transverse modes (the gradient)
  uint64_t green_total = 0, gphi_total = 0, score_stride = 0;
  uint32_t mode_stride = 0;
};

struct negf_tally_s {
  negf_ctx ctx = nullptr;
  int n_tasks = 0;
  int start_lead = 0;
  uint64_t* d_counts = nullptr;
  uint64_t* d_score = nullptr;        // score tallies [2][score_stride] (negf_walk_score)
  uint64_t* d_mode_score = nullptr;   // [2][mode_stride]
  uint64_t score_stride = 0;
  uint32_t mode_stride = 0;
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
  dfree(t->d_green, s);
  dfree(t->d_gphi, s);
  dfree(t->d_phi, s);
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
  cudaStream_t stream = nullptr;
  cudaEvent_t a = nullptr, b = nullptr;
  ProfScope(negf_ctx c, const char* name, uint64_t n_kernels = 1, cudaStream_t s = nullptr)
      : ctx(c), kernels(n_kernels), stream(s ? s : (c ? c->stream : nullptr)) {
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
    if (a && b) cudaEventRecord(a, stream);
  }
  ~ProfScope() {
    if (idx < 0 || !a || !b) return;
    cudaEventRecord(b, stream);
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
  if (e & negf::ERR_TIMEOUT) s += " a bounded device wait gave up;";
  return s;
}

// Status for a device error word (input errors first, then timeouts, then numerics).
negf_status err_status(int32_t e) {
  if (e & negf::ERR_INPUT) return NEGF_E_INVALID;
  if (e & negf::ERR_TIMEOUT) return NEGF_E_TIMEOUT;
  return NEGF_E_NUMERIC;
}

// Synchronise and report any device-side error recorded for the tables.
negf_status check_device(negf_ctx ctx, negf_tables t) {
  int32_t e = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&e, t->d_err, sizeof e, cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  if (e) return fail(ctx, err_status(e), "device check:%s", err_bits(e).c_str());
  return NEGF_OK;
}

bool band_edge(double E, int W, double t) {
  for (int m = 1; m <= W; ++m) {
    const double eps = -2.0 * t * cos(m * M_PI / (W + 1));
    if (fabs(fabs(E - eps) - 2.0 * t) <= 1e-12 * t) return true;
  }
  return false;
}

// Walkers per lane of a walk launch when no tuning picked them: two when the launch has
// two-level tables (tables far larger than L2, two dependent gathers per transition: more
// walks in flight hide more of the latency), one otherwise (L2-resident one-level tables and
// short walks, where the start and refill work of a second walker costs more than it hides).
int walk_slots(bool any_two) { return any_two ? 2 : 1; }

}  // namespace

extern "C" {

int negf_abi_version(void) { return NEGF_ABI_VERSION; }

negf_status negf_device_error_status(int32_t word, char* msg, size_t cap) {
  if (msg && cap > 0) {
    const std::string s = word ? err_bits(word) : std::string();
    const size_t k = std::min(s.size(), cap - 1);
    memcpy(msg, s.data(), k);
    msg[k] = 0;
  }
  return word ? err_status(word) : NEGF_OK;
}

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
  if (ctx->walk_stream) {
    cudaStreamSynchronize(ctx->walk_stream);
    cudaStreamDestroy(ctx->walk_stream);
  }
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
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

}  // extern "C"

namespace negf {

// Jobs of the tensor-core and CTA-wide chains for task `k` (index in its wave): direction 0
// takes every block column (it also emits the start slices) in pairs of neighbouring start
// slices, from the far end; direction 1 the columns that have slices beyond their start.
void add_tc_jobs(std::vector<TcJob>& jobs, int k, int L) {
  std::vector<std::pair<int, int>> cols;             // (m0, y)
  for (int y = 0; y < L + 2; ++y) cols.emplace_back(y < L ? y : (y == L ? 0 : L - 1), y);
  std::vector<std::pair<int, int>> d0 = cols, d1;
  std::stable_sort(d0.begin(), d0.end(), [](auto a, auto b) { return a.first > b.first; });
  for (auto& c : cols)
    if (c.first < L - 1) d1.push_back(c);
  std::stable_sort(d1.begin(), d1.end(), [](auto a, auto b) { return a.first < b.first; });
  for (size_t i = 0; i < d0.size(); i += 2)
    jobs.push_back(TcJob{k, 0, d0[i].second, i + 1 < d0.size() ? d0[i + 1].second : -1});
  for (size_t i = 0; i < d1.size(); i += 2)
    jobs.push_back(TcJob{k, 1, d1[i].second, i + 1 < d1.size() ? d1[i + 1].second : -1});
}

// Jobs of the W = 64 CTA-wide FP32 chain, which uses G = G^T: every block column towards
// slice 0 (pairs of neighbouring start slices, from the far end), and towards slice L - 1 only
// the injection column of lead L (its rows need every slice and have no transposed partner).
void add_sym_jobs(std::vector<TcJob>& jobs, int k, int L) {
  std::vector<std::pair<int, int>> d0;               // (m0, y)
  for (int y = 0; y < L + 2; ++y) d0.emplace_back(y < L ? y : (y == L ? 0 : L - 1), y);
  std::stable_sort(d0.begin(), d0.end(), [](auto a, auto b) { return a.first > b.first; });
  for (size_t i = 0; i < d0.size(); i += 2)
    jobs.push_back(TcJob{k, 0, d0[i].second, i + 1 < d0.size() ? d0[i + 1].second : -1});
  if (L > 1) jobs.push_back(TcJob{k, 1, L, -1});
}

// Longest chains first (the length of a job is the number of its steps).
void sort_jobs_longest_first(std::vector<TcJob>& jobs, const TaskDesc* desc) {
  auto len = [&](const TcJob& j) {
    const TaskDesc& d = desc[j.task];
    auto m0 = [&](int y) { return y < d.L ? y : (y == d.L ? 0 : d.L - 1); };
    const int a = m0(j.y0), b = j.y1 >= 0 ? m0(j.y1) : a;
    return j.dir == 0 ? std::max(a, b) : d.L - 1 - std::min(a, b);
  };
  std::stable_sort(jobs.begin(), jobs.end(),
                   [&](const TcJob& x, const TcJob& y) { return len(x) > len(y); });
}

}  // namespace negf

namespace {

// Validated layout of a batch of wires: one descriptor per (wire, energy) task with offsets as
// if the whole batch were built at once.
struct Plan {
  std::vector<TaskDesc> tasks;
  std::vector<int32_t> wire_task0;
  uint64_t tab_total = 0, green_total = 0, gphi_total = 0, g_total = 0;
  uint64_t wt_total = 0, l1w_total = 0;    // weights, level-1 weights (after the weights)
  uint64_t wire_total = 0;                 // doubles: onsite then eta per wire
  uint32_t lead_total = 0, mode_total = 0, phi_total = 0;
  int max_W = 1, max_L = 1, max_K = 3;
  int max_KA = 3;                          // longest row the alias kernel builds
  bool any_two = false;
  bool any_slice_h = false;                // some wire has a multi-orbital slice block
  uint64_t edge_total = 0;                 // fused tasks' edge blocks (complex64)
};

// Descriptors for the alias kernel: a two-level task's level-1 rows (K = L + 2 slots, weights at
// l1w_off, entries at l1_off); one-level tasks unchanged.
std::vector<TaskDesc> alias_descs(const std::vector<TaskDesc>& desc) {
  std::vector<TaskDesc> a = desc;
  for (TaskDesc& d : a)
    if (d.layout == NEGF_LAYOUT_TWO_LEVEL) {
      d.K = d.L + 2;
      d.tab_off = d.l1_off;
      d.wt_off = d.l1w_off;
    }
  return a;
}

negf_status make_plan(negf_ctx ctx, const negf_wire* wires, int n_wires, bool dev_in, Plan& P,
                      int layout_opt = NEGF_LAYOUT_AUTO, bool tc = false, bool fp32 = false,
                      bool one_level_first = false, bool fuse_l2 = false) {
  if (layout_opt < NEGF_LAYOUT_AUTO || layout_opt > NEGF_LAYOUT_TWO_LEVEL)
    return fail(ctx, NEGF_E_INVALID, "unknown table layout %d", layout_opt);
  uint64_t tab_off = 0, g_off = 0, wire_off = 0, start_off = 0, green_off = 0, gphi_off = 0;
  uint64_t wt_off = 0, l1w_rel = 0, edge_off = 0;
  uint32_t mode_off = 0, lead_off = 0, row_base = 0, col_base = 0, phi_off = 0;
  P.wire_task0.assign(1, 0);
  for (int w = 0; w < n_wires; ++w) {
    const negf_wire& wr = wires[w];
    if (wr.W < 1 || wr.W > NEGF_MAX_W || wr.L < 1 || !(wr.t > 0.0) || !isfinite(wr.t) ||
        wr.n_energy < 0)
      return fail(ctx, NEGF_E_INVALID, "wire %d: need 1 <= W <= %d, L >= 1, t > 0, n_energy >= 0",
                  w, NEGF_MAX_W);
    if (wr.lead_model != NEGF_LEAD_STRIP && wr.lead_model != NEGF_LEAD_WIDE_BAND)
      return fail(ctx, NEGF_E_INVALID, "wire %d: unknown lead model %d", w, wr.lead_model);
    if (wr.lead_model == NEGF_LEAD_WIDE_BAND && !(wr.gamma_lead > 0.0 && isfinite(wr.gamma_lead)))
      return fail(ctx, NEGF_E_INVALID, "wire %d: wide-band lead needs gamma_lead > 0", w);
    const int64_t n = (int64_t)wr.W * wr.L;
    const int64_t K = n + 2, rows = n + 2 * wr.W;
    // the tensor-core chain (split-TF32 builds of W = 64 wires) emits two-level tables
    const bool tc_wire = tc && wr.W == 64 && layout_opt != NEGF_LAYOUT_ONE_LEVEL;
    // automatic layout: two-level above the threshold, unless one-level tables are wanted
    // (the gradient) and the wire still fits them
    const int64_t auto_max = one_level_first ? NEGF_MAX_SITES : NEGF_AUTO_TWO_LEVEL_SITES;
    const int layout = tc_wire || (layout_opt == NEGF_LAYOUT_AUTO && n > auto_max)
                           ? NEGF_LAYOUT_TWO_LEVEL
                           : (layout_opt == NEGF_LAYOUT_AUTO ? NEGF_LAYOUT_ONE_LEVEL : layout_opt);
    const int64_t max_n = layout == NEGF_LAYOUT_TWO_LEVEL ? NEGF_MAX_SITES_TWO_LEVEL : NEGF_MAX_SITES;
    if (n > max_n)
      return fail(ctx, NEGF_E_INVALID, "wire %d: W*L = %lld exceeds the %lld sites of %s tables", w,
                  (long long)n, (long long)max_n,
                  layout == NEGF_LAYOUT_TWO_LEVEL ? "two-level" : "one-level");
    if (!wr.onsite || !wr.eta || (wr.n_energy > 0 && !wr.energy))
      return fail(ctx, NEGF_E_INVALID, "wire %d: NULL array", w);
    if (!dev_in) {
      for (int64_t i = 0; i < n; ++i)
        if (!isfinite(wr.onsite[i]) || !isfinite(wr.eta[i]) || !(wr.eta[i] >= 0.0))
          return fail(ctx, NEGF_E_INVALID, "wire %d: site %lld: onsite/eta not finite or eta < 0",
                      w, (long long)i);
      if (wr.slice_h)
        for (int a = 0; a < wr.W; ++a)
          for (int b = 0; b < wr.W; ++b)
            if (!isfinite(wr.slice_h[a * wr.W + b]) ||
                wr.slice_h[a * wr.W + b] != wr.slice_h[b * wr.W + a])
              return fail(ctx, NEGF_E_INVALID,
                          "wire %d: slice_h[%d][%d] not finite or not symmetric", w, a, b);
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
      if (!isfinite(E[k]) || !isfinite(wE[k]))
        return fail(ctx, NEGF_E_INVALID, "wire %d: energy %d not finite", w, k);
      // (the levels of a slice block are known on the device only: there the lead-mode kernel
      // reports an energy on a band edge as NEGF_E_INVALID)
      if (wr.lead_model == NEGF_LEAD_STRIP && !wr.slice_h && band_edge(E[k], wr.W, wr.t))
        return fail(ctx, NEGF_E_INVALID, "wire %d: energy %.17g lies on a lead band edge", w, E[k]);
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
      d.layout = layout;
      d.fused = tc_wire ? 1 : 0;
      d.cta_chain = (fp32 && (wr.W == 64 || (wr.W > 16 && wr.W <= 32)) && !tc_wire) ? 1 : 0;
      d.slice_h = wr.slice_h ? 1 : 0;
      // W = 64 two-level tables on the CTA chain, no weights kept: the chain writes level 2
      d.l2_fused = (fuse_l2 && d.cta_chain && wr.W == 64 && layout == NEGF_LAYOUT_TWO_LEVEL) ? 1 : 0;
      if (layout == NEGF_LAYOUT_TWO_LEVEL) tab_off = (tab_off + 3) & ~3ull;   // level 2: 32-byte aligned
      d.tab_off = tab_off;
      d.wt_off = wt_off;
      if (tc_wire) {
        d.edge_off = edge_off;
        edge_off += (uint64_t)(wr.L + 2) * 2 * wr.W * wr.W;
      }
      if (layout == NEGF_LAYOUT_TWO_LEVEL) {
        const uint64_t l2_u64 = (uint64_t)rows * wr.L * negf::level2_words(wr.W) / 2;
        d.l1_off = tab_off + l2_u64;
        d.l1w_off = l1w_rel;               // rebased past the weights below
        l1w_rel += (uint64_t)rows * (wr.L + 2);
        tab_off += l2_u64 + (uint64_t)rows * (wr.L + 2);
        P.max_KA = std::max(P.max_KA, wr.L + 2);
        P.any_two = true;
      } else {
        tab_off += (uint64_t)rows * K;
        P.max_KA = std::max(P.max_KA, (int)K);
      }
      if (!d.l2_fused) wt_off += (uint64_t)rows * K;
      d.g_off = g_off;
      d.mode_off = mode_off;
      d.lead_off = lead_off;
      d.onsite_off = (uint32_t)wire_off;
      d.row_base = row_base;
      d.col_base = col_base;
      d.phi_off = phi_off;
      d.start_off = start_off;
      d.green_off = green_off;
      d.gphi_off = gphi_off;
      P.tasks.push_back(d);
      green_off += (uint64_t)n * n;
      gphi_off += (uint64_t)n * 2 * wr.W;
      g_off += (uint64_t)wr.L * wr.W * wr.W;
      mode_off += 2 * wr.W;
      lead_off += wr.W;
      row_base += (uint32_t)(rows + 2);
      col_base += (uint32_t)(wr.L + 2);
      start_off += (uint64_t)(wr.L + 2) * wr.W * wr.W;
      P.max_W = std::max(P.max_W, wr.W);
      P.max_L = std::max(P.max_L, wr.L);
      P.max_K = std::max(P.max_K, (int)K);
    }
    // onsite, eta, then (multi-orbital slices) the block h and its eigenvalues: W (W + 1) is
    // even, so onsite_off / 2 still indexes each wire's own FP32 copy of eta
    wire_off += 2 * (uint64_t)n + (wr.slice_h ? (uint64_t)wr.W * (wr.W + 1) : 0);
    phi_off += (uint32_t)(wr.W * wr.W);
    P.wire_task0.push_back((int32_t)P.tasks.size());
    if (wr.slice_h) P.any_slice_h = true;
  }
  for (TaskDesc& d : P.tasks)
    if (d.layout == NEGF_LAYOUT_TWO_LEVEL) d.l1w_off += wt_off;
  P.wt_total = wt_off;
  P.l1w_total = l1w_rel;
  P.edge_total = edge_off;
  P.wire_total = wire_off;
  P.tab_total = tab_off;
  P.g_total = g_off;
  P.green_total = green_off;
  P.gphi_total = gphi_off;
  P.lead_total = lead_off;
  P.mode_total = mode_off;
  P.phi_total = phi_off;
  return NEGF_OK;
}

// A contiguous range of tasks built on its own: descriptors rebased to the range's buffers
// (tables, weights, RGF and start blocks, row sums); lead, mode, wire and phi offsets stay global.
struct Wave {
  int t0 = 0, t1 = 0;
  uint64_t tab = 0, g = 0, start = 0, green = 0, gphi = 0;
  uint64_t wt = 0, l1w = 0;          // weights and level-1 weights (elements)
  uint64_t edge = 0;                 // edge blocks of fused tasks (complex64)
  uint32_t rows = 0, cols = 0;
  bool any_two = false;
  std::vector<TaskDesc> desc;
  std::vector<TaskDesc> adesc;       // alias_descs(desc)
  std::vector<TcJob> tcjobs;         // tensor-core chain jobs (task = index into desc), then
  size_t n_tc = 0;                   // the CTA-chain jobs: tcjobs[n_tc ..], those of W = 64
  size_t n_cta_wide = 0;             // tasks first
  int cols_max_W = 0;                // widest task of the warp-per-column chains
  int two_max_W = 0;                 // widest task with two-level tables
  bool any_two_split = false;        // two-level tasks whose level 2 comes from stored weights
  uint32_t cta_narrow() const { return (uint32_t)(tcjobs.size() - n_tc - n_cta_wide); }
};

using negf::add_tc_jobs;

Wave make_wave(const Plan& P, int t0, int t1) {
  Wave w;
  std::vector<TcJob> cta, cta_n;
  w.t0 = t0;
  w.t1 = t1;
  for (int k = t0; k < t1; ++k) {
    TaskDesc d = P.tasks[k];
    const uint64_t l2_u64 = (uint64_t)d.rows * d.L * negf::level2_words(d.W) / 2;
    const uint64_t sz = d.layout == NEGF_LAYOUT_TWO_LEVEL
                            ? l2_u64 + (uint64_t)d.rows * (d.L + 2)
                            : (uint64_t)d.rows * d.K;
    if (d.layout == NEGF_LAYOUT_TWO_LEVEL) w.tab = (w.tab + 3) & ~3ull;   // 32-byte aligned
    d.tab_off = w.tab;
    d.wt_off = w.wt;
    if (!d.l2_fused) w.wt += (uint64_t)d.rows * d.K;   // fused: no rows x K weights stored
    if (d.fused) {
      d.edge_off = w.edge;
      w.edge += (uint64_t)(d.L + 2) * 2 * d.W * d.W;
      add_tc_jobs(w.tcjobs, k - t0, d.L);
    }
    if (d.cta_chain) {
      if (d.W == 64) negf::add_sym_jobs(cta, k - t0, d.L);
      else add_tc_jobs(cta_n, k - t0, d.L);
    }
    if (!d.cta_chain && !d.fused) w.cols_max_W = std::max(w.cols_max_W, d.W);
    if (d.layout == NEGF_LAYOUT_TWO_LEVEL) {
      d.l1_off = w.tab + l2_u64;
      d.l1w_off = w.l1w;                 // rebased past the wave's weights below
      w.l1w += (uint64_t)d.rows * (d.L + 2);
      w.any_two = true;
      w.two_max_W = std::max(w.two_max_W, d.W);
      if (!d.l2_fused) w.any_two_split = true;
    }
    d.start_off = w.start;
    d.row_base = w.rows;
    d.col_base = w.cols;          // g_off stays global: the sweeps run once for the batch
    d.green_off = w.green;
    d.gphi_off = w.gphi;
    w.green += (uint64_t)d.n * d.n;
    w.gphi += (uint64_t)d.n * 2 * d.W;
    w.tab += sz;
    w.g += (uint64_t)d.L * d.W * d.W;
    w.start += (uint64_t)(d.L + 2) * d.W * d.W;
    w.rows += (uint32_t)(d.rows + 2);
    w.cols += (uint32_t)(d.L + 2);
    w.desc.push_back(d);
  }
  for (TaskDesc& d : w.desc)
    if (d.layout == NEGF_LAYOUT_TWO_LEVEL) d.l1w_off += w.wt;
  w.adesc = alias_descs(w.desc);
  negf::sort_jobs_longest_first(w.tcjobs, w.desc.data());
  negf::sort_jobs_longest_first(cta, w.desc.data());
  negf::sort_jobs_longest_first(cta_n, w.desc.data());
  w.n_tc = w.tcjobs.size();
  w.n_cta_wide = cta.size();
  w.tcjobs.insert(w.tcjobs.end(), cta.begin(), cta.end());
  w.tcjobs.insert(w.tcjobs.end(), cta_n.begin(), cta_n.end());
  return w;
}

// device bytes a wave needs while it is built (tables + every scratch buffer)
uint64_t wave_bytes(const Wave& w, int prec) {
  const uint64_t cb = negf::block_bytes(prec);
  const uint64_t wsz = prec == NEGF_FP64 ? 8 : 4;
  return w.tab * 8 + (w.wt + w.l1w) * wsz + w.start * cb + 8ull * w.rows + 8ull * w.edge;
}

// Buffers shared by every wave of a batch.
struct Persist {
  TaskDesc* d_tasks = nullptr;       // global descriptors (current assembly)
  int32_t* d_wire_task0 = nullptr;
  double* d_wire = nullptr;
  cd* d_sig = nullptr;
  double* d_gam = nullptr;
  double* d_phi = nullptr;           // FP64 modes, then their FP32 copy
  float* d_eta32 = nullptr;
  uint64_t* d_mode_tab = nullptr;
  double* d_mode_w = nullptr;
  double* d_c = nullptr;
  int32_t* d_err = nullptr;
};

void free_persist_scratch(Persist& q, cudaStream_t s) {
  dfree(q.d_phi, s);
  dfree(q.d_eta32, s);
}

// Allocate and fill the shared buffers, then run validation (device inputs) and the lead
// kernel for every task.  Records the allocated bytes in *bytes.
negf_status setup_batch(negf_ctx ctx, cudaStream_t s, const negf_wire* wires, int n_wires,
                        bool dev_in, const Plan& P, Persist& q, uint64_t* bytes) {
  const int nt = (int)P.tasks.size();
#define PALLOC(ptr, count)                                                                   \
  do {                                                                                       \
    cudaError_t e_ = dalloc(&(ptr), (count), s, bytes);                                      \
    if (e_ != cudaSuccess)                                                                   \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,         \
                  "allocation of %s (%zu elements): %s", #ptr, (size_t)(count),              \
                  cudaGetErrorString(e_));                                                   \
  } while (0)
  PALLOC(q.d_tasks, nt);
  PALLOC(q.d_wire_task0, n_wires + 1);
  PALLOC(q.d_wire, P.wire_total);
  PALLOC(q.d_sig, P.lead_total);
  PALLOC(q.d_gam, P.lead_total);
  PALLOC(q.d_phi, (uint64_t)P.phi_total + (P.phi_total + 1) / 2);
  PALLOC(q.d_eta32, P.wire_total / 2);
  PALLOC(q.d_mode_tab, P.mode_total);
  PALLOC(q.d_mode_w, P.mode_total);
  PALLOC(q.d_c, 2 * (size_t)nt);
  PALLOC(q.d_err, 1);
#undef PALLOC
  CUDA_TRY(ctx, cudaMemsetAsync(q.d_err, 0, sizeof(int32_t), s));
  if (nt > 0)
    CUDA_TRY(ctx, cudaMemcpyAsync(q.d_tasks, P.tasks.data(), sizeof(TaskDesc) * nt,
                                  cudaMemcpyHostToDevice, s));
  CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire_task0, P.wire_task0.data(),
                                sizeof(int32_t) * (n_wires + 1), cudaMemcpyHostToDevice, s));
  std::vector<double> stage;
  uint64_t off = 0;
  for (int w = 0; w < n_wires; ++w) {
    const int64_t n = (int64_t)wires[w].W * wires[w].L;
    const int64_t hw = wires[w].slice_h ? (int64_t)wires[w].W * wires[w].W : 0;
    if (dev_in) {
      CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire + off, wires[w].onsite, sizeof(double) * n,
                                    cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire + off + n, wires[w].eta, sizeof(double) * n,
                                    cudaMemcpyDeviceToDevice, s));
      if (hw)
        CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire + off + 2 * n, wires[w].slice_h,
                                      sizeof(double) * hw, cudaMemcpyDeviceToDevice, s));
    } else {
      stage.insert(stage.end(), wires[w].onsite, wires[w].onsite + n);
      stage.insert(stage.end(), wires[w].eta, wires[w].eta + n);
      if (hw) {
        stage.insert(stage.end(), wires[w].slice_h, wires[w].slice_h + hw);
        stage.insert(stage.end(), (size_t)wires[w].W, 0.0);      // eigenvalues, set on device
      }
    }
    off += 2 * n + (hw ? hw + wires[w].W : 0);
  }
  if (!dev_in && off > 0) {
    CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire, stage.data(), sizeof(double) * off,
                                  cudaMemcpyHostToDevice, s));
    CUDA_TRY(ctx, cudaStreamSynchronize(s));   // the staging vector dies here
  }
  if (nt > 0) {
    if (dev_in) {
      ProfScope ps(ctx, "validate_kernel", 2, s);
      CUDA_TRY(ctx, negf::launch_validate(q.d_tasks, nt, q.d_wire, q.d_err, s));
    }
    if (P.any_slice_h) {
      ProfScope ps(ctx, "slice_modes_kernel", 1, s);
      CUDA_TRY(ctx, negf::launch_slice_modes(q.d_tasks, nt, P.max_W, q.d_wire, q.d_phi,
                                             reinterpret_cast<float*>(q.d_phi + P.phi_total),
                                             q.d_err, s));
    }
    ProfScope ps(ctx, "lead_modes_kernel", 1, s);
    CUDA_TRY(ctx, negf::launch_lead_modes(q.d_tasks, nt, P.max_W, q.d_wire, q.d_phi,
                                          reinterpret_cast<float*>(q.d_phi + P.phi_total),
                                          q.d_eta32, q.d_sig, q.d_gam, q.d_err, s));
  }
  return NEGF_OK;
}

// RGF sweeps of every task of the batch (one launch: the sweep is a sequential chain per task,
// so its latency is paid once) into gL / gR at the tasks' global offsets.
negf_status sweep_all(negf_ctx ctx, cudaStream_t s, const Plan& P, const Persist& q, int prec,
                      void* d_gL, void* d_gR) {
  const int nt = (int)P.tasks.size();
  if (nt == 0) return NEGF_OK;
  ProfScope ps(ctx, "rgf_sweep_kernel", 1, s);
  CUDA_TRY(ctx, negf::launch_rgf_sweep(q.d_tasks, nt, P.max_W, prec, q.d_wire, q.d_phi, q.d_sig,
                                       d_gL, d_gR, q.d_err, s));
  return NEGF_OK;
}

// Enqueue the rest of the build of one wave on stream s (the sweeps are done): diagonal blocks
// + chains (weights), alias tables into d_tab.  Scratch is allocated and freed on s; the
// weights go to *weights_out when it is non-null (kept), else they are freed too.  Row sums go
// to d_rowsum.
negf_status build_wave(negf_ctx ctx, cudaStream_t s, const Plan& P, const Wave& w,
                       TaskDesc* d_wdesc, TaskDesc* d_adesc, const Persist& q, int prec,
                       const void* d_gL,
                       const void* d_gR, uint64_t* d_tab, double* d_rowsum, void** weights_out,
                       void* d_green = nullptr, void* d_gphi = nullptr,
                       double* pre_start = nullptr, void* pre_weights = nullptr,
                       int chain_warps = 0, int alias_warps = 0,
                       const TcJob* d_tcjobs = nullptr, void* pre_edge = nullptr) {
  const int nt = w.t1 - w.t0;
  if (nt == 0) return NEGF_OK;
  const uint64_t cw = negf::block_bytes(prec) / sizeof(double);
  const size_t wsz = prec == NEGF_FP64 ? sizeof(double) : sizeof(float);
  // scratch: the caller's buffers when given (captured plans), else allocated on s
  const bool own = pre_start == nullptr;
  double* d_start = pre_start;
  void* d_weights = pre_weights;
  void* d_edge = pre_edge;
  cudaError_t e = cudaSuccess;
  if (own) {
    e = dalloc(&d_start, w.start * cw, s, nullptr);
    if (e == cudaSuccess)
      e = cudaMallocAsync(&d_weights, std::max<uint64_t>(w.wt + w.l1w, 1) * wsz, s);
    if (e == cudaSuccess && w.edge) e = cudaMallocAsync(&d_edge, w.edge * sizeof(negf::cf), s);
  }
  auto cleanup = [&]() {
    if (!own) return;
    dfree(d_start, s);
    if (d_weights) cudaFreeAsync(d_weights, s);
    if (d_edge) cudaFreeAsync(d_edge, s);
    d_weights = nullptr;
    d_edge = nullptr;
  };
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, e == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                "build scratch allocation: %s", cudaGetErrorString(e));
  }
  {
    ProfScope ps(ctx, "diag_chain_kernels", 2, s);
    e = negf::launch_block_columns(d_wdesc, nt, w.cols, P.max_W, prec, q.d_wire, q.d_eta32,
                                   q.d_phi, reinterpret_cast<float*>(q.d_phi + P.phi_total),
                                   q.d_sig, q.d_gam, d_gL, d_gR, d_start, d_weights, d_rowsum,
                                   q.d_mode_w, q.d_c + 2 * (size_t)w.t0, q.d_err, d_green,
                                   d_gphi, s, chain_warps, w.cols_max_W);
  }
  if (e == cudaSuccess && w.tcjobs.size() > w.n_tc) {
    ProfScope ps(ctx, "chain_cta_kernel", 1, s);
    e = negf::launch_chain_cta(d_wdesc, d_tcjobs + w.n_tc, (uint32_t)w.n_cta_wide,
                               w.cta_narrow(), q.d_eta32, reinterpret_cast<const float*>(q.d_phi + P.phi_total),
                               q.d_gam, d_gL, d_gR, d_start, d_weights, d_tab, q.d_err, s);
  }
  if (e == cudaSuccess && w.n_tc) {
    ProfScope ps(ctx, "chain_tc_kernel", 2, s);
    e = negf::launch_chain_tc(d_wdesc, nt, w.cols, d_tcjobs, (uint32_t)w.n_tc,
                              q.d_eta32, reinterpret_cast<const float*>(q.d_phi + P.phi_total),
                              q.d_gam, d_gL, d_gR, d_start, d_weights, d_tab, d_edge, q.d_err, s);
  }
  if (e == cudaSuccess && w.any_two_split) {
    ProfScope ps(ctx, "two_level_kernel", 1, s);
    e = negf::launch_two_level_split(d_wdesc, nt, w.rows, prec, d_weights, d_tab, q.d_err, s,
                                     w.two_max_W);
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "alias_kernel", 1, s);
    e = negf::launch_alias_build(d_adesc, nt, w.rows, P.max_KA, prec, d_weights, d_rowsum,
                                 q.d_mode_w, d_tab, q.d_mode_tab, q.d_err, s, alias_warps);
  }
  if (e != cudaSuccess) {
    cleanup();
    return fail(ctx, NEGF_E_CUDA, "table build: %s", cudaGetErrorString(e));
  }
  if (weights_out && own) {
    *weights_out = d_weights;
    d_weights = nullptr;
  }
  cleanup();
  return NEGF_OK;
}

void adopt_persist(negf_tables t, const Persist& q) {
  t->d_tasks = q.d_tasks;
  t->d_wire_task0 = q.d_wire_task0;
  t->d_wire = q.d_wire;
  t->d_sig = q.d_sig;
  t->d_gam = q.d_gam;
  t->d_mode_tab = q.d_mode_tab;
  t->d_mode_w = q.d_mode_w;
  t->d_c = q.d_c;
  t->d_err = q.d_err;
}

negf_status check_opts(negf_ctx ctx, const negf_build_opts* opts, negf_build_opts& o) {
  o = negf_build_opts{NEGF_FP64, NEGF_MEM_HOST, 0, 0, NEGF_LAYOUT_AUTO};
  if (opts) o = *opts;
  if (o.precision < NEGF_FP64 || o.precision > NEGF_SPLIT_TF32)
    return fail(ctx, NEGF_E_INVALID, "unknown precision %d", o.precision);
  if (o.memspace != NEGF_MEM_HOST && o.memspace != NEGF_MEM_DEVICE)
    return fail(ctx, NEGF_E_INVALID, "unknown memspace %d", o.memspace);
  if (o.keep_green < 0) return fail(ctx, NEGF_E_INVALID, "build opts: keep_green < 0");
  return NEGF_OK;
}

}  // namespace

extern "C" {

negf_status negf_build_tables(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                              const negf_build_opts* opts, negf_tables* out) {
  if (!ctx) return NEGF_E_INVALID;
  if (!out) return fail(ctx, NEGF_E_INVALID, "negf_build_tables: out is NULL");
  *out = nullptr;
  if (n_wires < 0 || (n_wires > 0 && !wires))
    return fail(ctx, NEGF_E_INVALID, "negf_build_tables: bad wire list");
  negf_build_opts o;
  negf_status st = check_opts(ctx, opts, o);
  if (st != NEGF_OK) return st;
  const bool dev_in = o.memspace == NEGF_MEM_DEVICE;
  const int prec = o.precision == NEGF_FP64 ? NEGF_FP64 : NEGF_FP32;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;
  Plan P;
  // the gradient needs G itself, which only the warp-per-column chain keeps
  st = make_plan(ctx, wires, n_wires, dev_in, P, o.table_layout, o.precision == NEGF_SPLIT_TF32,
                 o.precision != NEGF_FP64 && !o.keep_green, o.keep_green != 0,
                 !o.keep_weights && !o.keep_green);
  if (st != NEGF_OK) return st;
  if (o.keep_green && P.any_two)
    return fail(ctx, NEGF_E_INVALID, "keep_green needs one-level tables (the gradient keeps dense G)");
  negf_tables t = new (std::nothrow) negf_tables_s;
  if (!t) return fail(ctx, NEGF_E_NOMEM, "negf_build_tables: host allocation");
  t->ctx = ctx;
  t->n_wires = n_wires;
  t->precision = prec;
  t->h_tasks = P.tasks;
  t->h_wire_task0 = P.wire_task0;
  t->n_tasks = (int)P.tasks.size();
  t->max_W = P.max_W;
  t->max_L = P.max_L;
  t->max_K = P.max_K;
  Persist q;
  st = setup_batch(ctx, s, wires, n_wires, dev_in, P, q, &t->bytes);
  adopt_persist(t, q);
  if (st != NEGF_OK) {
    free_persist_scratch(q, s);
    release_tables(t);
    return st;
  }
  // one wave holding every task: its rebased descriptors equal the global ones
  const Wave w = make_wave(P, 0, t->n_tasks);
  t->total_jobs = w.rows;
  t->any_two = P.any_two;
  TaskDesc* d_adesc = nullptr;
  TcJob* d_tcjobs = nullptr;
  cudaError_t e = dalloc(&t->d_tab, w.tab, s, &t->bytes);
  if (e == cudaSuccess) e = dalloc(&t->d_rowsum, w.rows, s, &t->bytes);
  if (e == cudaSuccess && !w.adesc.empty()) e = dalloc(&d_adesc, w.adesc.size(), s, nullptr);
  if (e == cudaSuccess && !w.adesc.empty())
    e = cudaMemcpyAsync(d_adesc, w.adesc.data(), sizeof(TaskDesc) * w.adesc.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !w.tcjobs.empty()) e = dalloc(&d_tcjobs, w.tcjobs.size(), s, nullptr);
  if (e == cudaSuccess && !w.tcjobs.empty())
    e = cudaMemcpyAsync(d_tcjobs, w.tcjobs.data(), sizeof(TcJob) * w.tcjobs.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !w.adesc.empty()) e = cudaStreamSynchronize(s);   // host copy sources
  if (e != cudaSuccess) {
    dfree(d_adesc, s);
    dfree(d_tcjobs, s);
    free_persist_scratch(q, s);
    release_tables(t);
    return fail(ctx, e == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                "table allocation: %s", cudaGetErrorString(e));
  }
  void* kept = nullptr;
  t->score_stride = w.wt;         // score tallies and seeds share the weights' rows x K layout
  t->mode_stride = P.mode_total;
  if (o.keep_green) {
    const uint64_t cb = negf::block_bytes(prec);
    e = cudaMallocAsync(&t->d_green, std::max<uint64_t>(w.green, 1) * cb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&t->d_gphi, std::max<uint64_t>(w.gphi, 1) * cb, s);
    if (e != cudaSuccess) {
      dfree(d_adesc, s);
      dfree(d_tcjobs, s);
      free_persist_scratch(q, s);
      release_tables(t);
      return fail(ctx, e == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                  "allocation of the kept Green's functions: %s", cudaGetErrorString(e));
    }
    t->green_total = w.green;
    t->gphi_total = w.gphi;
    t->bytes += (w.green + w.gphi) * cb;
  }
  void* d_gL = nullptr;
  void* d_gR = nullptr;
  {
    const uint64_t gb = std::max<uint64_t>(P.g_total, 1) * negf::block_bytes(prec);
    e = cudaMallocAsync(&d_gL, gb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_gR, gb, s);
  }
  if (e != cudaSuccess) st = fail(ctx, NEGF_E_NOMEM, "RGF scratch: %s", cudaGetErrorString(e));
  if (st == NEGF_OK) st = sweep_all(ctx, s, P, q, prec, d_gL, d_gR);
  if (st == NEGF_OK)
    st = build_wave(ctx, s, P, w, t->d_tasks, d_adesc, q, prec, d_gL, d_gR, t->d_tab,
                    t->d_rowsum, (o.keep_weights || o.keep_green) ? &kept : nullptr, t->d_green,
                    t->d_gphi, nullptr, nullptr, 0, 0, d_tcjobs);
  dfree(d_adesc, s);
  dfree(d_tcjobs, s);
  if (d_gL) cudaFreeAsync(d_gL, s);
  if (d_gR) cudaFreeAsync(d_gR, s);
  if (o.keep_green || o.keep_weights) {
    t->d_phi = q.d_phi;          // the gradient needs the transverse modes
    q.d_phi = nullptr;
  }
  free_persist_scratch(q, s);
  if (st != NEGF_OK) {
    release_tables(t);
    return st;
  }
  if (kept) {
    t->d_weights = kept;
    t->bytes += std::max<uint64_t>(w.wt + w.l1w, 1) * (prec == NEGF_FP64 ? 8 : 4);
  }
  *out = t;
  return NEGF_OK;
}

negf_status negf_run(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                     const negf_build_opts* bopts, const negf_run_opts* ropts,
                     negf_tables* out_tasks, negf_tally* out_tally) {
  if (!ctx) return NEGF_E_INVALID;
  if (!out_tasks || !out_tally || !ropts)
    return fail(ctx, NEGF_E_INVALID, "negf_run: NULL output or options");
  *out_tasks = nullptr;
  *out_tally = nullptr;
  if (n_wires < 0 || (n_wires > 0 && !wires))
    return fail(ctx, NEGF_E_INVALID, "negf_run: bad wire list");
  negf_build_opts o;
  negf_status st = check_opts(ctx, bopts, o);
  if (st != NEGF_OK) return st;
  if (o.keep_weights) return fail(ctx, NEGF_E_INVALID, "negf_run releases tables; keep_weights must be 0");
  const negf_run_opts& r = *ropts;
  if (r.start_lead != 0 && r.start_lead != 1)
    return fail(ctx, NEGF_E_INVALID, "negf_run: start_lead must be 0 or 1");
  if (r.max_steps < 1 || r.max_steps > NEGF_MAX_STEPS)
    return fail(ctx, NEGF_E_INVALID, "negf_run: max_steps must be in [1, %u]", NEGF_MAX_STEPS);
  if (r.walkers_per_task > (1ull << 40) || r.tasks_per_wave < 0 || r.waves_in_flight < 0 ||
      r.walk_blocks_per_sm < 0 || r.reserved != 0)
    return fail(ctx, NEGF_E_INVALID, "negf_run: bad walker count, wave size, depth or reserved");
  const bool dev_in = o.memspace == NEGF_MEM_DEVICE;
  const int prec = o.precision == NEGF_FP64 ? NEGF_FP64 : NEGF_FP32;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;
  if (!ctx->walk_stream &&
      cudaStreamCreateWithFlags(&ctx->walk_stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(ctx, NEGF_E_CUDA, "negf_run: stream creation failed");
  cudaStream_t sw = ctx->walk_stream;
  Plan P;
  st = make_plan(ctx, wires, n_wires, dev_in, P, o.table_layout, o.precision == NEGF_SPLIT_TF32,
                 o.precision != NEGF_FP64, false, true);
  if (st != NEGF_OK) return st;
  const int nt = (int)P.tasks.size();
  negf_tables t = new (std::nothrow) negf_tables_s;
  negf_tally tl = new (std::nothrow) negf_tally_s;
  if (!t || !tl) {
    delete t;
    delete tl;
    return fail(ctx, NEGF_E_NOMEM, "negf_run: host allocation");
  }
  t->ctx = ctx;
  t->n_wires = n_wires;
  t->precision = prec;
  t->h_tasks = P.tasks;
  t->h_wire_task0 = P.wire_task0;
  t->n_tasks = nt;
  t->max_W = P.max_W;
  t->max_L = P.max_L;
  t->max_K = P.max_K;
  t->tables_released = true;
  t->any_two = P.any_two;
  tl->ctx = ctx;
  tl->n_tasks = nt;
  tl->start_lead = r.start_lead;
  Persist q;
  st = setup_batch(ctx, s, wires, n_wires, dev_in, P, q, &t->bytes);
  adopt_persist(t, q);
  cudaError_t e = cudaSuccess;
  if (st == NEGF_OK) {
    e = dalloc(&tl->d_counts, (size_t)std::max(1, nt) * NEGF_TALLY_FIELDS, s, nullptr);
    if (e == cudaSuccess)
      e = cudaMemsetAsync(tl->d_counts, 0,
                          sizeof(uint64_t) * (size_t)std::max(1, nt) * NEGF_TALLY_FIELDS, s);
    if (e != cudaSuccess) st = fail(ctx, NEGF_E_CUDA, "negf_run: tally: %s", cudaGetErrorString(e));
  }
  // ---- waves: consecutive tasks whose tables and scratch fit the budget (depth waves in flight)
  const int depth = r.waves_in_flight > 0 ? r.waves_in_flight : 2;
  uint64_t budget = r.memory_budget;
  if (budget == 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    budget = free_b / 2;
  }
  const int per_wave = r.tasks_per_wave > 0 ? r.tasks_per_wave : std::max(1, (nt + 7) / 8);
  std::vector<uint64_t> task_bytes(nt);
  for (int k = 0; k < nt; ++k) task_bytes[k] = wave_bytes(make_wave(P, k, k + 1), prec);
  std::vector<Wave> waves;
  for (int k = 0; k < nt && st == NEGF_OK;) {
    int k1 = k + 1;
    uint64_t bytes_w = task_bytes[k];
    while (k1 < nt && k1 - k < per_wave && (bytes_w + task_bytes[k1]) * depth <= budget)
      bytes_w += task_bytes[k1++];
    waves.push_back(make_wave(P, k, k1));
    k = k1;
  }
  TaskDesc* d_wdesc = nullptr;
  TaskDesc* d_adesc = nullptr;
  TcJob* d_tcjobs = nullptr;
  std::vector<size_t> job_off;
  if (st == NEGF_OK && nt > 0) {
    std::vector<TaskDesc> all, alla;
    std::vector<TcJob> jobs;
    for (const Wave& w : waves) {
      all.insert(all.end(), w.desc.begin(), w.desc.end());
      alla.insert(alla.end(), w.adesc.begin(), w.adesc.end());
      job_off.push_back(jobs.size());
      jobs.insert(jobs.end(), w.tcjobs.begin(), w.tcjobs.end());
    }
    e = dalloc(&d_wdesc, all.size(), s, nullptr);
    if (e == cudaSuccess) e = dalloc(&d_adesc, alla.size(), s, nullptr);
    if (e == cudaSuccess && !jobs.empty()) e = dalloc(&d_tcjobs, jobs.size(), s, nullptr);
    if (e == cudaSuccess && !jobs.empty())
      e = cudaMemcpyAsync(d_tcjobs, jobs.data(), sizeof(TcJob) * jobs.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_wdesc, all.data(), sizeof(TaskDesc) * all.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_adesc, alla.data(), sizeof(TaskDesc) * alla.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // `all` dies here
    if (e != cudaSuccess) st = fail(ctx, NEGF_E_CUDA, "negf_run: descriptors: %s", cudaGetErrorString(e));
  }
  // ---- RGF sweeps of every task, once
  void* d_gL = nullptr;
  void* d_gR = nullptr;
  if (st == NEGF_OK && nt > 0) {
    const uint64_t gb = std::max<uint64_t>(P.g_total, 1) * negf::block_bytes(prec);
    e = cudaMallocAsync(&d_gL, gb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&d_gR, gb, s);
    if (e != cudaSuccess) st = fail(ctx, NEGF_E_NOMEM, "negf_run: RGF scratch: %s", cudaGetErrorString(e));
    if (st == NEGF_OK) st = sweep_all(ctx, s, P, q, prec, d_gL, d_gR);
  }
  // ---- pipeline: build wave w on the context stream while wave w-1 walks on the second one
  std::vector<cudaEvent_t> built(waves.size(), nullptr), walked(waves.size(), nullptr);
  for (size_t w = 0; w < waves.size() && st == NEGF_OK; ++w) {
    const Wave& wv = waves[w];
    if (cudaEventCreateWithFlags(&built[w], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&walked[w], cudaEventDisableTiming) != cudaSuccess) {
      st = fail(ctx, NEGF_E_CUDA, "negf_run: event creation failed");
      break;
    }
    if (w >= (size_t)depth) cudaStreamWaitEvent(s, walked[w - depth], 0);
    uint64_t* d_tab = nullptr;
    double* d_rs = nullptr;
    e = dalloc(&d_tab, wv.tab, s, nullptr);
    if (e == cudaSuccess) e = dalloc(&d_rs, wv.rows, s, nullptr);
    if (e != cudaSuccess) {
      dfree(d_tab, s);
      dfree(d_rs, s);
      st = fail(ctx, e == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                "negf_run: wave %zu tables: %s", w, cudaGetErrorString(e));
      break;
    }
    size_t off = 0;
    for (size_t v = 0; v < w; ++v) off += waves[v].desc.size();
    st = build_wave(ctx, s, P, wv, d_wdesc + off, d_adesc + off, q, prec, d_gL, d_gR, d_tab, d_rs,
                    nullptr, nullptr, nullptr, nullptr, nullptr, 0, 0,
                    d_tcjobs ? d_tcjobs + job_off[w] : nullptr);
    dfree(d_rs, s);
    if (st != NEGF_OK) {
      dfree(d_tab, s);
      break;
    }
    cudaEventRecord(built[w], s);
    cudaStreamWaitEvent(sw, built[w], 0);
    {
      ProfScope ps(ctx, "walk_kernel", (uint64_t)(wv.t1 - wv.t0 + 1023) / 1024, sw);
      e = negf::launch_walk(d_wdesc + off, 0, wv.t1 - wv.t0, (uint32_t)wv.t0, d_tab,
                            q.d_mode_tab, q.d_c + 2 * (size_t)wv.t0, r.start_lead, r.seed,
                            r.walkers_per_task, r.walker_id_offset, r.max_steps, ctx->d_counter,
                            tl->d_counts + (size_t)wv.t0 * NEGF_TALLY_FIELDS, nullptr, nullptr,
                            nullptr, 0, nullptr, 0, ctx->sm_count, r.walk_blocks_per_sm, sw,
                            nullptr, walk_slots(wv.any_two), wv.any_two);
    }
    cudaFreeAsync(d_tab, sw);
    cudaEventRecord(walked[w], sw);
    if (e != cudaSuccess) st = fail(ctx, NEGF_E_CUDA, "negf_run: walk: %s", cudaGetErrorString(e));
  }
  // ---- join: the context stream waits for the last walk
  if (!waves.empty() && walked.back()) cudaStreamWaitEvent(s, walked.back(), 0);
  else {
    cudaEvent_t j = nullptr;
    if (cudaEventCreateWithFlags(&j, cudaEventDisableTiming) == cudaSuccess) {
      cudaEventRecord(j, sw);
      cudaStreamWaitEvent(s, j, 0);
      cudaEventDestroy(j);
    }
  }
  for (size_t w = 0; w < waves.size(); ++w) {
    if (built[w]) cudaEventDestroy(built[w]);
    if (walked[w]) cudaEventDestroy(walked[w]);
  }
  dfree(d_wdesc, s);
  dfree(d_adesc, s);
  dfree(d_tcjobs, s);
  if (d_gL) cudaFreeAsync(d_gL, s);
  if (d_gR) cudaFreeAsync(d_gR, s);
  free_persist_scratch(q, s);
  if (st != NEGF_OK) {
    if (tl->d_counts) cudaFreeAsync(tl->d_counts, s);
    delete tl;
    release_tables(t);
    return st;
  }
  t->n_waves = (int)waves.size();
  *out_tasks = t;
  *out_tally = tl;
  return NEGF_OK;
}

int32_t negf_tables_num_waves(negf_tables t) { return t ? t->n_waves : 0; }

negf_status negf_probe_gather(negf_ctx ctx, uint64_t table_bytes, int32_t ilp, int32_t chain,
                              double* gathers_per_s) {
  if (!ctx || !gathers_per_s) return NEGF_E_INVALID;
  DeviceGuard g(ctx->device);
  uint64_t n = 0;
  float ms = 0.f;
  cudaError_t e = negf::probe_gather(table_bytes, ilp, chain, ctx->sm_count, &n, &ms, ctx->stream);
  if (e == cudaErrorInvalidValue)
    return fail(ctx, NEGF_E_INVALID, "negf_probe_gather: table must hold 2 .. 2^32 entries");
  if (e != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "negf_probe_gather: %s", cudaGetErrorString(e));
  *gathers_per_s = ms > 0.f ? (double)n / (ms * 1e-3) : 0.0;
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
  out->table_layout = d.layout;
  out->table_offset = d.wt_off;
  out->mode_offset = d.mode_off;
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
  const bool two = d.layout == NEGF_LAYOUT_TWO_LEVEL;
  switch (what) {
    case NEGF_EXPORT_ALIAS:
      need = two ? sizeof(uint32_t) * (size_t)d.rows * d.L * negf::level2_words(d.W)
                 : sizeof(uint64_t) * (size_t)d.rows * (size_t)d.K;
      break;
    case NEGF_EXPORT_ALIAS_LEVEL1:
      if (!two) return fail(ctx, NEGF_E_INVALID, "task %d has one-level tables", task);
      need = sizeof(uint64_t) * (size_t)d.rows * (d.L + 2);
      break;
    case NEGF_EXPORT_MODE_ALIAS: need = sizeof(uint64_t) * 2 * (size_t)d.W; break;
    case NEGF_EXPORT_WEIGHTS:
      if (!t->d_weights) return fail(ctx, NEGF_E_INVALID, "weights were not kept (keep_weights = 0)");
      need = sizeof(double) * (size_t)d.rows * d.K;
      break;
    case NEGF_EXPORT_MODE_WEIGHTS: need = sizeof(double) * 2 * (size_t)d.W; break;
    case NEGF_EXPORT_ROWSUM: need = sizeof(double) * (size_t)d.rows; break;
    default: return fail(ctx, NEGF_E_INVALID, "unknown export kind %d", what);
  }
  if (t->tables_released && (what == NEGF_EXPORT_ALIAS || what == NEGF_EXPORT_ALIAS_LEVEL1 ||
                             what == NEGF_EXPORT_ROWSUM))
    return fail(ctx, NEGF_E_INVALID, "the alias tables of this handle were released (negf_run)");
  if (!host_buf) { *bytes = need; return NEGF_OK; }
  if (*bytes < need) return fail(ctx, NEGF_E_INVALID, "export buffer too small (%zu < %zu)", *bytes, need);
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  switch (what) {
    case NEGF_EXPORT_ALIAS:
      CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, t->d_tab + d.tab_off, need, cudaMemcpyDeviceToHost, s));
      break;
    case NEGF_EXPORT_ALIAS_LEVEL1:
      CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, t->d_tab + d.l1_off, need, cudaMemcpyDeviceToHost, s));
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

negf_status negf_export_table_rows(negf_ctx ctx, negf_tables t, int32_t task, int32_t what,
                                  int64_t row0, int64_t n_rows, void* host_buf, size_t* bytes) {
  if (!ctx || !t || !bytes || t->ctx != ctx)
    return fail(ctx, NEGF_E_INVALID, "negf_export_table_rows: bad argument");
  if (task < 0 || task >= t->n_tasks) return fail(ctx, NEGF_E_INVALID, "task %d out of range", task);
  const TaskDesc& d = t->h_tasks[task];
  if (row0 < 0 || n_rows < 0 || row0 + n_rows > d.rows)
    return fail(ctx, NEGF_E_INVALID, "rows [%lld, %lld) outside [0, %d)", (long long)row0,
                (long long)(row0 + n_rows), d.rows);
  if (t->tables_released)
    return fail(ctx, NEGF_E_INVALID, "the alias tables of this handle were released (negf_run)");
  const bool two = d.layout == NEGF_LAYOUT_TWO_LEVEL;
  size_t per_row = 0;       // 8-byte elements per row
  uint64_t first = 0;       // first element of row0
  switch (what) {
    case NEGF_EXPORT_ALIAS:
      // two-level: the row's level-2 blocks, L * level2_words(W) u32 (an even count)
      per_row = two ? (size_t)d.L * negf::level2_words(d.W) / 2 : (size_t)d.K;
      first = d.tab_off + (uint64_t)row0 * per_row;
      break;
    case NEGF_EXPORT_ALIAS_LEVEL1:
      if (!two) return fail(ctx, NEGF_E_INVALID, "task %d has one-level tables", task);
      per_row = (size_t)d.L + 2;
      first = d.l1_off + (uint64_t)row0 * per_row;
      break;
    case NEGF_EXPORT_ROWSUM:
      per_row = 1;
      first = d.row_base + (uint64_t)row0;
      break;
    default:
      return fail(ctx, NEGF_E_INVALID, "negf_export_table_rows: kind %d not supported", what);
  }
  const size_t need = sizeof(uint64_t) * per_row * (size_t)n_rows;
  if (!host_buf) { *bytes = need; return NEGF_OK; }
  if (*bytes < need) return fail(ctx, NEGF_E_INVALID, "export buffer too small (%zu < %zu)", *bytes, need);
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  const void* src = what == NEGF_EXPORT_ROWSUM ? static_cast<const void*>(t->d_rowsum + first)
                                               : static_cast<const void*>(t->d_tab + first);
  if (need) CUDA_TRY(ctx, cudaMemcpyAsync(host_buf, src, need, cudaMemcpyDeviceToHost, s));
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
  cudaError_t e = dalloc(&tl->d_counts, (size_t)std::max(1, t->n_tasks) * NEGF_TALLY_FIELDS, ctx->stream, nullptr);
  if (e != cudaSuccess) {
    delete tl;
    return fail(ctx, NEGF_E_NOMEM, "negf_walk: tally allocation: %s", cudaGetErrorString(e));
  }
  e = cudaMemsetAsync(tl->d_counts, 0, sizeof(uint64_t) * std::max(1, t->n_tasks) * NEGF_TALLY_FIELDS,
                      ctx->stream);
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "walk_kernel", (t->n_tasks + 1023) / 1024);
    e = negf::launch_walk(t->d_tasks, 0, t->n_tasks, 0, t->d_tab, t->d_mode_tab, t->d_c,
                          start_lead, seed, walkers_per_task, walker_id_offset, max_steps,
                          ctx->d_counter, tl->d_counts, nullptr, nullptr, nullptr, 0, nullptr,
                          0, ctx->sm_count, 0, ctx->stream, nullptr, walk_slots(t->any_two),
                          t->any_two);
  }
  if (e != cudaSuccess) {
    cudaFreeAsync(tl->d_counts, ctx->stream);
    delete tl;
    return fail(ctx, NEGF_E_CUDA, "negf_walk: %s", cudaGetErrorString(e));
  }
  *out = tl;
  return NEGF_OK;
}

// Step 7' energy rows of every (task, site) of one-level tables (inelastic Buttiker probes):
// descriptors, job bases and the alias rows, on the ctx stream.  d_edesc and d_etab are the
// caller's to free (stream-ordered).
static negf_status energy_tables(negf_ctx ctx, negf_tables t, double sigma, const char* who,
                                 negf::EnergyDesc** d_edesc, uint64_t** d_etab,
                                 std::vector<negf::EnergyDesc>* h_out) {
  *d_edesc = nullptr;
  *d_etab = nullptr;
  if (!(sigma >= 0.0) || !isfinite(sigma))
    return fail(ctx, NEGF_E_INVALID, "%s: sigma_E must be finite and >= 0", who);
  if (t->any_two)
    return fail(ctx, NEGF_E_INVALID, "%s: inelastic walks need one-level tables", who);
  const cudaStream_t s = ctx->stream;
  std::vector<negf::EnergyDesc> ed(std::max(1, t->n_tasks));
  std::vector<uint32_t> jb(std::max(1, t->n_tasks));
  uint64_t eoff = 0, jobs = 0;
  int max_nE = 1;
  for (int w = 0; w < t->n_wires; ++w) {
    const int k0 = t->h_wire_task0[w], k1 = t->h_wire_task0[w + 1];
    for (int k = k0; k < k1; ++k) {
      ed[k].eoff = eoff;
      ed[k].nE = k1 - k0;
      ed[k].t0 = k0;
      jb[k] = (uint32_t)jobs;
      eoff += (uint64_t)t->h_tasks[k].n * (k1 - k0);
      jobs += (uint64_t)t->h_tasks[k].n;
      max_nE = std::max(max_nE, k1 - k0);
    }
  }
  if (jobs > 0xffffffffull || max_nE > 4096)
    return fail(ctx, NEGF_E_INVALID, "%s: too many sites or energies for the energy rows", who);
  cudaError_t e = dalloc(d_edesc, ed.size(), s, nullptr);
  uint32_t* d_jb = nullptr;
  if (e == cudaSuccess) e = dalloc(&d_jb, jb.size(), s, nullptr);
  if (e == cudaSuccess) e = dalloc(d_etab, std::max<uint64_t>(eoff, 1), s, nullptr);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(*d_edesc, ed.data(), sizeof(negf::EnergyDesc) * ed.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_jb, jb.data(), sizeof(uint32_t) * jb.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "energy_alias_kernel", 1);
    e = negf::launch_energy_tables(t->d_tasks, t->n_tasks, *d_edesc, d_jb, (uint32_t)jobs,
                                   max_nE, sigma, t->d_rowsum, *d_etab, t->d_err, s);
  }
  // the host copies of ed and jb must outlive the asynchronous copies
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(d_jb, s);
  if (e != cudaSuccess) {
    dfree(*d_edesc, s);
    dfree(*d_etab, s);
    return fail(ctx, NEGF_E_CUDA, "%s: %s", who, cudaGetErrorString(e));
  }
  if (h_out) *h_out = ed;
  return NEGF_OK;
}

negf_status negf_walk_inelastic(negf_ctx ctx, negf_tables t, int32_t start_lead, uint64_t seed,
                                uint64_t walkers_per_task, uint64_t walker_id_offset,
                                uint32_t max_steps, double sigma_E, negf_tally* out) {
  negf_status st = walk_common(ctx, t, start_lead, max_steps, "negf_walk_inelastic");
  if (st != NEGF_OK) return st;
  if (!out) return fail(ctx, NEGF_E_INVALID, "negf_walk_inelastic: out is NULL");
  *out = nullptr;
  if (walkers_per_task > (1ull << 40))
    return fail(ctx, NEGF_E_INVALID, "negf_walk_inelastic: walkers_per_task above 2^40");
  DeviceGuard g(ctx->device);
  negf::EnergyDesc* d_edesc = nullptr;
  uint64_t* d_etab = nullptr;
  st = energy_tables(ctx, t, sigma_E, "negf_walk_inelastic", &d_edesc, &d_etab, nullptr);
  if (st != NEGF_OK) return st;
  negf_tally tl = new (std::nothrow) negf_tally_s;
  if (!tl) {
    dfree(d_edesc, ctx->stream);
    dfree(d_etab, ctx->stream);
    return fail(ctx, NEGF_E_NOMEM, "negf_walk_inelastic: host allocation");
  }
  tl->ctx = ctx;
  tl->n_tasks = t->n_tasks;
  tl->start_lead = start_lead;
  const size_t nc = (size_t)std::max(1, t->n_tasks) * NEGF_TALLY_FIELDS;
  cudaError_t e = dalloc(&tl->d_counts, nc, ctx->stream, nullptr);
  if (e == cudaSuccess) e = cudaMemsetAsync(tl->d_counts, 0, sizeof(uint64_t) * nc, ctx->stream);
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "inelastic_walk_kernel", (t->n_tasks + 1023) / 1024);
    e = negf::launch_inelastic_walk(t->d_tasks, t->n_tasks, d_edesc, t->d_tab, t->d_mode_tab,
                                    t->d_c, d_etab, start_lead, seed, walkers_per_task,
                                    walker_id_offset, max_steps, tl->d_counts, ctx->sm_count,
                                    ctx->stream);
  }
  dfree(d_edesc, ctx->stream);
  dfree(d_etab, ctx->stream);
  if (e != cudaSuccess) {
    dfree(tl->d_counts, ctx->stream);
    delete tl;
    return fail(ctx, NEGF_E_CUDA, "negf_walk_inelastic: %s", cudaGetErrorString(e));
  }
  *out = tl;
  return NEGF_OK;
}

negf_status negf_export_energy_tables(negf_ctx ctx, negf_tables t, int32_t task, double sigma_E,
                                      void* host_buf, size_t* bytes) {
  if (!ctx || !t || t->ctx != ctx || !bytes)
    return fail(ctx, NEGF_E_INVALID, "negf_export_energy_tables: bad argument");
  if (task < 0 || task >= t->n_tasks)
    return fail(ctx, NEGF_E_INVALID, "negf_export_energy_tables: task %d out of range", task);
  int nE = 0;
  for (int w = 0; w < t->n_wires; ++w)
    if (task >= t->h_wire_task0[w] && task < t->h_wire_task0[w + 1])
      nE = t->h_wire_task0[w + 1] - t->h_wire_task0[w];
  const size_t need = sizeof(uint64_t) * (size_t)t->h_tasks[task].n * nE;
  if (!host_buf) {
    *bytes = need;
    return NEGF_OK;
  }
  if (*bytes < need)
    return fail(ctx, NEGF_E_INVALID, "negf_export_energy_tables: buffer of %zu bytes, need %zu",
                *bytes, need);
  DeviceGuard g(ctx->device);
  negf::EnergyDesc* d_edesc = nullptr;
  uint64_t* d_etab = nullptr;
  std::vector<negf::EnergyDesc> ed;
  negf_status st = energy_tables(ctx, t, sigma_E, "negf_export_energy_tables", &d_edesc, &d_etab, &ed);
  if (st != NEGF_OK) return st;
  cudaError_t e = cudaMemcpyAsync(host_buf, d_etab + ed[task].eoff, need, cudaMemcpyDeviceToHost,
                                  ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  dfree(d_edesc, ctx->stream);
  dfree(d_etab, ctx->stream);
  if (e != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "negf_export_energy_tables: %s", cudaGetErrorString(e));
  int32_t err = 0;
  if (cudaMemcpy(&err, t->d_err, sizeof(err), cudaMemcpyDeviceToHost) == cudaSuccess && err)
    return fail(ctx, NEGF_E_NUMERIC, "negf_export_energy_tables: energy rows not finite");
  *bytes = need;
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
    e = negf::launch_walk(t->d_tasks, task, 1, 0, t->d_tab, t->d_mode_tab, t->d_c, start_lead,
                          seed, n_walkers, walker_id_offset, max_steps, ctx->d_counter, tmp,
                          d_lead, d_steps, nullptr, 0, nullptr, 0, ctx->sm_count, 0,
                          ctx->stream, nullptr, walk_slots(t->any_two), t->any_two);
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

negf_status negf_walk_score(negf_ctx ctx, negf_tables t, int32_t start_lead, uint64_t seed,
                            uint64_t walkers_per_task, uint64_t walker_id_offset,
                            uint32_t max_steps, negf_tally* out) {
  negf_status st = walk_common(ctx, t, start_lead, max_steps, "negf_walk_score");
  if (st != NEGF_OK) return st;
  if (!out) return fail(ctx, NEGF_E_INVALID, "negf_walk_score: out is NULL");
  *out = nullptr;
  if (t->tables_released || !t->d_tab)
    return fail(ctx, NEGF_E_INVALID, "negf_walk_score: the tables of this handle were released");
  if (walkers_per_task > (1ull << 40))
    return fail(ctx, NEGF_E_INVALID, "negf_walk_score: walkers_per_task above 2^40");
  for (const TaskDesc& d : t->h_tasks)
    if (d.l2_fused)
      return fail(ctx, NEGF_E_INVALID,
                  "negf_walk_score: score tallies need the tables' weights (keep_weights)");
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  negf_tally tl = new (std::nothrow) negf_tally_s;
  if (!tl) return fail(ctx, NEGF_E_NOMEM, "negf_walk_score: host allocation");
  tl->ctx = ctx;
  tl->n_tasks = t->n_tasks;
  tl->start_lead = start_lead;
  tl->score_stride = t->score_stride;
  tl->mode_stride = t->mode_stride;
  const size_t nc = (size_t)std::max(1, t->n_tasks) * NEGF_TALLY_FIELDS;
  cudaError_t e = dalloc(&tl->d_counts, nc, s, nullptr);
  if (e == cudaSuccess) e = dalloc(&tl->d_score, 2 * std::max<uint64_t>(tl->score_stride, 1), s, nullptr);
  // the injection-mode counts in negf::kModeReplicas copies, summed into the first by the walk
  const size_t mode_words = 2 * (size_t)std::max<uint32_t>(tl->mode_stride, 1) * negf::kModeReplicas;
  if (e == cudaSuccess) e = dalloc(&tl->d_mode_score, mode_words, s, nullptr);
  if (e == cudaSuccess) e = cudaMemsetAsync(tl->d_counts, 0, sizeof(uint64_t) * nc, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(tl->d_score, 0, sizeof(uint64_t) * 2 * std::max<uint64_t>(tl->score_stride, 1), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(tl->d_mode_score, 0, sizeof(uint64_t) * mode_words, s);
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "walk_score_kernel", (t->n_tasks + 1023) / 1024);
    e = negf::launch_walk(t->d_tasks, 0, t->n_tasks, 0, t->d_tab, t->d_mode_tab, t->d_c,
                          start_lead, seed, walkers_per_task, walker_id_offset, max_steps,
                          ctx->d_counter, tl->d_counts, nullptr, nullptr, tl->d_score,
                          tl->score_stride, tl->d_mode_score, tl->mode_stride, ctx->sm_count, 0,
                          s, nullptr, 1, t->any_two);
  }
  if (e != cudaSuccess) {
    negf_tally_free(tl);
    return fail(ctx, NEGF_E_CUDA, "negf_walk_score: %s", cudaGetErrorString(e));
  }
  *out = tl;
  return NEGF_OK;
}

negf_status negf_tally_score_counts(negf_ctx ctx, negf_tally tl, uint64_t* host_counts,
                                    uint64_t* host_mode_counts) {
  if (!ctx || !tl || tl->ctx != ctx || !tl->d_score || !host_counts || !host_mode_counts)
    return fail(ctx, NEGF_E_INVALID, "negf_tally_score_counts: bad argument or no score tallies");
  DeviceGuard g(ctx->device);
  CUDA_TRY(ctx, cudaMemcpyAsync(host_counts, tl->d_score, sizeof(uint64_t) * 2 * tl->score_stride,
                                cudaMemcpyDeviceToHost, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(host_mode_counts, tl->d_mode_score,
                                sizeof(uint64_t) * 2 * tl->mode_stride, cudaMemcpyDeviceToHost,
                                ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return NEGF_OK;
}

negf_status negf_tally_score_accumulate(negf_ctx ctx, negf_tally tl, const uint64_t* host_counts,
                                        const uint64_t* host_mode_counts) {
  if (!ctx || !tl || tl->ctx != ctx || !tl->d_score || !host_counts || !host_mode_counts)
    return fail(ctx, NEGF_E_INVALID, "negf_tally_score_accumulate: bad argument or no score tallies");
  std::vector<uint64_t> c(2 * tl->score_stride), m(2 * (size_t)tl->mode_stride);
  negf_status st = negf_tally_score_counts(ctx, tl, c.data(), m.data());
  if (st != NEGF_OK) return st;
  for (size_t i = 0; i < c.size(); ++i) c[i] += host_counts[i];
  for (size_t i = 0; i < m.size(); ++i) m[i] += host_mode_counts[i];
  DeviceGuard g(ctx->device);
  CUDA_TRY(ctx, cudaMemcpyAsync(tl->d_score, c.data(), sizeof(uint64_t) * c.size(),
                                cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaMemcpyAsync(tl->d_mode_score, m.data(), sizeof(uint64_t) * m.size(),
                                cudaMemcpyHostToDevice, ctx->stream));
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream));
  return NEGF_OK;
}

uint64_t negf_tally_score_size(negf_tally tl) { return tl ? tl->score_stride : 0; }
uint32_t negf_tally_mode_size(negf_tally tl) { return tl ? tl->mode_stride : 0; }

negf_status negf_current_backward(negf_ctx ctx, negf_tables t, negf_tally tl, double mu_p,
                                  double mu_q, double kT, const double* dI, double* d_onsite,
                                  double* d_eta) {
  if (!ctx || !t || !tl || t->ctx != ctx || tl->ctx != ctx || tl->n_tasks != t->n_tasks)
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward: bad or mismatched handles");
  if (!t->d_green || !t->d_weights || !t->d_phi)
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward: build the tables with keep_green");
  if (!tl->d_score) return fail(ctx, NEGF_E_INVALID, "negf_current_backward: tally has no score counts (use negf_walk_score)");
  if (!(kT > 0.0) || !isfinite(mu_p) || !isfinite(mu_q) || !isfinite(kT))
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward: need finite mu and kT > 0");
  if (t->n_wires > 0 && (!dI || !d_onsite || !d_eta))
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward: NULL seed or output");
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  const int nt = t->n_tasks, nw = t->n_wires, prec = t->precision;
  const size_t cb = negf::block_bytes(prec);
  // per-task and per-wire site offsets; the largest task sizes the scratch
  std::vector<uint64_t> tso(nt), wso(nw);
  uint64_t n_sites_tasks = 0, n_sites_wires = 0;
  int max_n = 1;
  for (int k = 0; k < nt; ++k) {
    tso[k] = n_sites_tasks;
    n_sites_tasks += t->h_tasks[k].n;
    max_n = std::max(max_n, t->h_tasks[k].n);
  }
  for (int w = 0; w < nw; ++w) {
    wso[w] = n_sites_wires;
    const int k0 = t->h_wire_task0[w];
    if (k0 < t->h_wire_task0[w + 1]) n_sites_wires += t->h_tasks[k0].n;
  }
  // wires without energies still own sites in the output: size them from the caller's view
  double* d_wbar = nullptr;
  double* d_ubar = nullptr;
  double* d_dT = nullptr;
  double* d_seed = nullptr;
  double* d_out = nullptr;
  uint64_t* d_tso = nullptr;
  uint64_t* d_wso = nullptr;
  void* d_Gbar = nullptr;
  void* d_Y = nullptr;
  cudaError_t e = dalloc(&d_wbar, std::max<uint64_t>(t->score_stride, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_ubar, std::max<uint32_t>(t->mode_stride, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_dT, 2 * std::max<uint64_t>(n_sites_tasks, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_seed, std::max(nw, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_out, 2 * std::max<uint64_t>(n_sites_wires, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_tso, std::max(nt, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_wso, std::max(nw, 1), s, nullptr);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_Gbar, (size_t)max_n * max_n * cb, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&d_Y, (size_t)max_n * max_n * cb, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ubar, 0, sizeof(double) * std::max<uint32_t>(t->mode_stride, 1), s);
  if (e == cudaSuccess && nt > 0)
    e = cudaMemcpyAsync(d_tso, tso.data(), sizeof(uint64_t) * nt, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && nw > 0) {
    e = cudaMemcpyAsync(d_wso, wso.data(), sizeof(uint64_t) * nw, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_seed, dI, sizeof(double) * nw, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "backward_seeds_kernel", 1);
    e = negf::launch_backward_seeds(t->d_tasks, nt, t->total_jobs, prec, t->d_weights, t->d_rowsum,
                                    t->d_mode_w, t->d_c, tl->d_counts, tl->d_score,
                                    tl->score_stride, tl->d_mode_score, tl->mode_stride,
                                    tl->start_lead, d_wbar, 0, d_ubar, s);
  }
  for (int k = 0; k < nt && e == cudaSuccess; ++k) {
    const TaskDesc& d = t->h_tasks[k];
    ProfScope ps(ctx, "backward_task_kernels", 8);
    e = negf::launch_backward_task(
        d, prec, static_cast<const char*>(t->d_green) + d.green_off * cb,
        static_cast<const char*>(t->d_gphi) + d.gphi_off * cb, d_wbar, d_ubar,
        t->d_wire + d.onsite_off + d.n, t->d_phi + d.phi_off, t->d_gam + d.lead_off,
        tl->start_lead, d_Gbar, d_Y, d_dT + tso[k], d_dT + n_sites_tasks + tso[k],
        ctx->sm_count, t->d_err, s);
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "grad_sum_kernel", 1);
    e = negf::launch_grad_sum(t->d_tasks, nw, t->d_wire_task0, d_tso, d_wso, d_dT,
                              d_dT + n_sites_tasks, d_seed, mu_p, mu_q, kT, d_out,
                              d_out + n_sites_wires, s);
  }
  std::vector<double> h(2 * n_sites_wires);
  if (e == cudaSuccess && n_sites_wires > 0)
    e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  dfree(d_wbar, s);
  dfree(d_ubar, s);
  dfree(d_dT, s);
  dfree(d_seed, s);
  dfree(d_out, s);
  dfree(d_tso, s);
  dfree(d_wso, s);
  if (d_Gbar) cudaFreeAsync(d_Gbar, s);
  if (d_Y) cudaFreeAsync(d_Y, s);
  if (e != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "negf_current_backward: %s", cudaGetErrorString(e));
  negf_status st = check_device(ctx, t);
  if (st != NEGF_OK) return st;
  // scatter per wire into the caller's layout (sites of wire w at sum of n of earlier wires;
  // wires without energies get zeros)
  uint64_t off = 0;
  for (int w = 0; w < nw; ++w) {
    const int k0 = t->h_wire_task0[w];
    const bool has = k0 < t->h_wire_task0[w + 1];
    int n = 0;
    if (has) n = t->h_tasks[k0].n;
    for (int i = 0; i < n; ++i) {
      d_onsite[off + i] = h[wso[w] + i];
      d_eta[off + i] = h[n_sites_wires + wso[w] + i];
    }
    off += n;
  }
  std::vector<uint64_t> cnt((size_t)nt * NEGF_TALLY_FIELDS);
  if (nt > 0) {
    st = negf_tally_counts(ctx, tl, cnt.data());
    if (st != NEGF_OK) return st;
    for (int k = 0; k < nt; ++k)
      if (cnt[(size_t)k * NEGF_TALLY_FIELDS + 3] > 0)
        return fail(ctx, NEGF_E_STEPCAP, "negf_current_backward: truncated walks bias the gradient");
  }
  return NEGF_OK;
}

negf_status negf_current_backward_rgf(negf_ctx ctx, negf_tables t, negf_tally tl, double mu_p,
                                      double mu_q, double kT, const double* dI,
                                      int32_t ckpt_stride, double* d_onsite, double* d_eta) {
  if (!ctx || !t || !tl || t->ctx != ctx || tl->ctx != ctx || tl->n_tasks != t->n_tasks)
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward_rgf: bad or mismatched handles");
  if (!t->d_weights || !t->d_phi)
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward_rgf: build the tables with keep_weights");
  if (!tl->d_score)
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward_rgf: tally has no score counts (use negf_walk_score)");
  if (!(kT > 0.0) || !isfinite(mu_p) || !isfinite(mu_q) || !isfinite(kT))
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward_rgf: need finite mu and kT > 0");
  if (ckpt_stride < 0)
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward_rgf: ckpt_stride < 0");
  if (t->n_wires > 0 && (!dI || !d_onsite || !d_eta))
    return fail(ctx, NEGF_E_INVALID, "negf_current_backward_rgf: NULL seed or output");
  for (const TaskDesc& d : t->h_tasks)
    if (d.fused)
      return fail(ctx, NEGF_E_INVALID,
                  "negf_current_backward_rgf: split-TF32 tables keep no weights (use FP32 or FP64)");
  const int stride = ckpt_stride == 0 ? NEGF_CKPT_STRIDE_DEFAULT : ckpt_stride;
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  const int nt = t->n_tasks, nw = t->n_wires, prec = t->precision;
  const uint64_t cb = negf::block_bytes(prec);
  std::vector<uint64_t> tso(nt), wso(nw), ck_off(nt);
  uint64_t n_sites_tasks = 0, n_sites_wires = 0, ck_total = 0;
  for (int k = 0; k < nt; ++k) {
    const TaskDesc& d = t->h_tasks[k];
    tso[k] = n_sites_tasks;
    n_sites_tasks += d.n;
    ck_off[k] = ck_total;
    ck_total += 2ull * ((d.L + stride - 1) / stride) * d.W * d.W;
  }
  for (int w = 0; w < nw; ++w) {
    wso[w] = n_sites_wires;
    const int k0 = t->h_wire_task0[w];
    if (k0 < t->h_wire_task0[w + 1]) n_sites_wires += t->h_tasks[k0].n;
  }
  // groups: runs of tasks of one wire (same W, L), as many as the scratch budget holds
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) free_b = 1ull << 30;
  const uint64_t budget = std::max<uint64_t>(std::min<uint64_t>(free_b / 2, 16ull << 30), 64ull << 20);
  struct Group { int t0, n, slots; };
  std::vector<Group> groups;
  uint64_t max_task_buf = 0, max_slot_buf = 0;
  int max_slots = 0;
  for (int w = 0; w < nw; ++w) {
    const int k0 = t->h_wire_task0[w], k1 = t->h_wire_task0[w + 1];
    if (k0 == k1) continue;
    const TaskDesc& d = t->h_tasks[k0];
    const uint64_t blk = (uint64_t)d.W * d.W * cb;
    const int nc = negf::adjoint_cols_per_job(d.W);
    const uint64_t jobs_per_task = 1 + (uint64_t)(d.L - 1 + nc - 1) / nc;
    const uint64_t per_task = (3ull * d.L + 2) * blk;   // gl, gr, Psi, Tl
    const uint64_t per_slot = 2ull * d.L * blk * nc;     // X, Y panels of nc block columns
    const int per_sm = negf::adjoint_column_occupancy(d.W, prec);
    for (int k = k0; k < k1;) {
      int n = std::min(k1 - k, 64);
      int slots = 0;
      while (true) {
        slots = (int)std::min<uint64_t>((uint64_t)n * jobs_per_task,
                                        (uint64_t)ctx->sm_count * per_sm);
        if (n == 1 || n * per_task + slots * per_slot <= budget) break;
        n = std::max(1, n / 2);
      }
      while (slots > 1 && n * per_task + slots * per_slot > budget) slots /= 2;
      groups.push_back(Group{k, n, slots});
      max_task_buf = std::max(max_task_buf, (uint64_t)n * per_task);
      max_slot_buf = std::max(max_slot_buf, (uint64_t)slots * per_slot);
      max_slots = std::max(max_slots, slots);
      k += n;
    }
  }
  double* d_wbar = nullptr;
  double* d_ubar = nullptr;
  double* d_dT = nullptr;
  double* d_seed = nullptr;
  double* d_out = nullptr;
  uint64_t* d_tso = nullptr;
  uint64_t* d_wso = nullptr;
  uint64_t* d_ck_off = nullptr;
  unsigned char* d_ck = nullptr;
  unsigned char* d_tbuf = nullptr;
  unsigned char* d_sbuf = nullptr;
  // the weight seeds in the precision of the tables (FP32 tables: FP32 seeds, half the words)
  const bool wbar32 = prec != NEGF_FP64;
  const uint64_t wbar_words = std::max<uint64_t>(t->score_stride, 1);
  cudaError_t e = dalloc(&d_wbar, wbar32 ? (wbar_words + 1) / 2 : wbar_words, s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_ubar, std::max<uint32_t>(t->mode_stride, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_dT, 2 * std::max<uint64_t>(n_sites_tasks, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_seed, std::max(nw, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_out, 2 * std::max<uint64_t>(n_sites_wires, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_tso, std::max(nt, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_wso, std::max(nw, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_ck_off, std::max(nt, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_ck, std::max<uint64_t>(ck_total * cb, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_tbuf, std::max<uint64_t>(max_task_buf, 1), s, nullptr);
  if (e == cudaSuccess) e = dalloc(&d_sbuf, std::max<uint64_t>(max_slot_buf, 1), s, nullptr);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_ubar, 0, sizeof(double) * std::max<uint32_t>(t->mode_stride, 1), s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(d_dT, 0, sizeof(double) * 2 * std::max<uint64_t>(n_sites_tasks, 1), s);
  if (e == cudaSuccess && nt > 0) {
    e = cudaMemcpyAsync(d_tso, tso.data(), sizeof(uint64_t) * nt, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_ck_off, ck_off.data(), sizeof(uint64_t) * nt, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess && nw > 0) {
    e = cudaMemcpyAsync(d_wso, wso.data(), sizeof(uint64_t) * nw, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_seed, dI, sizeof(double) * nw, cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "backward_seeds_kernel", 1);
    e = negf::launch_backward_seeds(t->d_tasks, nt, t->total_jobs, prec, t->d_weights, t->d_rowsum,
                                    t->d_mode_w, t->d_c, tl->d_counts, tl->d_score,
                                    tl->score_stride, tl->d_mode_score, tl->mode_stride,
                                    tl->start_lead, d_wbar, wbar32 ? 1 : 0, d_ubar, s);
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "adjoint_sweep_kernel", 1);
    e = negf::launch_adjoint_sweep(t->d_tasks, nt, t->max_W, prec, t->d_wire, t->d_phi, t->d_sig,
                                   d_ck_off, stride, d_ck, t->d_err, s);
  }
  for (const Group& gr : groups) {
    if (e != cudaSuccess) break;
    const TaskDesc& d = t->h_tasks[gr.t0];
    const uint64_t blk = (uint64_t)d.W * d.W * cb;
    unsigned char* gl = d_tbuf;
    unsigned char* grr = gl + (uint64_t)gr.n * d.L * blk;
    unsigned char* psi = grr + (uint64_t)gr.n * d.L * blk;
    unsigned char* tlb = psi + (uint64_t)gr.n * d.L * blk;
    unsigned char* xs = d_sbuf;
    unsigned char* ys = xs + (uint64_t)gr.slots * d.L * blk * negf::adjoint_cols_per_job(d.W);
    {
      ProfScope ps(ctx, "adjoint_expand_kernel", 1);
      e = negf::launch_adjoint_expand(t->d_tasks, gr.t0, gr.n, d.W, d.L, prec, t->d_wire,
                                      t->d_phi, t->d_sig, d_ck_off, stride, d_ck, gl, grr,
                                      t->d_err, s);
    }
    if (e != cudaSuccess) break;
    ProfScope ps(ctx, "adjoint_column_kernel", 1);
    e = negf::launch_adjoint_columns(t->d_tasks, gr.t0, gr.n, d.W, prec, tl->start_lead,
                                     t->d_wire, t->d_phi, t->d_sig, t->d_gam, d_wbar, d_ubar,
                                     tso[gr.t0], d_dT, d_dT + n_sites_tasks, gl, grr, psi, tlb,
                                     xs, ys, gr.slots, t->d_err, s);
  }
  if (e == cudaSuccess) {
    ProfScope ps(ctx, "grad_sum_kernel", 1);
    e = negf::launch_grad_sum(t->d_tasks, nw, t->d_wire_task0, d_tso, d_wso, d_dT,
                              d_dT + n_sites_tasks, d_seed, mu_p, mu_q, kT, d_out,
                              d_out + n_sites_wires, s);
  }
  std::vector<double> h(2 * n_sites_wires);
  if (e == cudaSuccess && n_sites_wires > 0)
    e = cudaMemcpyAsync(h.data(), d_out, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(d_wbar, s);
  dfree(d_ubar, s);
  dfree(d_dT, s);
  dfree(d_seed, s);
  dfree(d_out, s);
  dfree(d_tso, s);
  dfree(d_wso, s);
  dfree(d_ck_off, s);
  dfree(d_ck, s);
  dfree(d_tbuf, s);
  dfree(d_sbuf, s);
  if (e != cudaSuccess)
    return fail(ctx, e == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                "negf_current_backward_rgf: %s", cudaGetErrorString(e));
  negf_status st = check_device(ctx, t);
  if (st != NEGF_OK) return st;
  uint64_t off = 0;
  for (int w = 0; w < nw; ++w) {
    const int k0 = t->h_wire_task0[w];
    const int n = k0 < t->h_wire_task0[w + 1] ? t->h_tasks[k0].n : 0;
    for (int i = 0; i < n; ++i) {
      d_onsite[off + i] = h[wso[w] + i];
      d_eta[off + i] = h[n_sites_wires + wso[w] + i];
    }
    off += n;
  }
  std::vector<uint64_t> cnt((size_t)nt * NEGF_TALLY_FIELDS);
  if (nt > 0) {
    st = negf_tally_counts(ctx, tl, cnt.data());
    if (st != NEGF_OK) return st;
    for (int k = 0; k < nt; ++k)
      if (cnt[(size_t)k * NEGF_TALLY_FIELDS + 3] > 0)
        return fail(ctx, NEGF_E_STEPCAP, "negf_current_backward_rgf: truncated walks bias the gradient");
  }
  return NEGF_OK;
}

int32_t negf_tally_start_lead(negf_tally tl) { return tl ? tl->start_lead : -1; }

void negf_tally_free(negf_tally tl) {
  if (!tl) return;
  DeviceGuard g(tl->ctx->device);
  if (tl->d_counts) cudaFreeAsync(tl->d_counts, tl->ctx->stream);
  if (tl->d_score) cudaFreeAsync(tl->d_score, tl->ctx->stream);
  if (tl->d_mode_score) cudaFreeAsync(tl->d_mode_score, tl->ctx->stream);
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

negf_status negf_interval_distance(negf_ctx ctx, negf_tables t, int32_t wire, int32_t start_lead,
                                  double* d) {
  if (!ctx || !t || t->ctx != ctx || !d)
    return fail(ctx, NEGF_E_INVALID, "negf_interval_distance: bad argument");
  if (wire < 0 || wire >= t->n_wires)
    return fail(ctx, NEGF_E_INVALID, "negf_interval_distance: wire %d out of range", wire);
  if (start_lead != 0 && start_lead != 1)
    return fail(ctx, NEGF_E_INVALID, "negf_interval_distance: start_lead must be 0 or 1");
  if (!t->d_weights)
    return fail(ctx, NEGF_E_INVALID, "negf_interval_distance: build the tables with keep_weights");
  const int task0 = t->h_wire_task0[wire], task1 = t->h_wire_task0[wire + 1];
  const int M = task1 - task0;
  if (M < 2) return fail(ctx, NEGF_E_INVALID, "negf_interval_distance: the wire needs two energies");
  DeviceGuard g(ctx->device);
  cudaStream_t s = ctx->stream;
  double* d_out = nullptr;
  CUDA_TRY(ctx, dalloc(&d_out, (size_t)(M - 1), s, nullptr));
  cudaError_t e = negf::launch_interval_distance(t->d_tasks, task0, M, t->h_tasks[task0].rows,
                                                 t->precision, t->d_weights, t->d_rowsum,
                                                 t->d_mode_w, t->d_c, start_lead, d_out, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d, d_out, sizeof(double) * (M - 1), cudaMemcpyDeviceToHost, s);
  dfree(d_out, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "negf_interval_distance: %s", cudaGetErrorString(e));
  return check_device(ctx, t);
}

negf_status negf_thermal_grid(negf_ctx ctx, const negf_wire* wire, int32_t precision, double e_lo,
                              double e_hi, int32_t n_init, double tol, int32_t max_points,
                              int32_t start_lead, double* energies, int32_t* n_out) {
  if (!ctx) return NEGF_E_INVALID;
  if (!wire || !energies || !n_out)
    return fail(ctx, NEGF_E_INVALID, "negf_thermal_grid: NULL argument");
  if (!(e_hi > e_lo) || !isfinite(e_lo) || !isfinite(e_hi) || n_init < 2 || max_points < n_init ||
      !(tol > 0.0) || !isfinite(tol))
    return fail(ctx, NEGF_E_INVALID,
                "negf_thermal_grid: need e_lo < e_hi, 2 <= n_init <= max_points, tol > 0");
  // evenly spaced as i * step + e_lo with step = (e_hi - e_lo) / (n_init - 1), the last e_hi
  std::vector<double> grid(n_init);
  const double step = (e_hi - e_lo) / (n_init - 1);
  for (int i = 0; i < n_init; ++i) grid[i] = i + 1 == n_init ? e_hi : i * step + e_lo;
  negf_build_opts o{precision, NEGF_MEM_HOST, 1, 0, NEGF_LAYOUT_AUTO};
  while (true) {
    negf_wire w = *wire;
    w.n_energy = (int32_t)grid.size();
    w.energy = grid.data();
    w.energy_weight = nullptr;
    negf_tables t = nullptr;
    negf_status st = negf_build_tables(ctx, &w, 1, &o, &t);
    if (st != NEGF_OK) return st;
    std::vector<double> d(grid.size() - 1);
    st = negf_interval_distance(ctx, t, 0, start_lead, d.data());
    negf_tables_free(t);
    if (st != NEGF_OK) return st;
    std::vector<double> add;
    for (size_t i = 0; i < d.size(); ++i)
      if (d[i] > tol && (int)(grid.size() + add.size()) < max_points)
        add.push_back(0.5 * (grid[i] + grid[i + 1]));
    if (add.empty()) break;
    grid.insert(grid.end(), add.begin(), add.end());
    std::sort(grid.begin(), grid.end());
  }
  for (size_t i = 0; i < grid.size(); ++i) energies[i] = grid[i];
  *n_out = (int32_t)grid.size();
  return NEGF_OK;
}

negf_status negf_walk_thermal(negf_ctx ctx, negf_tables t, int32_t wire, int32_t start_lead,
                              uint64_t seed, uint64_t walkers, uint64_t walker_id_offset,
                              double mu, double kT, uint32_t max_steps, int32_t* d_lead,
                              uint32_t* d_steps, int32_t* d_interval, uint32_t* d_a,
                              negf_thermal_result* out) {
  negf_status st = walk_common(ctx, t, start_lead, max_steps, "negf_walk_thermal");
  if (st != NEGF_OK) return st;
  if (!out) return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: out is NULL");
  if (wire < 0 || wire >= t->n_wires)
    return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: wire %d out of range", wire);
  if (!(kT > 0.0) || !isfinite(kT) || !isfinite(mu))
    return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: need finite mu and kT > 0");
  if (walkers > (1ull << 40))
    return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: walkers above 2^40");
  if (t->tables_released || !t->d_tab)
    return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: the tables were released");
  const int task0 = t->h_wire_task0[wire];
  const int task1 = wire + 1 < t->n_wires ? t->h_wire_task0[wire + 1] : t->n_tasks;
  const int M = task1 - task0;
  if (M < 2) return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: the wire needs two energies");
  const bool two = t->h_tasks[task0].layout == NEGF_LAYOUT_TWO_LEVEL;
  for (int e = 0; e < M; ++e) {
    const TaskDesc& d = t->h_tasks[task0 + e];
    if ((d.layout == NEGF_LAYOUT_TWO_LEVEL) != two)
      return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: the grid mixes one- and two-level tables");
    if (e > 0 && !(d.E > t->h_tasks[task0 + e - 1].E))
      return fail(ctx, NEGF_E_INVALID, "negf_walk_thermal: energies must be strictly ascending");
  }
  // the thermal window Th is the logistic density: CDF F(E) = 1 / (1 + exp(-(E - mu) / kT))
  auto cdf = [&](double E) { return 1.0 / (1.0 + exp(-(E - mu) / kT)); };
  const double F0 = cdf(t->h_tasks[task0].E), F1 = cdf(t->h_tasks[task1 - 1].E);
  const double window = F1 - F0;
  DeviceGuard g(ctx->device);
  const size_t nf = 3 * (size_t)(M - 1) + 5;
  // The energy's interval: the last grid index i with F(E_i) <= F, F = F0 + u window,
  // u = (v + 1/2) 2^-53 for the walker's 53-bit integer v (each step rounded in FP64).  F is
  // non-decreasing in v, so the comparison with grid point i is v >= thr_i, thr_i the least
  // such v (2^53 when none); the device compares integers only.
  std::vector<double> Fg(M);
  for (int k = 0; k < M; ++k) Fg[k] = cdf(t->h_tasks[task0 + k].E);
  auto F_of = [&](uint64_t v) {
    volatile double u = ((double)v + 0.5) * 0x1p-53;
    volatile double du = u * window;                 // rounded before the sum, as written
    return F0 + du;
  };
  std::vector<unsigned long long> thr(M - 1);
  for (int i = 1; i < M; ++i) {
    uint64_t lo = 0, hi = 1ull << 53;                  // least v in [lo, hi] with F >= Fg[i]
    while (lo < hi) {
      const uint64_t mid = lo + (hi - lo) / 2;
      if (F_of(mid) >= Fg[i]) hi = mid; else lo = mid + 1;
    }
    thr[i - 1] = lo;
  }
  // one allocation: the tally, then the interval thresholds
  unsigned long long* d_tally = nullptr;
  CUDA_TRY(ctx, dalloc(&d_tally, nf + (M - 1), ctx->stream, nullptr));
  const unsigned long long* d_thr = d_tally + nf;
  cudaError_t e = cudaMemsetAsync(d_tally, 0, sizeof(unsigned long long) * nf, ctx->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_tally + nf, thr.data(), sizeof(unsigned long long) * (M - 1),
                        cudaMemcpyHostToDevice, ctx->stream);
  if (e == cudaSuccess && window > 0.0) {
    ProfScope ps(ctx, "thermal_walk_kernel");
    e = negf::launch_thermal_walk(t->d_tasks, task0, M, wire, t->d_tab, t->d_mode_tab, t->d_c,
                                  start_lead, seed, walkers, walker_id_offset, max_steps, mu, kT,
                                  F0, window, d_thr, d_tally, d_lead, d_steps, d_interval, d_a,
                                  ctx->sm_count, ctx->stream, two);
  }
  std::vector<unsigned long long> h(nf, 0ull);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h.data(), d_tally, sizeof(unsigned long long) * nf,
                        cudaMemcpyDeviceToHost, ctx->stream);
  cudaFreeAsync(d_tally, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  if (e != cudaSuccess)
    return fail(ctx, NEGF_E_CUDA, "negf_walk_thermal: %s", cudaGetErrorString(e));
  st = check_device(ctx, t);
  if (st != NEGF_OK) return st;
  // X = c_i + alpha (c_{i+1} - c_i) for walkers absorbed at q; alpha = a / 2^32 and
  // alpha^2 ~ (a >> 16)^2 / 2^32 from the integer sums
  std::vector<double> c(M);
  for (int k = 0; k < M; ++k)
    CUDA_TRY(ctx, cudaMemcpy(&c[k], t->d_c + 2 * (task0 + k) + start_lead, sizeof(double),
                             cudaMemcpyDeviceToHost));
  double S1 = 0.0, S2 = 0.0;
  for (int i = 0; i < M - 1; ++i) {
    const double nq = (double)h[3 * i], sa = (double)h[3 * i + 1] * 0x1p-32,
                 sa2 = (double)h[3 * i + 2] * 0x1p-32;
    const double ci = c[i] > 0.0 ? c[i] : 0.0, dc = (c[i + 1] > 0.0 ? c[i + 1] : 0.0) - ci;
    S1 += nq * ci + sa * dc;
    S2 += nq * ci * ci + 2.0 * ci * dc * sa + dc * dc * sa2;
  }
  const size_t G0 = 3 * (size_t)(M - 1);
  const double N = (double)walkers;
  const double mean = N > 0 ? S1 / N : 0.0;
  const double var = N > 0 ? std::max(0.0, S2 / N - mean * mean) : 0.0;
  out->G = window * mean;
  out->se = N > 0 ? window * sqrt(var / N) : 0.0;
  out->window = window;
  out->mean_steps = N > 0 ? (double)h[G0 + 4] / N : 0.0;
  out->walkers = walkers;
  out->absorbed[0] = h[G0 + 0];
  out->absorbed[1] = h[G0 + 1];
  out->closed = h[G0 + 2];
  out->truncated = h[G0 + 3];
  if (out->truncated)
    return fail(ctx, NEGF_E_STEPCAP, "negf_walk_thermal: %llu walks reached max_steps",
                (unsigned long long)out->truncated);
  return NEGF_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------
// Plans: the whole path (inputs -> lead modes -> RGF sweeps -> block columns -> alias tables ->
// walks -> current) captured once into a CUDA graph over preallocated buffers and relaunched
// with a new seed / walker range.  The launch shapes are picked by timing candidates on the
// plan's own first wave before the capture.

struct negf_plan_s {
  negf_ctx ctx = nullptr;
  int prec = NEGF_FP32;
  bool dev_in = false;
  int n_wires = 0;
  Plan P;
  Persist q;
  std::vector<Wave> waves;
  std::vector<size_t> wave_off;              // first rebased descriptor of each wave
  TaskDesc* d_wdesc = nullptr;
  TaskDesc* d_adesc = nullptr;               // alias descriptors of every wave
  TcJob* d_tcjobs = nullptr;                 // tensor-core chain jobs of every wave
  std::vector<size_t> job_off;
  void* d_gL = nullptr;
  void* d_gR = nullptr;
  int slots = 1;                             // waves whose tables exist at once
  std::vector<uint64_t*> d_tab;              // per slot
  std::vector<double*> d_rs, d_start;
  std::vector<void*> d_weights, d_edge;
  uint64_t* d_counts = nullptr;              // [n_tasks][5]
  double* d_out = nullptr;                   // current outputs (launch_current layout)
  uint64_t* d_run = nullptr;                 // seed, walker id offset
  uint64_t* h_ring = nullptr;                // pinned staging of the run parameters
  std::vector<cudaEvent_t> ring_ev;
  unsigned ring_next = 0;
  std::vector<const double*> src_onsite, src_eta, src_slice_h;
  std::vector<int32_t> wire_W;
  std::vector<int64_t> wire_n;               // sites per wire
  negf_run_opts run{};
  double mu_p = 0.0, mu_q = 0.0, kT = 0.0;
  negf_plan_tuning tune{};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> sync_ev;          // fork/join events of the capture
  struct Seg {
    std::string name;
    uint64_t kernels;
    cudaEvent_t a, b;
  };
  std::vector<Seg> segs;                     // timed segments (event nodes in the graph)
  uint64_t bytes = 0;
  uint64_t launches = 0;
};

namespace {

constexpr unsigned kRing = 64;

void plan_release(negf_plan p) {
  if (!p) return;
  negf_ctx ctx = p->ctx;
  cudaStream_t s = ctx ? ctx->stream : nullptr;
  if (s) cudaStreamSynchronize(s);
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  for (cudaEvent_t e : p->sync_ev) cudaEventDestroy(e);
  for (auto& g : p->segs) {
    cudaEventDestroy(g.a);
    cudaEventDestroy(g.b);
  }
  for (cudaEvent_t e : p->ring_ev) cudaEventDestroy(e);
  if (p->h_ring) cudaFreeHost(p->h_ring);
  Persist& q = p->q;
  dfree(q.d_tasks, s);
  dfree(q.d_wire_task0, s);
  dfree(q.d_wire, s);
  dfree(q.d_sig, s);
  dfree(q.d_gam, s);
  dfree(q.d_phi, s);
  dfree(q.d_eta32, s);
  dfree(q.d_mode_tab, s);
  dfree(q.d_mode_w, s);
  dfree(q.d_c, s);
  dfree(q.d_err, s);
  dfree(p->d_wdesc, s);
  dfree(p->d_adesc, s);
  dfree(p->d_tcjobs, s);
  for (auto& x : p->d_edge)
    if (x) cudaFreeAsync(x, s);
  if (p->d_gL) cudaFreeAsync(p->d_gL, s);
  if (p->d_gR) cudaFreeAsync(p->d_gR, s);
  for (auto& x : p->d_tab) dfree(x, s);
  for (auto& x : p->d_rs) dfree(x, s);
  for (auto& x : p->d_start) dfree(x, s);
  for (auto& x : p->d_weights)
    if (x) cudaFreeAsync(x, s);
  dfree(p->d_counts, s);
  dfree(p->d_out, s);
  dfree(p->d_run, s);
  if (s) cudaStreamSynchronize(s);
  delete p;
}

// A timed segment inside the capture: external event-record nodes around the launches.
struct SegScope {
  negf_plan p;
  cudaStream_t s;
  int idx = -1;
  SegScope(negf_plan plan, const char* name, uint64_t kernels, cudaStream_t st, bool on)
      : p(plan), s(st) {
    if (!on) return;
    cudaEvent_t a = nullptr, b = nullptr;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) {
      cudaEventDestroy(a);
      return;
    }
    p->segs.push_back(negf_plan_s::Seg{name, kernels, a, b});
    idx = (int)p->segs.size() - 1;
    cudaEventRecordWithFlags(a, s, cudaEventRecordExternal);
  }
  ~SegScope() {
    if (idx >= 0) cudaEventRecordWithFlags(p->segs[idx].b, s, cudaEventRecordExternal);
  }
};

// Enqueue every step that one launch repeats (inside the capture); `timed` adds event nodes
// around the kernel groups.
negf_status plan_enqueue(negf_plan p, bool timed, cudaStream_t s) {
  negf_ctx ctx = p->ctx;
  cudaStream_t sw = ctx->walk_stream;
  const Plan& P = p->P;
  Persist& q = p->q;
  const int nt = (int)P.tasks.size();
  const int prec = p->prec;
  CUDA_TRY(ctx, cudaMemsetAsync(q.d_err, 0, sizeof(int32_t), s));
  CUDA_TRY(ctx, cudaMemsetAsync(p->d_counts, 0,
                                sizeof(uint64_t) * (size_t)std::max(1, nt) * NEGF_TALLY_FIELDS, s));
  if (p->dev_in) {
    // device inputs are re-read by every launch (same layout as the batch setup)
    uint64_t off = 0;
    for (int w = 0; w < p->n_wires; ++w) {
      const int64_t n = p->wire_n[w];
      CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire + off, p->src_onsite[w], sizeof(double) * n,
                                    cudaMemcpyDeviceToDevice, s));
      CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire + off + n, p->src_eta[w], sizeof(double) * n,
                                    cudaMemcpyDeviceToDevice, s));
      const int64_t W = p->wire_W[w];
      if (p->src_slice_h[w])
        CUDA_TRY(ctx, cudaMemcpyAsync(q.d_wire + off + 2 * n, p->src_slice_h[w],
                                      sizeof(double) * W * W, cudaMemcpyDeviceToDevice, s));
      off += 2 * (uint64_t)n + (p->src_slice_h[w] ? (uint64_t)W * (W + 1) : 0);
    }
  }
  if (nt == 0) return NEGF_OK;
  if (p->dev_in) {
    SegScope sg(p, "validate_kernel", 2, s, timed);
    CUDA_TRY(ctx, negf::launch_validate(q.d_tasks, nt, q.d_wire, q.d_err, s));
  }
  if (P.any_slice_h) {
    SegScope sg(p, "slice_modes_kernel", 1, s, timed);
    CUDA_TRY(ctx, negf::launch_slice_modes(q.d_tasks, nt, P.max_W, q.d_wire, q.d_phi,
                                           reinterpret_cast<float*>(q.d_phi + P.phi_total),
                                           q.d_err, s));
  }
  {
    SegScope sg(p, "lead_modes_kernel", 1, s, timed);
    CUDA_TRY(ctx, negf::launch_lead_modes(q.d_tasks, nt, P.max_W, q.d_wire, q.d_phi,
                                          reinterpret_cast<float*>(q.d_phi + P.phi_total),
                                          q.d_eta32, q.d_sig, q.d_gam, q.d_err, s));
  }
  {
    SegScope sg(p, "rgf_sweep_kernel", 1, s, timed);
    CUDA_TRY(ctx, negf::launch_rgf_sweep(q.d_tasks, nt, P.max_W, prec, q.d_wire, q.d_phi,
                                         q.d_sig, p->d_gL, p->d_gR, q.d_err, s));
  }
  const bool split = p->waves.size() > 1;     // walks on the second stream, overlapped
  for (size_t w = 0; w < p->waves.size(); ++w) {
    const Wave& wv = p->waves[w];
    const int slot = (int)(w % (size_t)p->slots);
    cudaEvent_t built = split ? p->sync_ev[2 * w] : nullptr;
    cudaEvent_t walked = split ? p->sync_ev[2 * w + 1] : nullptr;
    if (split && w >= (size_t)p->slots)
      CUDA_TRY(ctx, cudaStreamWaitEvent(s, p->sync_ev[2 * (w - p->slots) + 1], 0));
    TaskDesc* dd = p->d_wdesc + p->wave_off[w];
    TaskDesc* da = p->d_adesc + p->wave_off[w];
    const int ntw = wv.t1 - wv.t0;
    {
      SegScope sg(p, "diag_chain_kernels", 2, s, timed);
      CUDA_TRY(ctx, negf::launch_block_columns(
                        dd, ntw, wv.cols, P.max_W, prec, q.d_wire, q.d_eta32, q.d_phi,
                        reinterpret_cast<float*>(q.d_phi + P.phi_total), q.d_sig, q.d_gam,
                        p->d_gL, p->d_gR, p->d_start[slot], p->d_weights[slot], p->d_rs[slot],
                        q.d_mode_w, q.d_c + 2 * (size_t)wv.t0, q.d_err, nullptr, nullptr, s,
                        p->tune.chain_warps, wv.cols_max_W));
    }
    if (wv.tcjobs.size() > wv.n_tc) {
      SegScope sg(p, "chain_cta_kernel", 1, s, timed);
      CUDA_TRY(ctx, negf::launch_chain_cta(
                        dd, p->d_tcjobs + p->job_off[w] + wv.n_tc, (uint32_t)wv.n_cta_wide,
                        wv.cta_narrow(), q.d_eta32,
                        reinterpret_cast<const float*>(q.d_phi + P.phi_total), q.d_gam, p->d_gL,
                        p->d_gR, p->d_start[slot], p->d_weights[slot], p->d_tab[slot],
                        q.d_err, s));
    }
    if (wv.n_tc) {
      SegScope sg(p, "chain_tc_kernel", 2, s, timed);
      CUDA_TRY(ctx, negf::launch_chain_tc(
                        dd, ntw, wv.cols, p->d_tcjobs + p->job_off[w], (uint32_t)wv.n_tc,
                        q.d_eta32, reinterpret_cast<const float*>(q.d_phi + P.phi_total),
                        q.d_gam, p->d_gL, p->d_gR, p->d_start[slot], p->d_weights[slot],
                        p->d_tab[slot], p->d_edge[slot], q.d_err, s));
    }
    if (wv.any_two_split) {
      SegScope sg(p, "two_level_kernel", 1, s, timed);
      CUDA_TRY(ctx, negf::launch_two_level_split(dd, ntw, wv.rows, prec, p->d_weights[slot],
                                                 p->d_tab[slot], q.d_err, s, wv.two_max_W));
    }
    {
      SegScope sg(p, "alias_kernel", 1, s, timed);
      CUDA_TRY(ctx, negf::launch_alias_build(da, ntw, wv.rows, P.max_KA, prec, p->d_weights[slot],
                                             p->d_rs[slot], q.d_mode_w, p->d_tab[slot],
                                             q.d_mode_tab, q.d_err, s, p->tune.alias_warps));
    }
    cudaStream_t ws = s;
    if (split) {
      CUDA_TRY(ctx, cudaEventRecord(built, s));
      CUDA_TRY(ctx, cudaStreamWaitEvent(sw, built, 0));
      ws = sw;
    }
    {
      SegScope sg(p, "walk_kernel", (uint64_t)(ntw + 1023) / 1024, ws, timed);
      CUDA_TRY(ctx, negf::launch_walk(dd, 0, ntw, (uint32_t)wv.t0, p->d_tab[slot], q.d_mode_tab,
                                      q.d_c + 2 * (size_t)wv.t0, p->run.start_lead, 0,
                                      p->run.walkers_per_task, 0, p->run.max_steps,
                                      ctx->d_counter,
                                      p->d_counts + (size_t)wv.t0 * NEGF_TALLY_FIELDS, nullptr,
                                      nullptr, nullptr, 0, nullptr, 0, ctx->sm_count,
                                      p->tune.walk_blocks_per_sm, ws, p->d_run,
                                      p->tune.walk_slots > 0 ? p->tune.walk_slots
                                                             : walk_slots(wv.any_two),
                                      wv.any_two));
    }
    if (split) CUDA_TRY(ctx, cudaEventRecord(walked, sw));
  }
  if (split) CUDA_TRY(ctx, cudaStreamWaitEvent(s, p->sync_ev.back(), 0));
  {
    SegScope sg(p, "current_kernel", 1, s, timed);
    CUDA_TRY(ctx, negf::launch_current(q.d_tasks, nt, p->n_wires, q.d_wire_task0, q.d_c,
                                       p->d_counts, p->run.start_lead, p->mu_p, p->mu_q, p->kT,
                                       p->d_out, s));
  }
  return NEGF_OK;
}

// Device time of `f` enqueued on s (best of `reps`).
template <typename F>
float time_on(cudaStream_t s, int reps, F f) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    return -1.f;
  }
  float best = -1.f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(a, s);
    const cudaError_t e = f();
    cudaEventRecord(b, s);
    float ms = 0.f;
    if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess ||
        cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
      best = -1.f;
      break;
    }
    if (best < 0.f || ms < best) best = ms;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// Pick chain warps, alias warps and walk CTAs per SM by timing candidates on wave 0 (its
// inputs, lead modes and sweeps are already on the device).  Leaves wave 0 built.
negf_status plan_autotune(negf_plan p) {
  negf_ctx ctx = p->ctx;
  cudaStream_t s = ctx->stream;
  const Plan& P = p->P;
  Persist& q = p->q;
  const Wave& wv = p->waves[0];
  TaskDesc* dd = p->d_wdesc;
  TaskDesc* da = p->d_adesc;
  const int prec = p->prec;
  const int nt0 = wv.t1 - wv.t0;
  auto columns = [&](int cw) {
    return negf::launch_block_columns(dd, nt0, wv.cols, P.max_W, prec, q.d_wire, q.d_eta32,
                                      q.d_phi, reinterpret_cast<float*>(q.d_phi + P.phi_total),
                                      q.d_sig, q.d_gam, p->d_gL, p->d_gR, p->d_start[0],
                                      p->d_weights[0], p->d_rs[0], q.d_mode_w, q.d_c, q.d_err,
                                      nullptr, nullptr, s, cw, wv.cols_max_W);
  };
  auto columns_split = [&](int cw) {
    cudaError_t e = columns(cw);
    if (e == cudaSuccess && wv.tcjobs.size() > wv.n_tc)
      e = negf::launch_chain_cta(dd, p->d_tcjobs + wv.n_tc, (uint32_t)wv.n_cta_wide,
                                 wv.cta_narrow(), q.d_eta32,
                                 reinterpret_cast<const float*>(q.d_phi + P.phi_total), q.d_gam,
                                 p->d_gL, p->d_gR, p->d_start[0], p->d_weights[0],
                                 p->d_tab[0], q.d_err, s);
    if (e == cudaSuccess && wv.n_tc)
      e = negf::launch_chain_tc(dd, nt0, wv.cols, p->d_tcjobs, (uint32_t)wv.n_tc,
                                q.d_eta32, reinterpret_cast<const float*>(q.d_phi + P.phi_total),
                                q.d_gam, p->d_gL, p->d_gR, p->d_start[0], p->d_weights[0],
                                p->d_tab[0], p->d_edge[0], q.d_err, s);
    if (e == cudaSuccess && wv.any_two_split)
      e = negf::launch_two_level_split(dd, nt0, wv.rows, prec, p->d_weights[0], p->d_tab[0],
                                       q.d_err, s, wv.two_max_W);
    return e;
  };
  auto alias = [&](int aw) {
    return negf::launch_alias_build(da, nt0, wv.rows, P.max_KA, prec, p->d_weights[0],
                                    p->d_rs[0], q.d_mode_w, p->d_tab[0], q.d_mode_tab, q.d_err,
                                    s, aw);
  };
  // chain warps
  int best_cw = 0;
  float best_c = -1.f;
  const int cmax = negf::chain_warps_max(P.max_W, prec);
  for (int cw : {1, 2, 4, 8, 16}) {
    if (cw > cmax) break;
    const float ms = time_on(s, 2, [&]() { return columns(cw); });
    if (ms < 0.f) return fail(ctx, NEGF_E_CUDA, "autotune: block columns failed");
    if (best_c < 0.f || ms < best_c) best_c = ms, best_cw = cw;
  }
  // alias warps (each candidate runs on freshly computed row values)
  int best_aw = 0;
  float best_a = -1.f;
  const int amax = negf::alias_warps_max(P.max_KA);
  for (int aw : {2, 4, 8, 12, 16}) {
    if (aw > amax) break;
    // fresh row values (the alias kernel replaces A by the row sums)
    if (columns_split(best_cw) != cudaSuccess) return fail(ctx, NEGF_E_CUDA, "autotune: columns");
    const float ms = time_on(s, 1, [&]() { return alias(aw); });
    if (ms < 0.f) return fail(ctx, NEGF_E_CUDA, "autotune: alias build failed");
    if (best_a < 0.f || ms < best_a) best_a = ms, best_aw = aw;
  }
  if (best_aw == 0) best_aw = amax;
  // leave wave 0 built with the chosen shapes
  if (columns_split(best_cw) != cudaSuccess || alias(best_aw) != cudaSuccess)
    return fail(ctx, NEGF_E_CUDA, "autotune: rebuild failed");
  // walk grid: CTAs per SM (the tally of the candidates is discarded)
  int best_wb = 0;
  float best_w = -1.f;
  const uint64_t h_run[2] = {0x5eedull, 0ull};
  CUDA_TRY(ctx, cudaMemcpyAsync(p->d_run, h_run, sizeof h_run, cudaMemcpyHostToDevice, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  // (walkers per lane, CTAs per SM): two walkers per lane fit four CTAs per SM
  int best_ws = 1;
  const int cand[][2] = {{1, 2}, {1, 3}, {1, 4}, {1, 5}, {2, 2}, {2, 3}, {2, 4}};
  for (const auto& c : cand) {
    const int ws = c[0], wb = c[1];
    const float ms = time_on(s, 2, [&]() {
      return negf::launch_walk(dd, 0, nt0, (uint32_t)wv.t0, p->d_tab[0], q.d_mode_tab, q.d_c,
                               p->run.start_lead, 0, p->run.walkers_per_task, 0,
                               p->run.max_steps, ctx->d_counter, p->d_counts, nullptr, nullptr,
                               nullptr, 0, nullptr, 0, ctx->sm_count, wb, s, p->d_run, ws,
                               wv.any_two);
    });
    if (ms < 0.f) return fail(ctx, NEGF_E_CUDA, "autotune: walk failed");
    if (best_w < 0.f || ms < best_w) best_w = ms, best_wb = wb, best_ws = ws;
  }
  p->tune.chain_warps = best_cw;
  p->tune.alias_warps = best_aw;
  p->tune.walk_blocks_per_sm = best_wb;
  p->tune.walk_slots = best_ws;
  p->tune.tuned = 1;
  p->tune.chain_ms = best_c;
  p->tune.alias_ms = best_a;
  p->tune.walk_ms = best_w;
  int32_t h_err = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&h_err, q.d_err, sizeof h_err, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h_err) return fail(ctx, err_status(h_err), "device check:%s", err_bits(h_err).c_str());
  return NEGF_OK;
}

}  // namespace

extern "C" {

negf_status negf_plan_create(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                             const negf_build_opts* bopts, const negf_run_opts* ropts,
                             double mu_p, double mu_q, double kT, int32_t autotune,
                             negf_plan* out) {
  if (!ctx) return NEGF_E_INVALID;
  if (!out || !ropts) return fail(ctx, NEGF_E_INVALID, "negf_plan_create: NULL output or options");
  *out = nullptr;
  if (n_wires < 0 || (n_wires > 0 && !wires))
    return fail(ctx, NEGF_E_INVALID, "negf_plan_create: bad wire list");
  negf_build_opts o;
  negf_status st = check_opts(ctx, bopts, o);
  if (st != NEGF_OK) return st;
  if (o.keep_weights || o.keep_green)
    return fail(ctx, NEGF_E_INVALID, "negf_plan_create: keep_weights / keep_green must be 0");
  const negf_run_opts& r = *ropts;
  if (r.start_lead != 0 && r.start_lead != 1)
    return fail(ctx, NEGF_E_INVALID, "negf_plan_create: start_lead must be 0 or 1");
  if (r.max_steps < 1 || r.max_steps > NEGF_MAX_STEPS)
    return fail(ctx, NEGF_E_INVALID, "negf_plan_create: max_steps must be in [1, %u]",
                NEGF_MAX_STEPS);
  if (r.walkers_per_task > (1ull << 40) || r.tasks_per_wave < 0 || r.waves_in_flight < 0 ||
      r.walk_blocks_per_sm < 0 || r.reserved != 0)
    return fail(ctx, NEGF_E_INVALID, "negf_plan_create: bad walker count, wave size, depth or reserved");
  if (!isfinite(mu_p) || !isfinite(mu_q) || !(kT > 0.0) || !isfinite(kT))
    return fail(ctx, NEGF_E_INVALID, "negf_plan_create: need finite mu and kT > 0");
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;
  negf_plan p = new (std::nothrow) negf_plan_s;
  if (!p) return fail(ctx, NEGF_E_NOMEM, "negf_plan_create: host allocation");
  p->ctx = ctx;
  p->prec = o.precision == NEGF_FP64 ? NEGF_FP64 : NEGF_FP32;
  p->dev_in = o.memspace == NEGF_MEM_DEVICE;
  p->n_wires = n_wires;
  p->run = r;
  p->mu_p = mu_p;
  p->mu_q = mu_q;
  p->kT = kT;
  auto bail = [&](negf_status code) {
    plan_release(p);
    return code;
  };
  st = make_plan(ctx, wires, n_wires, p->dev_in, p->P, o.table_layout,
                 o.precision == NEGF_SPLIT_TF32, o.precision != NEGF_FP64, false, true);
  if (st != NEGF_OK) return bail(st);
  const Plan& P = p->P;
  const int nt = (int)P.tasks.size();
  for (int w = 0; w < n_wires; ++w) {
    p->wire_n.push_back((int64_t)wires[w].W * wires[w].L);
    p->wire_W.push_back(wires[w].W);
    if (p->dev_in) {
      p->src_onsite.push_back(wires[w].onsite);
      p->src_eta.push_back(wires[w].eta);
      p->src_slice_h.push_back(wires[w].slice_h);
    }
  }
  if ((!ctx->walk_stream &&
       cudaStreamCreateWithFlags(&ctx->walk_stream, cudaStreamNonBlocking) != cudaSuccess) ||
      (!ctx->capture_stream &&
       cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking) != cudaSuccess))
    return bail(fail(ctx, NEGF_E_CUDA, "negf_plan_create: stream creation failed"));
  // persistent buffers (and a first fill of inputs and lead modes)
  st = setup_batch(ctx, s, wires, n_wires, p->dev_in, P, p->q, &p->bytes);
  if (st != NEGF_OK) return bail(st);
  cudaError_t e = dalloc(&p->d_counts, (size_t)std::max(1, nt) * NEGF_TALLY_FIELDS, s, &p->bytes);
  const size_t m_out = 2 * (size_t)n_wires + 2 * (size_t)nt + 1;
  if (e == cudaSuccess) e = dalloc(&p->d_out, m_out, s, &p->bytes);
  if (e == cudaSuccess) e = dalloc(&p->d_run, 2, s, &p->bytes);
  if (e != cudaSuccess) return bail(fail(ctx, NEGF_E_NOMEM, "plan buffers: %s", cudaGetErrorString(e)));
  // waves: as negf_run, but every slot's tables and scratch stay allocated
  const int depth = r.waves_in_flight > 0 ? r.waves_in_flight : 2;
  uint64_t budget = r.memory_budget;
  if (budget == 0) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    budget = free_b / 2;
  }
  const int per_wave = r.tasks_per_wave > 0 ? r.tasks_per_wave : std::max(1, nt);
  std::vector<uint64_t> task_bytes(nt);
  for (int k = 0; k < nt; ++k) task_bytes[k] = wave_bytes(make_wave(P, k, k + 1), p->prec);
  for (int k = 0; k < nt;) {
    int k1 = k + 1;
    uint64_t bytes_w = task_bytes[k];
    while (k1 < nt && k1 - k < per_wave && (bytes_w + task_bytes[k1]) * depth <= budget)
      bytes_w += task_bytes[k1++];
    p->waves.push_back(make_wave(P, k, k1));
    k = k1;
  }
  p->slots = p->waves.size() > 1 ? std::min<int>(depth, (int)p->waves.size()) : 1;
  uint64_t max_tab = 1, max_rows = 1, max_start = 1, max_wt = 1, max_edge = 0;
  std::vector<TaskDesc> all, alla;
  std::vector<TcJob> jobs;
  for (const Wave& w : p->waves) {
    p->wave_off.push_back(all.size());
    p->job_off.push_back(jobs.size());
    all.insert(all.end(), w.desc.begin(), w.desc.end());
    alla.insert(alla.end(), w.adesc.begin(), w.adesc.end());
    jobs.insert(jobs.end(), w.tcjobs.begin(), w.tcjobs.end());
    max_edge = std::max(max_edge, w.edge);
    max_wt = std::max(max_wt, w.wt + w.l1w);
    max_tab = std::max(max_tab, w.tab);
    max_rows = std::max<uint64_t>(max_rows, w.rows);
    max_start = std::max(max_start, w.start);
  }
  if (nt > 0) {
    e = dalloc(&p->d_wdesc, all.size(), s, &p->bytes);
    if (e == cudaSuccess) e = dalloc(&p->d_adesc, alla.size(), s, &p->bytes);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_wdesc, all.data(), sizeof(TaskDesc) * all.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(p->d_adesc, alla.data(), sizeof(TaskDesc) * alla.size(),
                          cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && !jobs.empty()) e = dalloc(&p->d_tcjobs, jobs.size(), s, &p->bytes);
    if (e == cudaSuccess && !jobs.empty())
      e = cudaMemcpyAsync(p->d_tcjobs, jobs.data(), sizeof(TcJob) * jobs.size(),
                          cudaMemcpyHostToDevice, s);
    const uint64_t gb = std::max<uint64_t>(P.g_total, 1) * negf::block_bytes(p->prec);
    if (e == cudaSuccess) e = cudaMallocAsync(&p->d_gL, gb, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&p->d_gR, gb, s);
    p->bytes += 2 * gb;
    const uint64_t cw = negf::block_bytes(p->prec) / sizeof(double);
    const size_t wsz = p->prec == NEGF_FP64 ? sizeof(double) : sizeof(float);
    p->d_tab.assign(p->slots, nullptr);
    p->d_rs.assign(p->slots, nullptr);
    p->d_start.assign(p->slots, nullptr);
    p->d_weights.assign(p->slots, nullptr);
    p->d_edge.assign(p->slots, nullptr);
    for (int k = 0; k < p->slots && e == cudaSuccess; ++k) {
      if (max_edge) {
        e = cudaMallocAsync(&p->d_edge[k], max_edge * sizeof(negf::cf), s);
        p->bytes += max_edge * sizeof(negf::cf);
      }
      e = dalloc(&p->d_tab[k], max_tab, s, &p->bytes);
      if (e == cudaSuccess) e = dalloc(&p->d_rs[k], max_rows, s, &p->bytes);
      if (e == cudaSuccess) e = dalloc(&p->d_start[k], max_start * cw, s, &p->bytes);
      if (e == cudaSuccess) e = cudaMallocAsync(&p->d_weights[k], max_wt * wsz, s);
      p->bytes += max_wt * wsz;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);   // `all` dies here
    if (e != cudaSuccess)
      return bail(fail(ctx, e == cudaErrorMemoryAllocation ? NEGF_E_NOMEM : NEGF_E_CUDA,
                       "plan tables: %s", cudaGetErrorString(e)));
  }
  // staging ring of the per-launch run parameters
  if (cudaMallocHost(reinterpret_cast<void**>(&p->h_ring), kRing * 2 * sizeof(uint64_t)) !=
      cudaSuccess)
    return bail(fail(ctx, NEGF_E_NOMEM, "plan: pinned staging"));
  p->ring_ev.assign(kRing, nullptr);
  for (unsigned k = 0; k < kRing; ++k)
    if (cudaEventCreateWithFlags(&p->ring_ev[k], cudaEventDisableTiming) != cudaSuccess)
      return bail(fail(ctx, NEGF_E_CUDA, "plan: events"));
  if (p->waves.size() > 1) {
    p->sync_ev.assign(2 * p->waves.size(), nullptr);
    for (auto& ev : p->sync_ev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess)
        return bail(fail(ctx, NEGF_E_CUDA, "plan: events"));
  }
  // launch shapes: tuned on wave 0, or the caller's / built-in defaults
  p->tune.walk_blocks_per_sm = r.walk_blocks_per_sm;
  if (autotune && nt > 0) {
    {
      const bool prof = ctx->prof;
      ctx->prof = false;
      st = sweep_all(ctx, s, P, p->q, p->prec, p->d_gL, p->d_gR);
      if (st == NEGF_OK) st = plan_autotune(p);
      ctx->prof = prof;
    }
    if (st != NEGF_OK) return bail(st);
    if (r.walk_blocks_per_sm > 0) p->tune.walk_blocks_per_sm = r.walk_blocks_per_sm;
  }
  // capture on the context's capture stream; launches go to the context stream
  {
    cudaStream_t cs = ctx->capture_stream;
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    const bool prof = ctx->prof;
    ctx->prof = false;
    e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      ctx->prof = prof;
      return bail(fail(ctx, NEGF_E_CUDA, "plan: begin capture: %s", cudaGetErrorString(e)));
    }
    st = plan_enqueue(p, true, cs);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(cs, &g);
    ctx->prof = prof;
    p->graph = g;
    if (st != NEGF_OK) return bail(st);
    if (e != cudaSuccess) return bail(fail(ctx, NEGF_E_CUDA, "plan: capture: %s", cudaGetErrorString(e)));
    e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess)
      return bail(fail(ctx, NEGF_E_CUDA, "plan: instantiate: %s", cudaGetErrorString(e)));
  }
  *out = p;
  return NEGF_OK;
}

negf_status negf_plan_launch(negf_ctx ctx, negf_plan p, uint64_t seed, uint64_t walker_id_offset) {
  if (!ctx || !p || p->ctx != ctx) return ctx ? fail(ctx, NEGF_E_INVALID, "negf_plan_launch: bad plan") : NEGF_E_INVALID;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;
  const unsigned k = p->ring_next++ % kRing;
  // the slot's previous copy must have been consumed before it is overwritten
  CUDA_TRY(ctx, cudaEventSynchronize(p->ring_ev[k]));
  p->h_ring[2 * k] = seed;
  p->h_ring[2 * k + 1] = walker_id_offset;
  CUDA_TRY(ctx, cudaMemcpyAsync(p->d_run, p->h_ring + 2 * k, 2 * sizeof(uint64_t),
                                cudaMemcpyHostToDevice, s));
  CUDA_TRY(ctx, cudaEventRecord(p->ring_ev[k], s));
  CUDA_TRY(ctx, cudaGraphLaunch(p->exec, s));
  ++p->launches;
  if (ctx->prof) {
    // profiling: wait for this launch and add its segment times to the context's accounts
    CUDA_TRY(ctx, cudaStreamSynchronize(s));
    for (auto& g : p->segs) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, g.a, g.b) != cudaSuccess) ms = 0.f;
      int idx = -1;
      for (size_t i = 0; i < ctx->prof_entries.size(); ++i)
        if (ctx->prof_entries[i].name == g.name) idx = (int)i;
      if (idx < 0) {
        ctx->prof_entries.push_back(ProfEntry{});
        ctx->prof_entries.back().name = g.name;
        idx = (int)ctx->prof_entries.size() - 1;
      }
      ctx->prof_entries[idx].launches += g.kernels;
      ctx->prof_entries[idx].ms += ms;
    }
  }
  return NEGF_OK;
}

negf_status negf_plan_result(negf_ctx ctx, negf_plan p, double* I, double* se, double* T,
                             double* T_se, uint64_t* counts) {
  if (!ctx || !p || p->ctx != ctx) return ctx ? fail(ctx, NEGF_E_INVALID, "negf_plan_result: bad plan") : NEGF_E_INVALID;
  DeviceGuard guard(ctx->device);
  cudaStream_t s = ctx->stream;
  const size_t nw = (size_t)p->n_wires, nt = p->P.tasks.size();
  const size_t m = 2 * nw + 2 * nt + 1;
  std::vector<double> h(m, 0.0);
  int32_t h_err = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(h.data(), p->d_out, sizeof(double) * m, cudaMemcpyDeviceToHost, s));
  if (counts)
    CUDA_TRY(ctx, cudaMemcpyAsync(counts, p->d_counts, sizeof(uint64_t) * nt * NEGF_TALLY_FIELDS,
                                  cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaMemcpyAsync(&h_err, p->q.d_err, sizeof h_err, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(ctx, cudaStreamSynchronize(s));
  if (h_err) return fail(ctx, err_status(h_err), "device check:%s", err_bits(h_err).c_str());
  for (size_t w = 0; w < nw; ++w) {
    if (I) I[w] = h[w];
    if (se) se[w] = h[nw + w];
  }
  if (T) for (size_t k = 0; k < nt; ++k) T[k] = h[2 * nw + k];
  if (T_se) for (size_t k = 0; k < nt; ++k) T_se[k] = h[2 * nw + nt + k];
  if (h[m - 1] > 0.0)
    return fail(ctx, NEGF_E_STEPCAP, "negf_plan_result: %.0f walks reached max_steps", h[m - 1]);
  return NEGF_OK;
}

negf_status negf_plan_get_tuning(negf_plan p, negf_plan_tuning* out) {
  if (!p || !out) return NEGF_E_INVALID;
  *out = p->tune;
  return NEGF_OK;
}

int32_t negf_plan_num_tasks(negf_plan p) { return p ? (int32_t)p->P.tasks.size() : 0; }
int32_t negf_plan_num_waves(negf_plan p) { return p ? (int32_t)p->waves.size() : 0; }
uint64_t negf_plan_device_bytes(negf_plan p) { return p ? p->bytes : 0; }

void negf_plan_destroy(negf_plan p) {
  if (!p) return;
  DeviceGuard guard(p->ctx ? p->ctx->device : 0);
  plan_release(p);
}

}  // extern "C"
