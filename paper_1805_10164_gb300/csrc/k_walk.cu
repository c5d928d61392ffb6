// Persistent random-walk kernel (Sec. II.D Steps 1-4 with the start lead fixed as in Sec. II.E,
// and Step 6' of Sec. II.F) and its tally.
//
// Each walker's state lives in registers: task, current table row, draw index s and steps
// taken.  Draw s takes Philox4x32-10 block s/2 with counter
// (s/2, id_lo, id_hi, task) and key (seed_lo, seed_hi), words (x0, x1) for even s, (x2, x3) for
// odd s (the odd half is cached from the even draw).  Draw 0 picks the injection eigenvector of
// Gamma_p from the mode alias row (Eq. lead_out_probability); every later draw is one Step 6'
// transition from the current row: slot c = (x*K)>>32, keep c if y < thr[c] else alias[c].
// Columns n and n+1 are the leads: drawing one ends the walk, and the sample's estimator is
// X_pq = Tr[Gamma_p A] delta_rq (Eq. elast_lin_xpq), tallied as counts per absorbing lead.
// A lane carries one or two walkers at a time (kSlots; with two, the dependent gathers of the
// two walks are in flight together, which pays when the gathers miss L2).  When a walk ends
// the lane starts the next walker of its own run of consecutive walker indices (32 per lane)
// with no warp coordination; once enough lanes of a warp have an idle slot and an empty run,
// one lane claims a new range for all of them from a global counter.  Every loop iteration
// consumes one whole Philox block per walker (two draws: the injection and the first
// transition for a new walker, two transitions afterwards), so the generator runs
// warp-uniformly.  Each lane counts its outcomes for its current task (shared by its slots) in
// registers and adds them to the block's shared tally when it moves to another task; the block
// adds its tally to global memory once.
#include <cuda_runtime.h>

#include "negf_internal.cuh"
#include "philox.cuh"

namespace negf {
namespace {

constexpr int kThreads = 256;
constexpr int kFields = NEGF_TALLY_FIELDS;   // done, absorbed L, absorbed R, truncated, steps
constexpr int kMaxWindow = 1024;             // tasks per launch (40 KB shared tally)
constexpr int kPath = 16;                     // score walks: transitions recorded in shared memory
constexpr int kPathExt = 112;                 // and, further, in the thread's local memory
constexpr unsigned kRun = 32;                // consecutive walkers handed to a lane at a time
constexpr int kClaimMin = 8;                 // dry lanes that trigger a claim
constexpr unsigned kFlushAt = 1u << 26;      // flush a lane's counters before they can overflow

// 64-bit shared counter kept as two 32-bit words (native 32-bit shared atomics).
__device__ __forceinline__ void smem_add64(unsigned* lohi, unsigned v) {
  const unsigned old = atomicAdd(lohi, v);
  if (old + v < old) atomicAdd(lohi + 1, 1u);
}

// copy 0 of the injection-mode counts <- the sum of the kModeReplicas copies (m2 = 2 mode_stride)
__global__ void mode_reduce_kernel(unsigned long long* __restrict__ mode, uint32_t m2) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m2) return;
  unsigned long long v = 0;
  for (int r = 0; r < kModeReplicas; ++r) v += mode[(size_t)r * m2 + i];
  mode[i] = v;
}

__device__ __forceinline__ void flush_lane(unsigned* s_tally, int task_local, unsigned (&a)[kFields]) {
  unsigned* t = s_tally + task_local * kFields * 2;
#pragma unroll
  for (int f = 0; f < kFields; ++f) {
    if (a[f]) smem_add64(t + 2 * f, a[f]);
    a[f] = 0u;
  }
}

// Score tallies (kScore): when a walk is absorbed at lead r every transition a -> b adds 1 to
// score[r][a][b] of its task (and the injection mode to mode_score[r][m]); these are the counts
// the score-function gradient needs.  The lead is known only at the end, so a walk records its
// first kPath + kPathExt transitions (the column drawn at each, the first kPath in shared memory
// and the rest in the thread's local memory: each row is the previous column) and commits them
// when it is absorbed; a longer walk is replayed from its first draw (same counters, same
// tables).  A replay runs on one lane while the warp waits: with a record of 16 the 3 % of
// walks that were longer, 40 % of the transitions, were replayed on the W=16 x L=100 wire.
struct ScoreOut {
  unsigned long long* cnt;        // [2][stride] at each task's wt_off (rows x K, either layout)
  unsigned long long* mode_cnt;   // [2][mode_stride] at each task's mode_off (2 x W)
  unsigned long long stride;
  unsigned mode_stride;
};

// One Step 6' transition from table row `row` of a two-level task: words (x, y) draw the slice
// or lead on the level-1 alias row, v = z >> 1 the site within a drawn slice (level 2: against
// the guide, then against the octet it points to).  Returns the next row: a site k W + a, or
// n + r for lead r.
__device__ __forceinline__ uint32_t two_level_draw(const uint64_t* __restrict__ l1row,
                                                   const uint64_t* __restrict__ trow, uint32_t row,
                                                   uint32_t L, uint32_t W, uint32_t B2, uint4 r) {
  const uint32_t K1 = L + 2;
  const uint32_t c = __umulhi(r.x, K1);
  const uint64_t e = __ldg(l1row + (uint64_t)row * K1 + c);
  const uint32_t k = r.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
  if (k >= L) return W * L + (k - L);
  const uint32_t v = r.z >> 1;
  const uint4* blk = reinterpret_cast<const uint4*>(trow) + (((uint64_t)row * L + k) * B2 >> 2);
  uint32_t g = 0;
  if (W > 8) {
    const uint4 q0 = __ldg(blk), q1 = __ldg(blk + 1);
    g = (q0.x <= v) + (q0.y <= v) + (q0.z <= v) + (q0.w <= v) + (q1.x <= v) + (q1.y <= v) +
        (q1.z <= v) + (q1.w <= v);
    blk += 2 + 2 * g;
  }
  const uint4 o0 = __ldg(blk), o1 = __ldg(blk + 1);
  return k * W + 8 * g + (o0.x <= v) + (o0.y <= v) + (o0.z <= v) + (o0.w <= v) + (o1.x <= v) +
         (o1.y <= v) + (o1.z <= v) + (o1.w <= v);
}

// kTwo: the launch may hold two-level tasks (one-level launches compile without that path).
template <bool kTrace, bool kScore, int kSlotsReq, bool kTwo>
__global__ void __launch_bounds__(kThreads, kScore ? 3 : (kSlotsReq == 2 ? 4 : 5)) walk_kernel(
    const TaskDesc* __restrict__ tasks, int task0, int n_tasks, uint32_t id_base,
    const uint64_t* __restrict__ tab, const uint64_t* __restrict__ mode_tab,
    const double* __restrict__ cvals, int start_lead, PhiloxKey key, uint64_t walkers_per_task,
    uint64_t id_offset, uint32_t max_steps,
    unsigned long long* __restrict__ counter, unsigned long long* __restrict__ tally /*window*/,
    int32_t* __restrict__ trace_lead, uint32_t* __restrict__ trace_steps, ScoreOut score,
    const uint64_t* __restrict__ run) {
  extern __shared__ unsigned s_tally[];   // [n_tasks][kFields][lo, hi], then (kScore) the paths
  uint32_t* s_path = s_tally + n_tasks * kFields * 2;   // [kSlots][kPath][kThreads]
  if (run) {
    // seed and walker id offset supplied on the device (relaunched graphs)
    const uint64_t seed = run[0];
    key = PhiloxKey{(uint32_t)seed, (uint32_t)(seed >> 32)};
    id_offset = run[1];
  }
  for (int i = threadIdx.x; i < n_tasks * kFields * 2; i += blockDim.x) s_tally[i] = 0u;
  __syncthreads();

  const unsigned FULL = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const unsigned long long total = (unsigned long long)n_tasks * walkers_per_task;

  // kSlots walkers per lane (registers), so that their dependent gathers overlap; b = next
  // Philox block (draws 2b, 2b + 1)
  constexpr int kSlots = kSlotsReq;
  bool has[kSlots];
  unsigned long long g[kSlots];
  uint32_t row[kSlots], b[kSlots], steps[kSlots], wid_lo[kSlots], wid_hi[kSlots];
  uint32_t inj[kSlots];                                  // kScore: the injection mode
  // kScore: the column drawn at transition st (1-based) of the lane's walker in slot sl
  uint32_t ext[kScore ? kSlots * kPathExt : 1];
  auto record = [&](int sl, uint32_t st, uint32_t j) {
    if (kScore) {
      if (st <= (uint32_t)kPath) s_path[((uint32_t)sl * kPath + st - 1) * kThreads + threadIdx.x] = j;
      else if (st <= (uint32_t)(kPath + kPathExt)) ext[sl * kPathExt + (st - kPath - 1)] = j;
    }
  };
#pragma unroll
  for (int sl = 0; sl < kSlots; ++sl) {
    has[sl] = false;
    g[sl] = 0;
    row[sl] = b[sl] = steps[sl] = wid_lo[sl] = wid_hi[sl] = inj[sl] = 0;
  }
  // this lane's run of walker indices [r_next, r_end)
  unsigned long long r_next = 0, r_end = 0;
  // cached task (shared by the slots): index window [t_first, t_first + walkers_per_task)
  int tl = -1;
  unsigned long long t_first = 0;
  uint32_t task_id = 0, K = 0, n = 0, W = 0, inj_row0 = 0, L = 0, B2 = 0;
  bool two = false;                  // two-level tables (level 1 at l1row, level 2 at trow)
  uint64_t t_wt_off = 0;
  uint32_t t_mode_off = 0;
  bool t_open = false;
  const uint64_t* trow = nullptr;
  const uint64_t* l1row = nullptr;
  const uint64_t* mrow = nullptr;
  unsigned a[kFields] = {0u, 0u, 0u, 0u, 0u};    // counts of task tl not yet in shared memory
  bool no_more = false;

  while (true) {
    // ---- start walkers from the lane's own run (closed tasks are consumed on the spot); a
    // slot takes a walker of another task only when the other slots are idle
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      while (!has[sl] && r_next < r_end) {
        const unsigned long long gn = r_next;
        if (tl < 0 || gn - t_first >= walkers_per_task) {
          bool others = false;
#pragma unroll
          for (int o = 0; o < kSlots; ++o)
            if (o != sl) others |= has[o];
          if (others) break;
          if (tl >= 0) flush_lane(s_tally, tl, a);
          tl = (int)(gn / walkers_per_task);
          t_first = (unsigned long long)tl * walkers_per_task;
          const TaskDesc& d = tasks[task0 + tl];
          task_id = id_base + (uint32_t)(task0 + tl);
          K = (uint32_t)d.K;
          n = (uint32_t)d.n;
          W = (uint32_t)d.W;
          inj_row0 = (uint32_t)(d.n + start_lead * d.W);
          t_wt_off = d.wt_off;
          t_mode_off = d.mode_off + start_lead * d.W;
          trow = tab + d.tab_off;
          two = kTwo && d.layout == NEGF_LAYOUT_TWO_LEVEL;
          L = (uint32_t)d.L;
          B2 = (uint32_t)level2_words(d.W);
          l1row = tab + d.l1_off;
          mrow = mode_tab + d.mode_off + start_lead * d.W;
          t_open = cvals[2 * (task0 + tl) + start_lead] > 0.0;
        }
        ++r_next;
        if (!t_open) {
          // no open channel in the start lead: nothing to inject (T = 0 exactly)
          a[0] += 1u;
          if (kTrace) { trace_lead[gn] = -1; trace_steps[gn] = 0; }
          continue;
        }
        const uint64_t w = id_offset + (gn - t_first);
        g[sl] = gn;
        wid_lo[sl] = (uint32_t)w;
        wid_hi[sl] = (uint32_t)(w >> 32);
        b[sl] = 0;
        steps[sl] = 0;
        has[sl] = true;
      }
    }
    bool busy = false, idle = false;
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      busy |= has[sl];
      idle |= !has[sl];
    }
    // ---- claim new runs once enough lanes have an idle slot and an empty run (or none has
    // work left)
    const unsigned dry = __ballot_sync(FULL, idle && r_next >= r_end);
    if (dry && !no_more && (__popc(dry) >= kClaimMin || dry == FULL)) {
      unsigned long long base = 0;
      if (lane == 0) base = atomicAdd(counter, (unsigned long long)__popc(dry) * kRun);
      base = __shfl_sync(FULL, base, 0);
      if (base >= total) {
        no_more = true;
      } else if (dry & (1u << lane)) {
        const unsigned long long lo = base + (unsigned long long)__popc(dry & lt_mask) * kRun;
        r_next = lo < total ? lo : total;
        r_end = lo + kRun < total ? lo + kRun : total;
      }
      continue;      // start the new walkers first
    }
    // nothing in flight and nothing left to claim (with one slot an idle lane has an empty
    // run, so the ballot above already says it)
    if (kSlots == 1 ? dry == FULL : !__any_sync(FULL, busy)) break;
    if (!busy) continue;

    // ---- per walking slot one Philox block = two draws.  Block 0: the injection draw (Step 4)
    // then the first transition; later blocks: two Step 6' transitions.
#pragma unroll
    for (int sl = 0; sl < kSlots; ++sl) {
      if (!has[sl]) continue;
      const uint4 r = philox4x32_10(make_uint4(b[sl], wid_lo[sl], wid_hi[sl], task_id), key);
      int outcome = -3;                // -3: continue, 0/1: absorbed at L/R, -2: truncated
      if (kTwo && two) {
        // two-level tables: block 0 is the injection draw alone; block b >= 1 is transition
        // b, words (x, y) for the slice or lead (level 1, alias), z for the site in the slice
        // (level 2: v = z >> 1 against the guide, then against the octet it points to)
        if (b[sl] == 0) {
          const uint32_t c = __umulhi(r.x, W);
          const uint64_t e = __ldg(mrow + c);
          inj[sl] = r.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
          row[sl] = inj_row0 + inj[sl];
        } else {
          const uint32_t j = two_level_draw(l1row, trow, row[sl], L, W, B2, r);
          ++steps[sl];
          record(sl, steps[sl], j);
          if (j >= n) outcome = (int)(j - n);
          else if (steps[sl] >= max_steps) outcome = -2;
          else row[sl] = j;
        }
        ++b[sl];
      } else {
        if (b[sl] == 0) {
          const uint32_t c = __umulhi(r.x, W);
          const uint64_t e = __ldg(mrow + c);
          inj[sl] = r.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
          row[sl] = inj_row0 + inj[sl];
        } else {
          const uint32_t c = __umulhi(r.x, K);
          const uint64_t e = __ldg(trow + (uint64_t)row[sl] * K + c);
          const uint32_t j = r.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
          ++steps[sl];
          record(sl, steps[sl], j);
          if (j >= n) outcome = (int)(j - n);
          else if (steps[sl] >= max_steps) outcome = -2;
          else row[sl] = j;
        }
        if (outcome == -3) {
          const uint32_t c = __umulhi(r.z, K);
          const uint64_t e = __ldg(trow + (uint64_t)row[sl] * K + c);
          const uint32_t j = r.w < (uint32_t)e ? c : (uint32_t)(e >> 32);
          ++steps[sl];
          record(sl, steps[sl], j);
          if (j >= n) outcome = (int)(j - n);
          else if (steps[sl] >= max_steps) outcome = -2;
          else row[sl] = j;
        }
        ++b[sl];
      }
      if (kScore && outcome >= 0 && steps[sl] <= (uint32_t)(kPath + kPathExt)) {
        // count the recorded transitions of the finished walk under its absorbing lead
        unsigned long long* cnt = score.cnt + (size_t)outcome * score.stride + t_wt_off;
        atomicAdd(score.mode_cnt +
                      ((size_t)(blockIdx.x % kModeReplicas) * 2 + outcome) * score.mode_stride +
                      t_mode_off + inj[sl],
                  1ull);
        uint32_t rrow = inj_row0 + inj[sl];
        for (uint32_t st = 0; st < steps[sl]; ++st) {
          const uint32_t j = st < (uint32_t)kPath
                                 ? s_path[((uint32_t)sl * kPath + st) * kThreads + threadIdx.x]
                                 : ext[sl * kPathExt + (st - kPath)];
          atomicAdd(cnt + (uint64_t)rrow * K + j, 1ull);
          rrow = j;
        }
      } else if (kScore && outcome >= 0) {
        // a walk longer than the record: replay it and count its transitions
        unsigned long long* cnt = score.cnt + (size_t)outcome * score.stride + t_wt_off;
        unsigned long long* mcnt =
            score.mode_cnt + ((size_t)(blockIdx.x % kModeReplicas) * 2 + outcome) * score.mode_stride +
            t_mode_off;
        uint32_t rrow = 0;
        bool live = true;
        for (uint32_t bb = 0; live; ++bb) {
          const uint4 q = philox4x32_10(make_uint4(bb, wid_lo[sl], wid_hi[sl], task_id), key);
          if (kTwo && two) {
            // two-level: block 0 the injection, block bb >= 1 transition bb (as walked above)
            if (bb == 0) {
              const uint32_t c = __umulhi(q.x, W);
              const uint64_t e = __ldg(mrow + c);
              const uint32_t mode = q.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
              atomicAdd(mcnt + mode, 1ull);
              rrow = inj_row0 + mode;
            } else {
              const uint32_t j = two_level_draw(l1row, trow, rrow, L, W, B2, q);
              atomicAdd(cnt + (uint64_t)rrow * K + j, 1ull);
              if (j >= n) live = false;
              rrow = j;
            }
            continue;
          }
          if (bb == 0) {
            const uint32_t c = __umulhi(q.x, W);
            const uint64_t e = __ldg(mrow + c);
            const uint32_t mode = q.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
            atomicAdd(mcnt + mode, 1ull);
            rrow = inj_row0 + mode;
          } else {
            const uint32_t c = __umulhi(q.x, K);
            const uint64_t e = __ldg(trow + (uint64_t)rrow * K + c);
            const uint32_t j = q.y < (uint32_t)e ? c : (uint32_t)(e >> 32);
            atomicAdd(cnt + (uint64_t)rrow * K + j, 1ull);
            if (j >= n) live = false;
            rrow = j;
          }
          if (live) {
            const uint32_t c = __umulhi(q.z, K);
            const uint64_t e = __ldg(trow + (uint64_t)rrow * K + c);
            const uint32_t j = q.w < (uint32_t)e ? c : (uint32_t)(e >> 32);
            atomicAdd(cnt + (uint64_t)rrow * K + j, 1ull);
            if (j >= n) live = false;
            rrow = j;
          }
        }
      }
      if (outcome != -3) {
        a[0] += 1u;
        if (outcome == 0) a[1] += 1u;
        else if (outcome == 1) a[2] += 1u;
        else a[3] += 1u;
        a[4] += steps[sl];
        if (kTrace) { trace_lead[g[sl]] = outcome; trace_steps[g[sl]] = steps[sl]; }
        has[sl] = false;
        if (a[4] >= kFlushAt || a[0] >= kFlushAt) flush_lane(s_tally, tl, a);
      }
    }
  }
  if (tl >= 0) flush_lane(s_tally, tl, a);
  __syncthreads();
  for (int i = threadIdx.x; i < n_tasks * kFields; i += blockDim.x) {
    const unsigned long long v =
        (unsigned long long)s_tally[2 * i] | ((unsigned long long)s_tally[2 * i + 1] << 32);
    if (v) atomicAdd(&tally[i], v);
  }
}

// ---- gather probe: the memory-system ceiling the walk is measured against ------------------
// Each thread follows `ilp` independent chains of dependent random 8-byte loads over a table
// of n entries (the next index is derived from the loaded value, like a walk step that reads
// one alias entry).  With ilp = 1 this is the walk's access pattern at its occupancy; larger
// ilp gives the throughput ceiling of random 8-byte gathers from that table.

__device__ __forceinline__ uint64_t mix64(uint64_t x) {
  // splitmix64 finaliser (Steele, Lea, Flood, "Fast splittable pseudorandom number
  // generators", OOPSLA 2014)
  x ^= x >> 30;
  x *= 0xbf58476d1ce4e5b9ull;
  x ^= x >> 27;
  x *= 0x94d049bb133111ebull;
  x ^= x >> 31;
  return x;
}

__global__ void probe_fill_kernel(uint64_t* tab, uint64_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    tab[i] = mix64(i + 0x9e3779b97f4a7c15ull);
}

template <int ILP>
__global__ void __launch_bounds__(kThreads, 5) probe_gather_kernel(const uint64_t* __restrict__ tab,
                                                                    uint32_t n, int chain,
                                                                    unsigned long long* sink) {
  uint32_t idx[ILP];
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
#pragma unroll
  for (int c = 0; c < ILP; ++c) idx[c] = (uint32_t)(mix64(tid * ILP + c) % n);
  uint64_t acc = 0;
  for (int it = 0; it < chain; ++it) {
#pragma unroll
    for (int c = 0; c < ILP; ++c) {
      const uint64_t e = __ldg(tab + idx[c]);
      acc += e;
      idx[c] = __umulhi((uint32_t)e ^ (uint32_t)it, n);
    }
  }
  if (acc == 0x123456789ull) atomicAdd(sink, 1ull);   // keeps the loads alive
}

}  // namespace

cudaError_t launch_walk(const TaskDesc* d_tasks, int task0, int n_tasks, uint32_t id_base,
                        const uint64_t* d_tab, const uint64_t* d_mode_tab, const double* d_c,
                        int start_lead, uint64_t seed, uint64_t walkers_per_task,
                        uint64_t id_offset, uint32_t max_steps, unsigned long long* d_counter,
                        uint64_t* d_tally, int32_t* d_trace_lead, uint32_t* d_trace_steps,
                        uint64_t* d_score, uint64_t score_stride, uint64_t* d_mode_score,
                        uint32_t mode_stride, int sm_count, int max_blocks_per_sm,
                        cudaStream_t s, const uint64_t* d_run, int slots, bool two_level) {
  if (n_tasks <= 0 || walkers_per_task == 0) return cudaSuccess;
  const PhiloxKey key{(uint32_t)seed, (uint32_t)(seed >> 32)};
  unsigned long long* tally = reinterpret_cast<unsigned long long*>(d_tally);
  for (int w0 = 0; w0 < n_tasks; w0 += kMaxWindow) {
    const int nt = (n_tasks - w0) < kMaxWindow ? (n_tasks - w0) : kMaxWindow;
    cudaError_t e = cudaMemsetAsync(d_counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const unsigned long long total = (unsigned long long)nt * walkers_per_task;
    // score walks: one slot (a second measured slower), with its path record
    const size_t smem = sizeof(unsigned) * 2 * (size_t)nt * kFields +
                        (d_score ? sizeof(uint32_t) * kPath * kThreads : 0);
    const ScoreOut so{reinterpret_cast<unsigned long long*>(d_score),
                      reinterpret_cast<unsigned long long*>(d_mode_score),
                      (unsigned long long)score_stride, mode_stride};
    auto kern =
        d_score ? (two_level ? (d_trace_lead ? walk_kernel<true, true, 1, true>
                                             : walk_kernel<false, true, 1, true>)
                             : (d_trace_lead ? walk_kernel<true, true, 1, false>
                                             : walk_kernel<false, true, 1, false>))
        : two_level
            ? (slots == 2 ? (d_trace_lead ? walk_kernel<true, false, 2, true>
                                          : walk_kernel<false, false, 2, true>)
                          : (d_trace_lead ? walk_kernel<true, false, 1, true>
                                          : walk_kernel<false, false, 1, true>))
            : (slots == 2 ? (d_trace_lead ? walk_kernel<true, false, 2, false>
                                          : walk_kernel<false, false, 2, false>)
                          : (d_trace_lead ? walk_kernel<true, false, 1, false>
                                          : walk_kernel<false, false, 1, false>));
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem);
    if (e != cudaSuccess) return e;
    if (max_blocks_per_sm > 0 && per_sm > max_blocks_per_sm) per_sm = max_blocks_per_sm;
    if (per_sm < 1) per_sm = 1;
    unsigned long long blocks = (unsigned long long)sm_count * per_sm;
    const unsigned long long need = (total + kThreads - 1) / kThreads;
    if (blocks > need) blocks = need;
    kern<<<(unsigned)blocks, kThreads, smem, s>>>(
        d_tasks, task0 + w0, nt, id_base, d_tab, d_mode_tab, d_c, start_lead, key,
        walkers_per_task, id_offset, max_steps, d_counter, tally + (size_t)w0 * kFields,
        d_trace_lead, d_trace_steps, so, d_run);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (d_mode_score) {
    const uint32_t m2 = 2 * mode_stride;
    mode_reduce_kernel<<<(m2 + 255) / 256, 256, 0, s>>>(
        reinterpret_cast<unsigned long long*>(d_mode_score), m2);
    return cudaGetLastError();
  }
  return cudaSuccess;
}

}  // namespace negf

namespace negf {

cudaError_t probe_gather(uint64_t table_bytes, int ilp, int chain, int sm_count,
                         uint64_t* gathers, float* ms, cudaStream_t s) {
  const uint64_t n = table_bytes / 8;
  if (n < 2 || n > 0xffffffffull || chain < 1) return cudaErrorInvalidValue;
  uint64_t* tab = nullptr;
  unsigned long long* sink = nullptr;
  cudaError_t e = cudaMallocAsync(&tab, n * 8, s);
  if (e == cudaSuccess) e = cudaMallocAsync(&sink, 8, s);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  if (e == cudaSuccess) {
    probe_fill_kernel<<<sm_count * 8, 256, 0, s>>>(tab, n);
    const unsigned blocks = (unsigned)sm_count * 5;
    // warm the table into the cache hierarchy once, then time
    if (ilp >= 4) probe_gather_kernel<8><<<blocks, kThreads, 0, s>>>(tab, (uint32_t)n, 4, sink);
    else probe_gather_kernel<1><<<blocks, kThreads, 0, s>>>(tab, (uint32_t)n, 4, sink);
    cudaEventRecord(a, s);
    if (ilp >= 4) probe_gather_kernel<8><<<blocks, kThreads, 0, s>>>(tab, (uint32_t)n, chain, sink);
    else probe_gather_kernel<1><<<blocks, kThreads, 0, s>>>(tab, (uint32_t)n, chain, sink);
    cudaEventRecord(b, s);
    e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, a, b);
    *gathers = (uint64_t)blocks * kThreads * (ilp >= 4 ? 8 : 1) * (uint64_t)chain;
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (tab) cudaFreeAsync(tab, s);
  if (sink) cudaFreeAsync(sink, s);
  return e;
}

}  // namespace negf
