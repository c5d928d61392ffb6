/*
 * negf.h -- C ABI of the GB300 Monte Carlo NEGF walk library (libnegf.so).
 *
 * Method: Musland, Bergli, Flage-Larsen, "A Monte Carlo method for solving the NEGF equations
 * for electron transport" (arXiv:1805.10164).  The library computes, for wires with Buttiker
 * dephasing probes in the elastic linear-response limit (Sec. II.E-F, III.A):
 *   1. per (wire, energy) task, the retarded Green's function by recursive Green's function
 *      sweeps (Sec. III.B) and from it the Step 6' transition weights (Eq. draw_i_simult and
 *      the lead probability of Step 6') plus the Step 4 injection distribution
 *      (Eq. lead_out_probability), stored as integer alias tables;
 *   2. batches of random walks, one Monte Carlo sample each (Sec. II.D-F), absorbed at a lead;
 *   3. the estimator X_pq = Tr[Gamma_p A] delta_rq (Eq. elast_lin_xpq) tallied into the
 *      transmission T_qp(E) and the lead current of Eq. (iqof_t_el_db) with its binomial
 *      standard error (Sec. IV.B.2).
 * Units: e = h = 1, energies in units of the hopping scale chosen by the caller.
 *
 * Conventions shared by every call
 *  - A context binds one CUDA device and one CUDA stream; all device work of a call is enqueued
 *    on that stream.  Calls that return host data (negf_current, negf_tally_counts,
 *    negf_get_task_info, negf_export_tables) synchronise the stream.  Other calls are asynchronous:
 *    caller-owned device buffers must stay valid until the stream reaches the work.
 *  - Handles (negf_tables, negf_tally) are owned by the library and released with their free
 *    function; freeing NULL is a no-op.  Freeing is stream-ordered.
 *  - Nothing throws across the ABI.  Every call returns a negf_status; on failure the message
 *    is available from negf_last_error(ctx) until the next failing call on that context.
 *  - Numerical failures detected on the device (non-finite Green's function, a table row whose
 *    weights do not sum to a positive value) are recorded in the tables handle and reported as
 *    NEGF_E_NUMERIC by the next synchronising call that uses the handle.
 *  - A context must not be used by two host threads at once.
 */
#ifndef NEGF_H
#define NEGF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define NEGF_ABI_VERSION 6
#define NEGF_MAX_W 64            /* widest supported slice (sites across the wire) */
#define NEGF_MAX_SITES 6400      /* largest W*L per wire with one-level tables */
#define NEGF_MAX_SITES_TWO_LEVEL 65536 /* largest W*L per wire with two-level tables */
#define NEGF_AUTO_TWO_LEVEL_SITES 2048 /* NEGF_LAYOUT_AUTO picks two-level tables above this */
#define NEGF_MAX_STEPS (1u << 24) /* largest accepted per-walk step cap */
#define NEGF_TALLY_FIELDS 5      /* u64 counters per task, see negf_tally_counts */

typedef struct negf_ctx_s* negf_ctx;
typedef struct negf_tables_s* negf_tables;
typedef struct negf_tally_s* negf_tally;

typedef enum {
  NEGF_OK = 0,
  NEGF_E_INVALID = 1,  /* bad argument or input outside the supported domain */
  NEGF_E_NOMEM = 2,    /* device or host allocation failed */
  NEGF_E_CUDA = 3,     /* a CUDA runtime call failed */
  NEGF_E_NUMERIC = 4,  /* non-finite or non-positive quantity found on the device */
  NEGF_E_STEPCAP = 5,  /* some walks reached max_steps; outputs are still written */
  NEGF_E_TIMEOUT = 6   /* a bounded device wait gave up */
} negf_status;

/* Arithmetic of the table build.  NEGF_FP64: everything in FP64 (complex128 blocks).
 * NEGF_FP32: lead self-energies in FP64; the W x W inversions of the RGF sweeps and of the
 * diagonal blocks, the block-column propagation and the transition weights in complex64 /
 * FP32; the sum-rule values <i|A|i>, row sums, mode weights and c_p in FP64; alias thresholds
 * in exact integer arithmetic.  NEGF_SPLIT_TF32: as NEGF_FP32, except that wires of W = 64
 * get two-level tables whose block-column steps G_{k,m} = -t g_k G_{k+1,m} (Sec. III.B) run on
 * the tensor cores as a real GEMM of the complex64 blocks split into TF32 high and low parts
 * (three products, FP32 accumulation).  Measured on GB300, the tensor-core accumulation leaves
 * a systematic relative bias of about 1e-7 per step, so rows whose weight lies hundreds of
 * slices from their start are low by up to ~5e-5 (NEGF_FP32 stays within a few 1e-6). */
typedef enum { NEGF_FP64 = 0, NEGF_FP32 = 1, NEGF_SPLIT_TF32 = 2 } negf_precision;

/* Where the arrays of a negf_wire live. */
typedef enum { NEGF_MEM_HOST = 0, NEGF_MEM_DEVICE = 1 } negf_memspace;

/* Lead model.  NEGF_LEAD_STRIP: exact clean semi-infinite square-lattice strip of the wire's
 * width (onsite 0, hopping -t), diagonal in the transverse sine modes with self-energy
 * t^2 g_s(E - eps_m) per mode.  NEGF_LEAD_WIDE_BAND: the paper's Sigma_p = -(i/2) Gamma_l P_p
 * on the boundary slice (Sec. III.A, lead self energy paragraph). */
typedef enum { NEGF_LEAD_STRIP = 0, NEGF_LEAD_WIDE_BAND = 1 } negf_lead_model;

/* One wire (Sec. III.A model; Buttiker self-energy sigma_i = -i gamma_i / 2, Eq. for sigma_i).
 * Sites are slice-major: site (k, a) of slice k in [0, L) and row a in [0, W) has index k*W+a.
 * Lead L couples to slice 0, lead R to slice L-1.  H has onsite[k*W+a] on the diagonal and -t
 * between nearest neighbours along and across the slices. */
typedef struct {
  int32_t W, L;                  /* 1 <= W <= NEGF_MAX_W, L >= 1, W*L <= NEGF_MAX_SITES
                                    (one-level tables) or NEGF_MAX_SITES_TWO_LEVEL (two-level) */
  double t;                      /* hopping magnitude, > 0 */
  const double* onsite;          /* [L*W] onsite energies, finite */
  const double* eta;             /* [L*W] Buttiker gamma_i >= 0, finite */
  int32_t n_energy;              /* >= 0 */
  const double* energy;          /* [n_energy]; for NEGF_LEAD_STRIP no energy may lie within
                                    1e-12*t of a lead sub-band edge |E - eps_m| = 2t */
  const double* energy_weight;   /* [n_energy] quadrature weights, or NULL for all 1 */
  int32_t lead_model;            /* negf_lead_model */
  double gamma_lead;             /* Gamma_l for NEGF_LEAD_WIDE_BAND, > 0 */
  const double* slice_h;         /* NULL: the square-lattice cross-section above.  Else a
                                    multi-orbital slice (the "more orbitals per atom"
                                    generalisation of the Hamiltonian; W counts orbitals):
                                    [W*W] row-major real symmetric block h, and H_kk = h +
                                    diag(onsite of slice k); the coupling between slices stays
                                    -t between the same orbital of neighbouring slices.  The
                                    exact strip lead is then the clean strip of h: its modes
                                    are h's eigenvectors (computed on the device), eps_m its
                                    eigenvalues.  Same memspace as the other arrays; must be
                                    finite and exactly symmetric (NEGF_E_INVALID). */
} negf_wire;

typedef struct {
  int32_t precision;    /* negf_precision */
  int32_t memspace;     /* negf_memspace of every array in the wires */
  int32_t keep_weights; /* nonzero: keep the FP transition weights (negf_export_tables) and
                           the transverse modes, as negf_current_backward_rgf needs them */
  int32_t keep_green;   /* nonzero: also keep G (dense n x n per task), G Phi, the weights and
                           the transverse modes, as negf_current_backward needs them */
  int32_t table_layout; /* negf_table_layout */
} negf_build_opts;

/* Layout of the Step 6' tables of a task.
 * One-level: one alias row of K = n + 2 slots per table row (draw: one 8-byte entry).
 * Two-level: the draw over the n + 2 outcomes factorises exactly into a level-1 draw over the L
 * slices and the two leads (weights: the slice totals of the row and the lead weights; an
 * alias row of L + 2 slots) and, for a slice k, a level-2 draw over the W sites of that slice
 * (weights: the row's weights of those sites) by the inverse-CDF search of Sec. III.B in
 * integers.  A level-2 block holds G = ceil(W/8) octets of 31-bit cumulative thresholds
 * c_a = floor(2^31 P_a / S) (P_a the sum of the slice's weights up to site a, S their total;
 * c_{W-1} and the padding of the last octet are 2^31) and, for W > 8, an 8-word guide in front
 * (guide_g = c_{8g+7} for g < G - 1, then 2^31): NEGF_LEVEL2_WORDS(W) = 8 (W <= 8) or 8 + 8G
 * u32.  A draw with v uniform on [0, 2^31) takes g = #{guide words <= v}, then site
 * 8g + #{words of octet g <= v}: site a has probability (c_a - c_{a-1}) / 2^31.  Entries:
 * level 2 u32 [rows][L][NEGF_LEVEL2_WORDS(W)] (starting on a 32-byte boundary), level 1 u64
 * [rows][L + 2].  The build needs no per-row shared-memory pass over n + 2 entries (a one-level
 * row of K slots is built by one warp with 32 K bytes of shared memory, which leaves few warps
 * per SM once K is in the thousands) and level 2 costs a prefix sum per slice, which makes it
 * the layout of long wires.  NEGF_LAYOUT_AUTO: two-level when W*L > NEGF_AUTO_TWO_LEVEL_SITES,
 * or for W = 64 wires built with NEGF_SPLIT_TF32. */
#define NEGF_LEVEL2_WORDS(W) ((W) <= 8 ? 8 : 8 + 8 * (((W) + 7) / 8))
typedef enum { NEGF_LAYOUT_AUTO = 0, NEGF_LAYOUT_ONE_LEVEL = 1, NEGF_LAYOUT_TWO_LEVEL = 2 } negf_table_layout;

/* Per-task facts, read back from the device (synchronises). */
typedef struct {
  int32_t wire, energy_index;
  int32_t W, L, n;       /* n = W*L sites */
  int32_t K;             /* row length = n + 2 (sites, then lead L, lead R) */
  int32_t rows;          /* n site rows, then W injection rows of lead L, W of lead R */
  int32_t table_layout;  /* NEGF_LAYOUT_ONE_LEVEL or NEGF_LAYOUT_TWO_LEVEL */
  double energy, energy_weight;
  double c[2];           /* Tr[Gamma_p A] for p = L (0) and R (1), Eq. elast_lin_xpq */
  uint64_t table_offset; /* first entry of this task's rows x K block (weights, score
                            tallies; either layout) */
  uint64_t mode_offset;  /* first entry of this task's 2 x W block (mode tables / tallies) */
} negf_task_info;

/* --- context -------------------------------------------------------------------------- */

/* Create a context on CUDA device `device` enqueuing on `stream` (a cudaStream_t, NULL for the
 * legacy default stream).  The stream must outlive the context.  Device buffers of the library
 * come from the device's default stream-ordered memory pool; creating a context sets that
 * pool's release threshold to "keep everything" so repeated builds reuse their memory. */
negf_status negf_create(negf_ctx* out, int device, void* stream);
void negf_destroy(negf_ctx ctx);
const char* negf_last_error(negf_ctx ctx);
int negf_abi_version(void);

/* --- tables (Sec. III.B and Step 6') -------------------------------------------------- */

/* Build the transition tables of every (wire, energy) task.  Tasks are numbered wire-major:
 * all energies of wire 0, then wire 1, ...  Inputs are read during the call (host arrays) or by
 * the enqueued work (device arrays).  Per task the handle holds (rows x K) alias entries
 * (u64: low 32 bits threshold, high 32 bits alias; Sec. III.B inverse-CDF draw replaced by
 * Walker's alias method), 2 x W injection-mode alias entries and c[2].
 * Errors: NEGF_E_INVALID for bad sizes/values (host memspace checks every value; device
 * memspace checks sizes here and values on the device, reported later as NEGF_E_INVALID by the
 * next synchronising call), NEGF_E_NOMEM, NEGF_E_CUDA. */
negf_status negf_build_tables(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                              const negf_build_opts* opts, negf_tables* out);
int32_t negf_tables_num_tasks(negf_tables tables);
int32_t negf_tables_num_wires(negf_tables tables);
/* Device bytes held by the handle (tables, scratch kept, descriptors). */
uint64_t negf_tables_device_bytes(negf_tables tables);
negf_status negf_get_task_info(negf_ctx ctx, negf_tables tables, int32_t task,
                               negf_task_info* out);
void negf_tables_free(negf_tables tables);

/* Copy one task's data to host memory.  `what`:
 *   NEGF_EXPORT_ALIAS       u64 [rows*K]  alias entries, row-major (two-level tasks: the level-2
 *                                         blocks u32 [rows][L][NEGF_LEVEL2_WORDS(W)])
 *   NEGF_EXPORT_ALIAS_LEVEL1 u64 [rows][L+2] level-1 entries of a two-level task
 *   NEGF_EXPORT_MODE_ALIAS  u64 [2*W]     injection-mode alias entries, lead L then R
 *   NEGF_EXPORT_WEIGHTS     f64 [rows*K]  transition weights (needs keep_weights)
 *   NEGF_EXPORT_MODE_WEIGHTS f64 [2*W]    lambda_m <phi_m|A|phi_m> (Eq. lead_out_probability)
 *   NEGF_EXPORT_ROWSUM      f64 [rows]    FP64 sum of each row's weights (= <i|A|i>)
 * If host_buf is NULL, *bytes receives the size needed.  Otherwise *bytes must be at least
 * that size (NEGF_E_INVALID if not) and receives the bytes written.  Synchronises. */
enum { NEGF_EXPORT_ALIAS = 0, NEGF_EXPORT_MODE_ALIAS = 1, NEGF_EXPORT_WEIGHTS = 2,
       NEGF_EXPORT_MODE_WEIGHTS = 3, NEGF_EXPORT_ROWSUM = 4, NEGF_EXPORT_ALIAS_LEVEL1 = 5 };
negf_status negf_export_tables(negf_ctx ctx, negf_tables tables, int32_t task, int32_t what,
                               void* host_buf, size_t* bytes);
/* Rows [row0, row0 + n_rows) of one task's NEGF_EXPORT_ALIAS, NEGF_EXPORT_ALIAS_LEVEL1 or
 * NEGF_EXPORT_ROWSUM data (same per-row layout as negf_export_tables: a two-level row's level 2
 * is L * NEGF_LEVEL2_WORDS(W) u32), for tables too large to copy whole.  Buffer sizing and errors as negf_export_tables; rows outside [0, rows) or
 * another kind give NEGF_E_INVALID.  Synchronises. */
negf_status negf_export_table_rows(negf_ctx ctx, negf_tables tables, int32_t task, int32_t what,
                                   int64_t row0, int64_t n_rows, void* host_buf, size_t* bytes);

/* --- walks (Sec. II.D Steps 1-4, Sec. II.F Step 6') ------------------------------------ */

/* Run walkers_per_task walks in every task, all starting at lead start_lead (0 = L, 1 = R;
 * the paper keeps the initial lead fixed, Sec. II.E).  Walker w of task k has id
 * walker_id_offset + w; its draw s uses Philox4x32-10 block s/2 with counter
 * (s/2, id_lo, id_hi, k) and key (seed_lo, seed_hi), words (x0,x1) for even s and (x2,x3) for
 * odd s.  Draw 0 picks the injection mode, draws 1.. are Step 6' transitions (steps).  A walk
 * stops when a lead is drawn or after max_steps steps (then it counts as truncated).
 * Results from disjoint id ranges add up exactly (negf_tally_accumulate), so runs can be split
 * or resumed.  1 <= max_steps <= NEGF_MAX_STEPS.  A new tally handle is returned in *out. */
negf_status negf_walk(negf_ctx ctx, negf_tables tables, int32_t start_lead, uint64_t seed,
                      uint64_t walkers_per_task, uint64_t walker_id_offset, uint32_t max_steps,
                      negf_tally* out);

/* Same walks for one task, recording each walker's outcome: d_lead[w] = 0 (L), 1 (R),
 * -1 (no open channel in the start lead: nothing injected), -2 (truncated); d_steps[w] = steps.
 * d_lead / d_steps are caller-owned device arrays of n_walkers entries. */
negf_status negf_walk_trace(negf_ctx ctx, negf_tables tables, int32_t task, int32_t start_lead,
                            uint64_t seed, uint64_t walker_id_offset, uint64_t n_walkers,
                            uint32_t max_steps, int32_t* d_lead, uint32_t* d_steps);

/* Per-task counters [n_tasks][NEGF_TALLY_FIELDS] u64: walkers done, absorbed at L, absorbed at
 * R, truncated, sum of steps.  Synchronises. */
negf_status negf_tally_counts(negf_ctx ctx, negf_tally tally, uint64_t* host_counts);
/* Add host counters (same layout) into a tally, e.g. from another rank or an earlier run. */
negf_status negf_tally_accumulate(negf_ctx ctx, negf_tally tally, const uint64_t* host_counts);
int32_t negf_tally_start_lead(negf_tally tally);
void negf_tally_free(negf_tally tally);

/* --- batched build + walk pipeline ------------------------------------------------------ */

typedef struct {
  int32_t start_lead;          /* 0 = L, 1 = R (as in negf_walk) */
  int32_t tasks_per_wave;      /* tasks built per wave; 0 = about an eighth of the tasks */
  uint64_t seed;
  uint64_t walkers_per_task;
  uint64_t walker_id_offset;
  uint32_t max_steps;          /* 1 <= max_steps <= NEGF_MAX_STEPS */
  int32_t waves_in_flight;     /* waves whose tables may coexist; 0 = 2 */
  uint64_t memory_budget;      /* bytes of tables + scratch in flight; 0 = half the free memory */
  int32_t walk_blocks_per_sm;  /* cap of the walk grid per SM; 0 = as many as fit */
  int32_t reserved;            /* must be 0 */
} negf_run_opts;

/* The whole hot path for a batch of wires of any sizes (paper silent; Sec. IV runs many
 * independent samples side by side): tasks are split into waves of consecutive tasks whose
 * tables fit the memory budget; wave w+1 is built on the context stream while wave w walks on
 * a second stream of the context, and each wave's tables are freed as soon as its walks are
 * done.  Walks are identical to negf_build_tables + negf_walk with the same seed and walker
 * ids (the Philox task number is the task's index in the batch), so tallies agree bit for bit.
 * Returns a task handle (descriptors and c_p; its alias tables are released, so
 * NEGF_EXPORT_ALIAS / NEGF_EXPORT_ROWSUM are refused) and the tally, both usable with
 * negf_current.  Asynchronous like negf_build_tables (host inputs are read during the call). */
negf_status negf_run(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                     const negf_build_opts* build, const negf_run_opts* run,
                     negf_tables* out_tasks, negf_tally* out_tally);
int32_t negf_tables_num_waves(negf_tables tables);

/* --- captured plans (CUDA graph) and launch-shape autotuning -------------------------------- */

typedef struct negf_plan_s* negf_plan;

/* Launch shapes of a plan.  Picked by timing candidates on the plan's first wave when
 * negf_plan_create is asked to autotune, else the built-in defaults (0 = default). */
typedef struct {
  int32_t walk_blocks_per_sm;   /* CTAs per SM of the persistent walk grid */
  int32_t chain_warps;          /* warps per CTA of the block-column chain kernel */
  int32_t alias_warps;          /* warps per CTA of the alias kernel */
  int32_t tuned;                /* 1 when picked by the autotuner */
  float walk_ms, chain_ms, alias_ms;   /* device time of the chosen shapes while tuning */
  int32_t walk_slots;           /* walks in flight per lane of the walk kernel (1 or 2); 0 =
                                   by the wave's tables: 2 with two-level tables, else 1 */
} negf_plan_tuning;

/* A plan is the whole path of negf_run followed by negf_current — lead modes, RGF sweeps,
 * block columns, Step 6' weights, alias tables, walks, tally, current and standard error —
 * for a fixed batch of wires (paper silent: Sec. IV repeats the same calculation for many
 * samples), captured once into a CUDA graph over buffers allocated here, and relaunched by
 * negf_plan_launch with a new seed and walker-id range.  build->memspace: for
 * NEGF_MEM_DEVICE every launch re-reads the wires' onsite and eta arrays, which must stay
 * allocated at the same addresses until negf_plan_destroy; host arrays, energies and energy
 * weights are read once here.  run: start_lead, tasks_per_wave (0 = all tasks in one wave),
 * walkers_per_task, max_steps, waves_in_flight, memory_budget as in negf_run; run->seed and
 * run->walker_id_offset are ignored (given per launch); walk_blocks_per_sm > 0 overrides the
 * tuned value.  mu_p, mu_q, kT: as negf_current.  autotune nonzero: time candidate launch
 * shapes on the first wave first (one build and a few walks of that wave).  keep_weights and
 * keep_green must be 0.  Device memory: every wave slot's tables and scratch stay allocated
 * (negf_plan_device_bytes).  Synchronises the context stream. */
negf_status negf_plan_create(negf_ctx ctx, const negf_wire* wires, int32_t n_wires,
                             const negf_build_opts* build, const negf_run_opts* run,
                             double mu_p, double mu_q, double kT, int32_t autotune,
                             negf_plan* out);
/* Enqueue one launch of the plan on the context stream: walkers
 * [walker_id_offset, walker_id_offset + walkers_per_task) of every task, Philox key seed.
 * Tallies and walks equal those of negf_run / negf_build_tables + negf_walk with the same
 * seed and walker ids.  Asynchronous (with profiling enabled it waits for the launch and adds
 * the kernel groups' device times to the context's profile). */
negf_status negf_plan_launch(negf_ctx ctx, negf_plan plan, uint64_t seed,
                             uint64_t walker_id_offset);
/* Results of the last launch (synchronises): I, se [n_wires], T, T_se [n_tasks], counts
 * [n_tasks][NEGF_TALLY_FIELDS]; any pointer may be NULL.  Returns NEGF_E_STEPCAP (results
 * written) when walks were cut at max_steps, NEGF_E_INVALID / NEGF_E_NUMERIC for device-side
 * input or numerical errors of the launch. */
negf_status negf_plan_result(negf_ctx ctx, negf_plan plan, double* I, double* se, double* T,
                             double* T_se, uint64_t* counts);
negf_status negf_plan_get_tuning(negf_plan plan, negf_plan_tuning* out);
int32_t negf_plan_num_tasks(negf_plan plan);
int32_t negf_plan_num_waves(negf_plan plan);
uint64_t negf_plan_device_bytes(negf_plan plan);
void negf_plan_destroy(negf_plan plan);

/* --- inelastic Buttiker probes (Sec. II.F, Step 7') ----------------------------------------- */

/* Walks in which the walker's energy changes at every probe it visits (Step 7', Eq.
 * draw_E_last): after Step 6' has drawn a site j at the walker's grid energy E_e, the next
 * energy E_e' of the wire's grid is drawn with probability proportional to
 * w_e' exp(-(E_e' - E_e)^2 / (2 sigma_E^2)) A_jj(E_e') (w_e' the energy's weight from
 * negf_wire.energy_weight, A_jj the row sum of site row j at E_e'; sigma_E = 0: the same energy,
 * the elastic walk's law).  This is Buttiker's inelastic probe with the redistribution rate
 * lambda~_j(E', E) = eta_j K(E' - E) / sum_E'' w K(E'' - E) A_jj(E''), which satisfies the
 * charge-conservation condition (Eq. condition4_buttiker) with gamma_j = eta_j, so the Step 6'
 * tables of every energy are the elastic ones.  Walker ids, seeds, max_steps and the tally are
 * as for negf_walk; counts go to the injection task, so that negf_current gives
 * T_qp(E_0) = c_p(E_0) P(q | p, E_0) per injection energy.  Random numbers: Philox block 0 is
 * the injection draw; block s >= 1 is transition s, words (x0, x1) for the next index from the
 * row at the walker's energy, (x2, x3) for the next energy from the energy row of the site
 * drawn.  Needs one-level tables (NEGF_E_INVALID for two-level ones) with every grid energy of
 * a wire in the same handle; sigma_E finite and >= 0.  The energy rows ([sites][nE] alias rows
 * per task, built on the device for the call) are freed before it returns. */
negf_status negf_walk_inelastic(negf_ctx ctx, negf_tables tables, int32_t start_lead,
                                uint64_t seed, uint64_t walkers_per_task,
                                uint64_t walker_id_offset, uint32_t max_steps, double sigma_E,
                                negf_tally* out);
/* The Step 7' energy rows of task `task` (the wire's energy E_e of that task): host_buf gets
 * n x nE alias entries (site-major; entry = threshold | alias << 32 over the wire's nE grid
 * energies), built as negf_walk_inelastic builds them.  host_buf NULL: *bytes receives the size
 * needed.  Synchronises. */
negf_status negf_export_energy_tables(negf_ctx ctx, negf_tables tables, int32_t task,
                                      double sigma_E, void* host_buf, size_t* bytes);

/* --- gradient (paper silent) ---------------------------------------------------------------- */

/* negf_walk that also records score tallies: for every walk absorbed at lead r each transition
 * a -> b adds 1 to counts[r][table_offset + a K + b] of its task (b a site, or n + r' for lead
 * r'; the same rows x K numbering for one- and two-level tables), its injection mode m to
 * mode_counts[r][mode_offset + p W + m] (offsets from negf_get_task_info).  A walk's transitions
 * are recorded as it walks (up to 128; longer walks are replayed from their first draw), the
 * same walks as negf_walk with the same arguments.  The tables must still hold their alias rows
 * (negf_build_tables). */
negf_status negf_walk_score(negf_ctx ctx, negf_tables tables, int32_t start_lead, uint64_t seed,
                            uint64_t walkers_per_task, uint64_t walker_id_offset,
                            uint32_t max_steps, negf_tally* out);
/* Score tallies of a tally from negf_walk_score: host_counts [2][negf_tally_score_size] and
 * host_mode_counts [2][negf_tally_mode_size] (lead-major).  Synchronises. */
negf_status negf_tally_score_counts(negf_ctx ctx, negf_tally tally, uint64_t* host_counts,
                                    uint64_t* host_mode_counts);
/* Add host score counts (same layout) into the tally: merges runs over disjoint walker ids. */
negf_status negf_tally_score_accumulate(negf_ctx ctx, negf_tally tally,
                                        const uint64_t* host_counts,
                                        const uint64_t* host_mode_counts);
uint64_t negf_tally_score_size(negf_tally tally);
uint32_t negf_tally_mode_size(negf_tally tally);

/* Gradient of the Monte Carlo current of every wire (as negf_current with the same mu, kT)
 * w.r.t. the onsite energies and the Buttiker dephasing of every site:
 *   d_onsite[s] = sum_w dI[w] dI_w/dV_s,   d_eta[s] = sum_w dI[w] dI_w/deta_s,
 * sites s numbered wire after wire (wire w's L*W sites follow those of wires < w).  The
 * transmission's derivative is the score-function estimator dT = dc_p P + c_p
 * E[(1_q - P) d log p(path)] from the score tallies, pushed through the tables' dependence on
 * G and of G on the parameters (dG = G e_k e_k^T G, resp. -(i/2) G e_k e_k^T G).  Requires
 * tables built with keep_green and a tally from negf_walk_score.  dI [n_wires], d_onsite and
 * d_eta are host arrays.  Returns NEGF_E_STEPCAP (after writing the outputs) if walks were
 * truncated.  Synchronises. */
negf_status negf_current_backward(negf_ctx ctx, negf_tables tables, negf_tally tally,
                                  double mu_p, double mu_q, double kT, const double* dI,
                                  double* d_onsite, double* d_eta);

/* The same gradient (same arguments, outputs, seeds and errors as negf_current_backward)
 * without any dense G: per block column m of slice m, G[:, m] from the RGF relations of
 * Sec. III.B (G_{k,m} = -t g^L_k G_{k+1,m} below m, -t g^R_k G_{k-1,m} above), the matching
 * column of the seed matrix, G times it by block-tridiagonal elimination with the
 * left-connected blocks, and the diagonal of G Gbar G accumulated column by column (about
 * 3 L^2 W^3 complex multiply-adds per task).  The left- and right-connected blocks are swept
 * once and kept only at every ckpt_stride-th slice (0: NEGF_CKPT_STRIDE_DEFAULT); the blocks
 * between are recomputed per segment before a task's columns run.  Requires tables built with
 * keep_weights (FP64 or FP32, one- or two-level layout; split-TF32 tables keep no weights:
 * NEGF_E_INVALID) and a tally from negf_walk_score on them.  ckpt_stride < 0: NEGF_E_INVALID.
 * Device scratch: at most half the free device memory (16 GiB at most).  Synchronises. */
#define NEGF_CKPT_STRIDE_DEFAULT 10
negf_status negf_current_backward_rgf(negf_ctx ctx, negf_tables tables, negf_tally tally,
                                      double mu_p, double mu_q, double kT, const double* dI,
                                      int32_t ckpt_stride, double* d_onsite, double* d_eta);

/* --- current (Eq. iqof_t_el_db, Eq. elast_lin_xpq, Sec. IV.B.2) --------------------------- */

/* From a tally of walks started at lead p = start_lead, with absorbing lead q = 1 - p:
 *   T_qp(task) = c_p n_q / N,  SE = c_p sqrt(P (1-P) / N)  (P = n_q / N, N = walkers done),
 *   I(wire) = sum_E w_E (f(E; mu_p, kT) - f(E; mu_q, kT)) T_qp(E),
 *   SE(I)^2 = sum_E (w_E (f_p - f_q))^2 SE(T_qp(E))^2,
 * computed on the device in FP64.  Host outputs: I[n_wires], se[n_wires]; T[n_tasks] and
 * T_se[n_tasks] may be NULL.  Returns NEGF_E_STEPCAP (after writing the outputs) if any walk
 * was truncated.  Synchronises. */
negf_status negf_current(negf_ctx ctx, negf_tables tables, negf_tally tally, double mu_p,
                         double mu_q, double kT, double* I, double* se, double* T,
                         double* T_se);

/* --- linear conductance with continuous energies (Eq. Gqp_expression, Eq. gpq_formula,
 *     Eq. elast_lin_xpq; Sec. "Interpolation") ------------------------------------------- */

/* Result of negf_walk_thermal.  G and se are in units of e^2/h. */
typedef struct {
  double G;              /* estimate of the integral over [E_0, E_{M-1}] of Th(E) T_qp(E) dE */
  double se;             /* its standard error (sample standard deviation / sqrt(walkers)) */
  double window;         /* F(E_{M-1}) - F(E_0): the share of Th inside the grid's span */
  double mean_steps;     /* transitions per walker (absorbed or truncated) */
  uint64_t walkers;      /* walkers run */
  uint64_t absorbed[2];  /* absorbed at lead L, R */
  uint64_t closed;       /* no open channel at either grid energy around E_0 (X = 0) */
  uint64_t truncated;    /* reached max_steps */
} negf_thermal_result;

/* The linear conductance G_qp = integral dE T_qp(E) Th(E), Th = -df/dE (Eq. Gqp_expression),
 * sampled as the paper does (Eq. gpq_formula, Eq. elast_lin_xpq): each walker draws its energy
 * E_0 from Th, restricted to the span [E_0, E_{M-1}] of wire `wire`'s energy grid (the M >= 2
 * energies of that wire in the tables, strictly ascending, all of one layout), and walks the
 * Markov chain whose Step 6' transition probabilities are interpolated linearly between the two
 * grid energies around E_0 (the paper's interpolation of the p_i, Sec. "Interpolation"): every
 * draw uses the table of the upper grid energy with probability alpha = (E_0 - E_i) /
 * (E_{i+1} - E_i), else the lower one; the injection mode likewise.  Where the start lead has
 * no open channel at one end (Tr Gamma_p A = 0 there), the interval walks with the other end's
 * tables alone (a chain without an open lead never absorbs); closed at both ends, X = 0.
 * A walker absorbed at q = 1 - start_lead scores
 * X = (1 - alpha) c_i + alpha c_{i+1} (c = Tr Gamma_p A); G = window * mean(X).
 * Th is the logistic density with scale kT around mu (Fermi function at mu, kT).
 * Random numbers: walker w (id walker_id_offset + w) takes Philox4x32-10 block b with counter
 * (b, id_lo, id_hi, 0x80000000 | wire) and key (seed_lo, seed_hi): block 0 words (x0, x1) give
 * u = (((x0 << 32 | x1) >> 11) + 1/2) / 2^53, the CDF value F = F(E_0) + u window of the drawn
 * energy (FP64, each operation rounded; its interval i: F(E_i) <= F < F(E_{i+1}), decided
 * exactly; alpha from F^-1(F) in FP32, to ~2^-20), word x2 the
 * injection table (upper iff x2 < a, a = min(floor(alpha 2^32), 2^32 - 1)); block 1 the injection
 * mode (x0, x1); block b >= 2 transition b - 1 ((x0, x1) on the row, x2 < a picks the table;
 * two-level tables: (x0, x1) on the level-1 row and v = x3 >> 1 for the site of a drawn slice).
 * d_lead, d_steps, d_interval, d_a: optional caller-owned device arrays of `walkers` entries
 * (any may be NULL) receiving each walker's outcome (0 / 1 lead, -1 closed, -2 truncated),
 * transitions, grid interval i and a.  Allocates a small tally on the context stream, runs on it
 * and synchronises.  Errors: NEGF_E_INVALID for bad handles, wire out of range, fewer than two
 * energies, energies not strictly ascending, one- and two-level tables mixed, tables released
 * by negf_run,
 * kT <= 0, non-finite mu, walkers above 2^40, max_steps outside [1, NEGF_MAX_STEPS];
 * NEGF_E_NOMEM; NEGF_E_CUDA. */
negf_status negf_walk_thermal(negf_ctx ctx, negf_tables tables, int32_t wire, int32_t start_lead,
                              uint64_t seed, uint64_t walkers, uint64_t walker_id_offset,
                              double mu, double kT, uint32_t max_steps, int32_t* d_lead,
                              uint32_t* d_steps, int32_t* d_interval, uint32_t* d_a,
                              negf_thermal_result* out);

/* Distances between the Step 6' probabilities of consecutive energies of wire `wire` (the
 * paper interpolates the probabilities between two nearby energies where they differ by less
 * than five percent, Sec. "Interpolation"): for energies e, e + 1 of the wire (in the order
 * given), d[e] = the largest of (1) the total-variation distance (1/2) sum_b |P_ab(e) -
 * P_ab(e+1)| of every table row a (P = weights / row sum; a row of zero sum counts as zero),
 * (2) the same between the injection-mode distributions of lead start_lead, (3) |c_e -
 * c_{e+1}| / max(c_e, c_{e+1}) for c = Tr[Gamma_p A] (0 when both vanish).  d: host array of
 * n_energy - 1 doubles.  Needs tables built with keep_weights.  Synchronises.  Errors:
 * NEGF_E_INVALID (bad handle or wire, fewer than two energies, weights not kept), NEGF_E_CUDA. */
negf_status negf_interval_distance(negf_ctx ctx, negf_tables tables, int32_t wire,
                                   int32_t start_lead, double* d);

/* The energy grid of the interpolating sampler (Sec. "Interpolation"): start from n_init
 * evenly spaced energies on [e_lo, e_hi] (the last one e_hi exactly); in each round, build the
 * wire's tables on the current grid (host arrays, as NEGF_MEM_HOST; the wire's own energies
 * and weights are ignored) and split every interval whose negf_interval_distance exceeds tol
 * at its midpoint (E_i + E_{i+1}) / 2, in grid order, while the grid holds fewer than
 * max_points energies; stop when every interval passes or no point can be added.  energies:
 * host array of max_points doubles receiving the ascending grid, *n_out its length.  The
 * grid is for negf_build_tables + negf_walk_thermal.  Synchronises.  Errors: NEGF_E_INVALID
 * for e_lo >= e_hi, n_init < 2, max_points < n_init, tol <= 0, and as negf_build_tables. */
negf_status negf_thermal_grid(negf_ctx ctx, const negf_wire* wire, int32_t precision, double e_lo,
                              double e_hi, int32_t n_init, double tol, int32_t max_points,
                              int32_t start_lead, double* energies, int32_t* n_out);

/* --- table build without device allocation ------------------------------------------------ */

/* The paper has no counterpart to this entry point; it exists for callers of this library that
 * cannot allocate device memory themselves or let a library do it: a host framework that owns
 * every device byte through its own pool, a process whose device footprint must not grow after
 * start-up, or code enqueuing work where a cudaMalloc would synchronise the device.
 *
 * It builds the one-level tables negf_build_tables builds for ONE wire (host arrays, as with
 * NEGF_MEM_HOST; energy_weight is ignored and never read) with the same kernels, block-column
 * chains included, so the alias entries are bit-identical; but it allocates nothing: all
 * scratch (task descriptors, lead self-energies, RGF blocks, FP weights, row sums, chain jobs)
 * lives in one file-scope device array of NEGF_NOALLOC_SCRATCH_BYTES (64 MiB) that every device
 * which loads the library holds until the process exits.  Inputs are copied into that array;
 * results go to caller-owned device buffers:
 *   d_alias       u64 [n_energy][rows][K]  alias entries (layout of NEGF_EXPORT_ALIAS per task,
 *                                          rows = W*L + 2W, K = W*L + 2)
 *   d_mode_alias  u64 [n_energy][2][W]     injection-mode alias entries
 *   d_c           f64 [n_energy][2]        Tr[Gamma_p A] for p = L, R
 * precision: NEGF_FP64 or NEGF_FP32 (NEGF_SPLIT_TF32 computes as NEGF_FP32 here, where
 * negf_build_tables would build two-level tables on the tensor cores for W = 64).
 * The call runs on `stream` (a cudaStream_t on the current device) and synchronises it before
 * returning, so device-side failures are reported by its status.
 * Limits and errors: 1 <= n_energy <= NEGF_NOALLOC_MAX_TASKS and W*L <= NEGF_MAX_SITES, else
 * NEGF_E_INVALID; a problem whose scratch exceeds the fixed array returns NEGF_E_NOMEM (split
 * the energies over several calls); bad values as for negf_build_tables (NEGF_E_INVALID);
 * NEGF_E_NUMERIC for device-detected numerical failures; NEGF_E_CUDA for runtime failures.
 * Every call looks up the array's device address on the current device (cudaGetSymbolAddress,
 * so the address stays right after a cudaDeviceReset); the first lookup on a device sets up
 * the library's device code there, so make the first call on each device before any stream
 * capture.  Every call uses the
 * same array, which keeps the previous call's contents (the parts that must start at zero are
 * cleared by each call): calls that overlap on the GPU - from two host threads, or on two
 * streams of one device - race on the array and corrupt each other's results. */
#define NEGF_NOALLOC_SCRATCH_BYTES (64u << 20)
#define NEGF_NOALLOC_MAX_TASKS 256
negf_status negf_build_tables_noalloc(const negf_wire* wire, int32_t precision, void* stream,
                                      uint64_t* d_alias, uint64_t* d_mode_alias, double* d_c);

/* --- device error words (paper silent) ------------------------------------------------------ */

/* Kernels record failures by OR-ing bits into a device word of the handle (or plan, or call)
 * that the next synchronising call reads: 1 a non-finite Green's function block or weight,
 * 2 a table row whose weights do not sum to a positive value, 4 a device-resident input outside
 * the domain, 8 a singular slice block, 16 a bounded device wait (the mbarrier waits of the
 * tensor-core kernels) that gave up.  Returns the status such a word is reported as: NEGF_OK
 * for 0, else NEGF_E_INVALID if bit 4 is set, else NEGF_E_TIMEOUT if bit 16 is set, else
 * NEGF_E_NUMERIC.  If msg is non-NULL and cap > 0, msg receives the description (truncated to
 * cap - 1 bytes, NUL-terminated).  Host only: touches no device. */
negf_status negf_device_error_status(int32_t word, char* msg, size_t cap);

/* --- profiling (CUDA events around every kernel launch) ----------------------------------- */

/* Turn per-kernel device-time accounting on (on != 0) or off; either way the counters reset.
 * While on, each kernel launch of the context is bracketed by two CUDA events on the context
 * stream. */
negf_status negf_profile_enable(negf_ctx ctx, int32_t on);
/* Read the counters (synchronises on the recorded events): for i < min(cap, *n_out) entries,
 * names[32*i ..] receives the kernel name (NUL-terminated), launches[i] the number of kernel
 * launches and total_ms[i] their summed device time.  *n_out = number of entries. */
negf_status negf_profile_read(negf_ctx ctx, int32_t cap, char* names, uint64_t* launches,
                              double* total_ms, int32_t* n_out);

/* Measurement aid (no counterpart in the paper): random 8-byte gathers over a device table of
 * table_bytes, each thread following `ilp` independent chains (1 or 8) of `chain` dependent
 * loads, on a grid shaped like the walk's.  Returns the achieved gathers per second, the
 * ceiling the walk's alias-entry loads are compared with.  Allocates and frees its table on
 * the context stream and synchronises it. */
negf_status negf_probe_gather(negf_ctx ctx, uint64_t table_bytes, int32_t ilp, int32_t chain,
                              double* gathers_per_s);

#ifdef __cplusplus
}
#endif
#endif /* NEGF_H */
