/*
 * tto.h -- C ABI of the B300 DC N-1 topology evaluator and MapElites search.
 *
 * The library evaluates candidate switching topologies (substation bus splits,
 * two-node operation) of a transmission grid by DC loadflow with full N-1
 * contingency analysis (paper Sec. "DC-Optimizer": PTDF-based flows with
 * low-rank topology updates), reduces each topology to the overload metrics of
 * Sec. "Fitness function heuristics" and the MapElites descriptors of Sec.
 * "Repertoire design", and runs the mutation and archive insert of Algorithms
 * 1 and 3 on the device.
 *
 * Conventions for every call:
 *   - return 0 (TTO_OK) on success, a negative TTO_E_* code otherwise; the
 *     thread-local message of the last failure is tto_last_error();
 *   - "host" pointers are read during the call only; "device" pointers are CUDA
 *     device memory owned by the caller, accessed asynchronously on the given
 *     stream (a cudaStream_t passed as void*; NULL = legacy default stream);
 *   - there is no CPU fallback: without a usable CUDA device every call that
 *     needs one returns TTO_E_CUDA.
 */
#ifndef TTO_H
#define TTO_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TTO_OK 0
#define TTO_E_ARG (-1)          /* invalid argument or inconsistent input */
#define TTO_E_DISCONNECTED (-2) /* the unsplit grid is not connected */
#define TTO_E_CUDA (-3)         /* CUDA runtime failure or no device */
#define TTO_E_NOMEM (-4)        /* host or device allocation failed */
#define TTO_E_TOPOLOGY (-5)     /* a genome named an unknown action or split a station twice */
#define TTO_E_TIMEOUT (-6)      /* a bounded device wait gave up */

#define TTO_MAX_K 8        /* split slots per genome */
#define TTO_MAX_T 32       /* timesteps per evaluation call */
#define TTO_MAX_ASSETS 16  /* assets per splittable station */

/* Precision of the low-rank term U V^T of the N-1 sweep (flows are FP32 and the
 * split/outage denominators FP64 in every mode). */
#define TTO_PREC_FP32 0    /* FP32 FMAs on the CUDA cores */
#define TTO_PREC_BF16X3 1  /* tensor cores, BF16 hi/lo split (3 products), FP32 accumulate */
#define TTO_PREC_BF16 2    /* tensor cores, single BF16 product, FP32 accumulate */
#define TTO_PREC_TF32X3 3  /* tensor cores, TF32 hi/lo split (3 products), FP32 accumulate */
#define TTO_PREC_FP16X3 4  /* tensor cores, FP16 hi/lo split (3 products in 2 mma), FP32 accumulate;
                              U and V are balanced per topology by a power-of-two scale */

#define TTO_FIT_WORKLOAD 0 /* fitness = -(lambda_o + max loading) */
#define TTO_FIT_F1 1       /* fitness = lambda_f1 = -(lambda_o + 200 lambda_c0 + 50 lambda_c) */
#define TTO_FIT_F2 2       /* fitness = lambda_f2 = lambda_f1 - Pi(lambda_b - lambda_b_pre): busbar outages too
                              (call tto_grid_busbar_reference first, with the same timesteps; the
                              busbar workspace is allocated on first use, so make one such call
                              outside stream capture before recording graphs) */

typedef struct tto_grid tto_grid;
typedef struct tto_archive tto_archive;

/* Grid description (all host pointers, copied by tto_grid_create).
 * Branch l joins from[l] -> to[l] with susceptance b[l] > 0 (p.u.); flows are
 * positive in the from->to direction.  p is [n_time][n_bus]; the slack bus
 * absorbs the imbalance of each timestep.  limit[l] > 0 is the thermal limit.
 * Stations: station s sits at bus station_bus[s] (not the slack) and owns the
 * assets asset_branch[asset_offset[s] .. asset_offset[s+1]) -- a branch id
 * incident to that bus, or -1 for the bus injection.  Actions: action a splits
 * station action_station[a]; bit i of action_mask[a] puts asset i on busbar B
 * (bit 0 must be clear; busbar B must hold at least one branch).
 * Disconnections (Sec. "Repertoire design": N_d disconnection slots beside the
 * N_a = k_max split slots): disc_branch[0 .. n_disc) lists the branches a
 * genome may open (distinct ids); n_dslot >= 0 slots, k_max + n_dslot <=
 * TTO_MAX_K, follow the split slots in every genome.  Zero-initialise the
 * struct so that grids without disconnections leave these fields 0. */
typedef struct {
  int32_t n_bus;
  int32_t n_branch;
  const int32_t* from;
  const int32_t* to;
  const double* b;
  int32_t slack;
  int32_t n_time;
  const double* p;
  const double* limit;
  int32_t n_monitored;
  const int32_t* monitored;
  int32_t n_outage;
  const int32_t* outage;
  int32_t n_station;
  const int32_t* station_bus;
  const int32_t* asset_offset;
  const int32_t* asset_branch;
  int32_t n_action;
  const int32_t* action_station;
  const uint32_t* action_mask;
  int32_t k_max;   /* split slots, 0 < k_max <= TTO_MAX_K */
  int32_t device;  /* CUDA device ordinal */
  int32_t n_disc;                /* size of the disconnection set (0: none) */
  const int32_t* disc_branch;    /* [n_disc] branch ids, or NULL when n_disc == 0 */
  int32_t n_dslot;               /* disconnection slots per genome */
} tto_grid_desc;

/* Options of one evaluation call. */
typedef struct {
  int32_t precision;     /* TTO_PREC_* */
  int32_t fitness_kind;  /* TTO_FIT_* */
  int32_t d_split;       /* archive extent over split stations (cell rows) */
  int32_t d_moved;       /* archive extent over moved assets (cell columns) */
  int32_t d_disc;        /* archive extent over opened branches lambda_d; 0 or 1: not a dimension */
} tto_eval_opts;

/* Mutation and crossover parameters (Algorithms 1-3).  The split part draws
 * N_mut ~ clip(Poisson(n_mut_mean), 1, k_max) operation rounds with
 * probabilities p_*; genomes with disconnection slots then take one
 * disconnection operation with probabilities dp_* (the paper's 0.25 / 0.25 /
 * 0.5 / 0).  crossover = 1 splits each batch as Algorithm 3 does: b_mc ~
 * Uniform{0..B} children by mutation, the others by Algorithm 2 on two parents
 * with bias p_c1 toward the first (crossover = 0: all by mutation). */
typedef struct {
  double p_add, p_remove, p_change, p_identity;
  double n_mut_mean;     /* Poisson mean of the number of mutation rounds */
  double dp_add, dp_remove, dp_change, dp_identity;
  int32_t crossover;
  double p_c1;
} tto_mut_params;

/* tto_grid_create -- copy the grid, check it, and run the one-time FP64
 * precompute: sparse LDL^T factorisation of the reduced susceptance matrix
 * (slack removed), the flow-response columns N = I - D A X A^T for every outage
 * and every branch that a split can move, the base flows f0 = D A X p for every
 * timestep (Sec. "Importer": PTDF of the pre-optimisation topology), and their
 * upload to the device.  *out owns all device copies.
 * Errors: TTO_E_ARG (sizes, ids, masks, station at slack, ...),
 * TTO_E_DISCONNECTED, TTO_E_CUDA, TTO_E_NOMEM. */
int tto_grid_create(const tto_grid_desc* d, tto_grid** out);

/* Release a grid and its device memory (NULL is accepted). */
int tto_grid_destroy(tto_grid* g);

/* Sizes of a created grid: n_branch, n_monitored, n_outage, n_time, k_max,
 * n_action (any pointer may be NULL). */
int tto_grid_info(const tto_grid* g, int32_t* n_branch, int32_t* n_monitored, int32_t* n_outage,
                  int32_t* n_time, int32_t* k_max, int32_t* n_action);

/* Size of the disconnection set and the number of disconnection slots per
 * genome (either pointer may be NULL); genomes are k_max + n_dslot wide. */
int tto_grid_disc_info(const tto_grid* g, int32_t* n_disc, int32_t* n_dslot);

/* Copy the FP64 base flows f0 [n_time][n_branch] of the unsplit grid into the
 * host buffer f0_host (the PTDF flows computed by tto_grid_create). */
int tto_grid_base_flows(const tto_grid* g, double* f0_host);

/* Replace the thermal limits (host [n_branch], all > 0). */
int tto_grid_set_limits(tto_grid* g, const double* limit_host);

/* Reserve evaluation workspace for batches of up to max_batch topologies and
 * n_t timesteps so that later calls allocate nothing (needed before capturing
 * evaluation calls in a CUDA graph). */
int tto_grid_reserve(tto_grid* g, int32_t max_batch, int32_t n_t);

/* tto_evaluate_batch -- exact DC N-1 evaluation of B topologies.
 *   topo      device int32 [B][k_max + n_dslot]: action ids, then indices into
 *             the disconnection set; -1 = empty slot;
 *   timesteps host int32 [n_t] indices into the grid's timesteps (NULL = all);
 *   fitness   device float [B]   (-inf when the split itself islands the grid);
 *   desc      device int32 [B][2] (split stations, moved assets);
 *   cell      device int32 [B]   archive cell of the descriptors: split stations,
 *             moved assets and, when opts->d_disc > 1, opened branches (fastest);
 *   island    device uint8 [B]   bit0: split islands the grid, bit1: some outage islands;
 *   metrics   device float [B][4] (lambda_o, max loading, lambda_c, lambda_c0) or NULL;
 *   fmax      device float [B][n_t][n_monitored] N-1 maximum |flow| or NULL.
 * Per topology: rank-k bus-split update of the base flows (FP64 split matrix
 * K and outage denominators N'_cc, islanding test N'_cc <= 1e-6), then a fused
 * sweep over all (monitored branch, outage) pairs that never stores the
 * post-contingency flows, reduced to the metrics of Sec. "Fitness function
 * heuristics" (an outage that islands the split grid is skipped and counted).
 * An opened branch is one more rank-1 term of the same update (a phase shift
 * across it with its post-topology flow held at zero); an outage of an opened
 * branch is no contingency and is skipped without counting; a split whose
 * busbar B keeps only opened branches islands the grid.
 * Asynchronous on stream.  A genome with an unknown action or disconnection
 * id, a repeated station or a repeated disconnection is reported by the
 * device; read it with tto_grid_sync_status.  With TTO_PREC_FP32 one call
 * takes at most 65535 x G topologies (G = 8, 4, 2, 1 up to 4, 8, 16, 32
 * timesteps, halved by the autotuner's shape 1); larger batches return
 * TTO_E_ARG. */
int tto_evaluate_batch(tto_grid* g, const int32_t* topo, int32_t B, const int32_t* timesteps,
                       int32_t n_t, const tto_eval_opts* opts, float* fitness, int32_t* desc,
                       int32_t* cell, uint8_t* island, float* metrics, float* fmax, void* stream);

/* tto_grid_autotune -- time every sweep tile variant of `precision` on this
 * grid with a batch of B unsplit topologies over the first n_t timesteps (the
 * sweep has no data-dependent work, so the timing holds for any batch of that
 * size) and keep the fastest for later calls on this grid with that
 * precision.  *shape_out receives the chosen variant, ms_out (host, may be
 * NULL, room for 8) the milliseconds of one evaluation per variant: 2 variants
 * for TTO_PREC_FP32, 4 for the mma.sync tensor-core modes, and for
 * TTO_PREC_TF32X3 a fifth, the tcgen05 sweep.  Synchronises the stream.
 * Call it outside stream capture (it may allocate workspace). */
int tto_grid_autotune(tto_grid* g, int32_t B, int32_t n_t, int32_t precision, int32_t* shape_out,
                      float* ms_out, void* stream);

/* Select the sweep tile variant of `precision` on this grid by hand (-1 = the
 * default); tto_grid_autotune makes the same choice by timing. */
int tto_grid_set_sweep_shape(tto_grid* g, int32_t precision, int32_t shape);

/* One (grid, topology batch) job of tto_evaluate_multi; the fields mean what
 * the arguments of tto_evaluate_batch mean (fmax is not produced). */
typedef struct {
  tto_grid* grid;
  const int32_t* topo;
  int32_t B;
  const int32_t* timesteps;  /* host, NULL = all */
  int32_t n_t;
  float* fitness;
  int32_t* desc;
  int32_t* cell;
  uint8_t* island;
  float* metrics;
} tto_eval_job;

#define TTO_MULTI_SEQUENTIAL 0 /* one grid after another on the stream */
#define TTO_MULTI_STREAMS 1    /* grids on forked streams, joined back into the stream */
#define TTO_MULTI_GRAPH 2      /* as STREAMS, recorded once as a CUDA graph and replayed */
#define TTO_MULTI_PERSISTENT 3 /* one launch per stage for all jobs: split update, persistent sweep, metrics */
#define TTO_MULTI_PERSISTENT_GRAPH 4 /* as PERSISTENT, recorded once as a CUDA graph and replayed */

/* tto_evaluate_multi -- evaluate n (1..16) jobs on grids of one device as one
 * unit of work (mixed grid sizes, timestep counts and batch sizes; each grid at
 * most once).  In TTO_MULTI_GRAPH mode the first call with a given set of jobs
 * (same grids, buffers, sizes, options and stream) runs them eagerly and
 * records the launch sequence as a CUDA graph; later identical calls replay it
 * with one graph launch.  Recorded graphs are dropped when a grid is destroyed
 * or its workspace is reallocated.
 * TTO_MULTI_PERSISTENT (TTO_PREC_FP32, fitness kinds WORKLOAD and F1) runs all
 * jobs with one launch per stage: one split update over every job's
 * topologies, one persistent FP32 sweep whose CTAs (a few per SM) take
 * (job, 128-row tile, topology group) items from a shared work-list counter
 * until none is left (jobs with the largest items first; each job's items use
 * its autotuned FP32 variant's group size), and one metric reduction (batching
 * row of the workload: mixed grids in one persistent launch).  Eager calls in
 * this mode share one counter per device, so such calls must not overlap on
 * the GPU; TTO_MULTI_PERSISTENT_GRAPH records the same launches as a graph
 * with a counter of its own.  Results equal the other modes bit for bit.
 * Asynchronous on stream. */
int tto_evaluate_multi(const tto_eval_job* jobs, int32_t n, const tto_eval_opts* opts, int32_t mode,
                       void* stream);

/* Per-stage CUDA-event timing of evaluation calls, off by default.
 * tto_grid_profile(g, 1) clears the record and times the next calls (at most
 * 256); tto_grid_profile(g, 0) stops.  tto_grid_profile_read synchronises on
 * the recorded events and returns, summed over the recorded calls, the
 * milliseconds of the split update, the N-1 sweep, the metric reduction and
 * the busbar sweep (lambda_f2; 0 without it) in ms_stage[0..3] (host float
 * [4]), and the number of calls in *n_calls. */
int tto_grid_profile(tto_grid* g, int32_t enable);
int tto_grid_profile_read(tto_grid* g, float* ms_stage, int32_t* n_calls);

/* tto_evaluate_batch_static -- tto_evaluate_batch (TTO_PREC_FP32 only) for
 * callers that cannot let the library allocate device memory: processes whose
 * device memory is owned by another allocator (a framework's caching
 * allocator or a fixed partition), and services that must keep their device
 * footprint constant after start-up.  The paper has no counterpart; this is a
 * deployment variant of the same evaluation.
 * Its workspace is a fixed 64 MiB __device__ array inside the library, present
 * on every device that loads the library until the process exits; the call
 * itself allocates nothing (no cudaMalloc or cudaFree).  A batch whose
 * workspace exceeds 64 MiB is rejected with TTO_E_ARG and a message giving the
 * bytes it needs (about 7 KB per topology on the 30-bus workload, 1 MB on the
 * 10000-bus one).  The first call on a device looks up the array's address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture, and do not use the entry point across
 * a cudaDeviceReset of the device.  The FP32 sweep runs in the variant that
 * tto_grid_autotune chose for the grid (the default variant otherwise), as in
 * tto_evaluate_batch.
 * All calls share the one array: calls that overlap on the GPU (other streams,
 * other threads) race and corrupt each other's results; serialise them.
 * Arguments, outputs and status reporting are those of tto_evaluate_batch. */
int tto_evaluate_batch_static(tto_grid* g, const int32_t* topo, int32_t B, const int32_t* timesteps,
                              int32_t n_t, const tto_eval_opts* opts, float* fitness, int32_t* desc,
                              int32_t* cell, uint8_t* island, float* metrics, float* fmax,
                              void* stream);

/* tto_evaluate_busbar -- busbar outages (Sec. "Fitness function heuristics":
 * lambda_b = sum_e Pi(max_{b in O_b} |f_e^(b)| - fbar_e), summed over the
 * selected timesteps like lambda_o).  O_b holds every splittable station's
 * node and both nodes of a split station; an outage takes its node out of
 * service (every branch at it opens, its injection is lost and the slack
 * balances).  One that leaves the rest of the grid in pieces islands: it is
 * skipped and counted.  Per topology (device int32 [B][k_max + n_dslot]):
 * the split update, a rank-(d - 1) outage of each busbar node with d live
 * branches (FP64 setup, FP32 sweep over the monitored rows), then
 *   lambda_b  device float [B] (NaN for a topology that islands the grid),
 *   n_island  device int32 [B] islanding busbar outages (-1: the topology islands), or NULL,
 *   bmax      device float [B][n_t][n_monitored] max over busbar outages of |flow|, or NULL.
 * Asynchronous on stream; genome errors as for tto_evaluate_batch. */
int tto_evaluate_busbar(tto_grid* g, const int32_t* topo, int32_t B, const int32_t* timesteps, int32_t n_t,
                        float* lambda_b, int32_t* n_island, float* bmax, void* stream);

/* lambda_b of the unsplit topology (lambda_b^pre) for these timesteps (host,
 * NULL = all), kept on the device for TTO_FIT_F2 evaluations with the same
 * timesteps; tto_grid_set_limits drops it.  Asynchronous on stream. */
int tto_grid_busbar_reference(tto_grid* g, const int32_t* timesteps, int32_t n_t, void* stream);

/* tto_worst_k -- worst-k N-1 export for AC validation (Sec. "AC-Validator":
 * the DC optimiser computes each N-1 case's overload energy and writes out the
 * worst k).  For n topologies (device int32 [n][k_max + n_dslot]) over the
 * selected timesteps (host, NULL = all): the split update, then per outage c
 *   E_c = sum_t sum_l max(|F_lc[t]| - limit_l, 0)   (FP32, fixed summation order),
 * and the k outages of largest E_c, larger first, the lower outage index first
 * among equal energies.  outage_out device int32 [n][k]: indices into the
 * grid's outage list, -1 where fewer than k qualify; energy_out device float
 * [n][k] (NaN with -1).  An outage that islands the topology, or whose branch
 * the topology opened, never qualifies (its all_energy entry is NaN); a
 * topology that islands the grid yields -1 throughout.  all_energy (device
 * float [n][n_outage], may be NULL) receives every E_c.  1 <= k <= 1024 and
 * n <= 262140 (TTO_E_ARG otherwise).
 * Shares the evaluation workspace with the other calls on this grid.
 * Asynchronous on stream; genome errors as for tto_evaluate_batch. */
int tto_worst_k(tto_grid* g, const int32_t* topo, int32_t n, const int32_t* timesteps, int32_t n_t, int32_t k,
                int32_t* outage_out, float* energy_out, float* all_energy, void* stream);

/* Test hook for the timeout path (the paper has no counterpart): runs one
 * thread that waits, through the sweeps' own bounded-wait routine, on an
 * mbarrier that nothing completes, for at most `cycles` SM clock cycles
 * (1 .. 2^32); when the wait gives up it writes TTO_E_TIMEOUT to the grid's
 * status word as a sweep would.  Faults, traps and unbounded waits are never
 * used.  Asynchronous on stream. */
int tto_debug_bounded_wait(tto_grid* g, int64_t cycles, void* stream);

/* Synchronise the stream and return (then clear) the device status word:
 * TTO_OK, TTO_E_TOPOLOGY or TTO_E_TIMEOUT.  After a TTO_E_TIMEOUT (a bounded
 * wait inside a sweep gave up), tcgen05 sweeps on the grid return at once
 * until this call clears the word. */
int tto_grid_sync_status(tto_grid* g, void* stream);

/* Archive of d_split x d_moved cells, one elite per cell, device resident.
 * Starts empty. */
int tto_archive_create(tto_grid* g, int32_t d_split, int32_t d_moved, tto_archive** out);
/* The same with a third descriptor, the number of opened branches lambda_d,
 * over d_disc >= 1 values (d_split x d_moved x d_disc cells, lambda_d fastest,
 * as the paper's cell map beta puts it first). */
int tto_archive_create_ex(tto_grid* g, int32_t d_split, int32_t d_moved, int32_t d_disc, tto_archive** out);
int tto_archive_destroy(tto_archive* a);

/* Copy the archive to host buffers: fitness [cells] (-inf = empty cell),
 * genome [cells][k_max + n_dslot], filled [cells] (0/1).  Synchronous. */
int tto_archive_export(const tto_archive* a, float* fitness, int32_t* genome, uint8_t* filled);
/* Overwrite the archive from host buffers of the same layout. */
int tto_archive_import(tto_archive* a, const float* fitness, const int32_t* genome,
                       const uint8_t* filled);

/* Scatter-insert B evaluated candidates (device arrays from
 * tto_evaluate_batch) into the archive: per cell, the candidate with the
 * highest fitness wins (lowest index on ties) and replaces the elite only if
 * strictly better; non-finite fitness is skipped.  Equals a sequential
 * in-order insert with strict '>' (Algorithm 3).  Asynchronous. */
int tto_archive_insert(tto_archive* a, const int32_t* topo, int32_t B, const float* fitness,
                       const int32_t* cell, void* stream);

/* Propose B genomes (device int32 [B][k_max + n_dslot]) from parents drawn
 * uniformly over the filled cells (an empty archive offers the unsplit
 * topology): Algorithm 1's mutation, and with mp->crossover Algorithm 2's
 * crossover for the children past b_mc, driven by Philox4x32-10 keyed by seed
 * and countered by (word block, candidate, iteration); b_mc comes from
 * candidate 0xFFFFFFFF's first word.  Deterministic given (archive, seed,
 * iteration). */
int tto_mapelites_propose(tto_archive* a, uint64_t seed, uint64_t iteration, int32_t B,
                          const tto_mut_params* mp, int32_t* topo_out, void* stream);

/* One full MapElites iteration on the device: propose B candidates, evaluate
 * them exactly (tto_evaluate_batch with opts, whose cell extents must equal
 * the archive's), insert them.  The candidates
 * and their fitness stay in library workspace; topo_out / fitness_out
 * (device, optional) receive copies.  Asynchronous. */
int tto_mapelites_step(tto_archive* a, uint64_t seed, uint64_t iteration, int32_t B,
                       const tto_mut_params* mp, const tto_eval_opts* opts, int32_t* topo_out,
                       float* fitness_out, void* stream);

/* tto_epoch_export -- the end-of-epoch hand-over (Sec. "High-level Genetic
 * Algorithm loop": iterations are grouped into epochs and results leave the
 * GPU only at an epoch's end).  Queued on stream after the epoch's
 * iterations: a device snapshot of the archive and, for k > 0, the worst-k N-1
 * cases (tto_worst_k) of every filled cell's genome (an empty cell's list is
 * -1 / NaN); the snapshot is then copied on
 * an internal stream to the host buffers fitness [cells], genome
 * [cells][k_max + n_dslot], filled [cells], worst_outage / worst_energy
 * [cells][k] (pinned memory keeps the copy asynchronous).  Iterations queued
 * on stream afterwards overlap the copy.  The host buffers are complete after
 * tto_epoch_export_wait; a later export orders itself after the previous
 * copy.  0 <= k <= 1024.  Uses the grid's evaluation workspace. */
int tto_epoch_export(tto_archive* a, int32_t k, float* fitness, int32_t* genome, uint8_t* filled,
                     int32_t* worst_outage, float* worst_energy, void* stream);
/* Block until the last tto_epoch_export's host buffers are complete. */
int tto_epoch_export_wait(tto_archive* a);

/* The 4x32-bit Philox words of counter block `block` of candidate `cand` in
 * `iteration` under `seed`, written to device uint32 [n][4] for blocks
 * block .. block+n-1 (exposes the generator that drives the mutation). */
int tto_philox_blocks(uint64_t seed, uint64_t iteration, uint32_t cand, uint32_t block, int32_t n,
                      uint32_t* out, void* stream);

/* ------------------------------------------------------------ surrogate
 * A learned screen for MapElites proposals.  The paper has no counterpart; the
 * network, its inputs and its online training are this library's own.
 *
 * Model: y = w4 . h3 + b4,  h3 = relu(W3 h2 + b3),  h2 = relu(W2 h1 + b2),
 * h1 = relu(W1 x + b1), predicting log1p(-fitness) (lower is better) of a
 * topology.  Input x (dimension D = 8 S + R, S stations): for every station
 * split by the genome eight values
 *   [1, min(|A|,|B|)/m, b(B)/b(station), p_B(t=0) / sum|p(t=0)|,
 *    branches on B / branches of the station, |B|/m, 0, 0]
 * (m assets, |B| assets on the second busbar, b() summed branch susceptance),
 * zero for unsplit stations; then the post-split N-0 loading |f'_l| / fbar_l
 * at timestep 0 of the R branches with the highest base-case loading (sorted
 * by loading, descending, ties by branch id; fixed when the surrogate is
 * created).  Parameters are kept in FP32, packed as W1 [H][D], b1 [H],
 * W2 [H][H], b2 [H], W3 [H][H], b3 [H], w4 [H], b4 [1]; every product rounds
 * both operands to BF16 and accumulates in FP32 (tensor cores for the dense
 * products).  Training: the network fits the standardised target
 * (log1p(-fitness) - mean) / deviation, mean and population standard
 * deviation taken over the finite targets in the replay ring (recomputed after
 * every append; 0 and 1 while it is empty), by mean squared error over a
 * minibatch drawn uniformly (Philox keyed by the seed) from the ring, and Adam
 * with bias correction.  All calls are deterministic for a given call
 * sequence. */
typedef struct tto_surrogate tto_surrogate;

typedef struct {
  int32_t hidden;    /* H, multiple of 16 in [16, 1024] */
  int32_t n_load;    /* R loading features, 1..n_branch */
  int32_t replay;    /* capacity of the replay ring (pairs) */
  int32_t minibatch; /* rows per training step */
  double lr, beta1, beta2, eps; /* Adam */
  uint64_t seed;     /* initial weights (He-uniform, zero biases) and minibatch draws */
} tto_surrogate_cfg;

/* Create a surrogate for grid g (which must outlive it).  Errors: TTO_E_ARG
 * for a configuration out of range, TTO_E_CUDA / TTO_E_NOMEM. */
int tto_surrogate_create(tto_grid* g, const tto_surrogate_cfg* cfg, tto_surrogate** out);
int tto_surrogate_destroy(tto_surrogate* s);

/* Sizes: number of packed parameters, input dimension D, pairs in the replay
 * ring; rows_out (host int32 [R], optional) receives the loading branches and
 * target_stats (host float [2], optional) the current target mean and
 * deviation (both synchronise the device).  Any pointer may be NULL. */
int tto_surrogate_info(const tto_surrogate* s, int64_t* n_params, int32_t* input_dim,
                       int32_t* replay_fill, int32_t* rows_out, float* target_stats);

/* Copy the packed FP32 parameters to get_host and/or replace them from
 * set_host (host float [n_params]; either may be NULL).  Setting clears the
 * Adam moments and step count.  Synchronises the device. */
int tto_surrogate_params(tto_surrogate* s, float* get_host, const float* set_host);

/* Predicted log1p(-fitness) of B genomes (device int32 [B][k_max]) into score
 * (device float [B]): mean + deviation * network output, +inf for a genome
 * whose split islands the grid or that splits a station twice.  Asynchronous
 * on stream. */
int tto_surrogate_score(tto_surrogate* s, const int32_t* topo, int32_t B, float* score, void* stream);

/* Host copies of the inputs of the last batch that was scored, added or
 * differentiated (B of its rows): station of each genome slot si [B][k_max]
 * (-1 = empty), that station's eight values sf [B][k_max][8], loadings
 * xd [B][R] and valid [B] (0 = the split islands the grid).  Any pointer may
 * be NULL.  Synchronises the device. */
int tto_surrogate_features(tto_surrogate* s, int32_t B, int32_t* si, float* sf, float* xd,
                           int32_t* valid);

/* Host copies of the network's intermediate values for the first B rows of the
 * last batch (for element-wise checks of each layer): hidden activations
 * h [3][B][H] (after the ReLU), output y [B] (the scores after
 * tto_surrogate_score, the unscaled network output after tto_surrogate_grad),
 * and, after tto_surrogate_grad, the training targets t [B]
 * (standardised), the output gradient dy [B] and the backward signals
 * dh [3][B][H] (dL/dz of hidden layers 1..3, ReLU mask applied).  Any pointer
 * may be NULL; values the last call did not compute are unspecified.
 * Synchronises the device.  TTO_E_ARG when B exceeds the last batch. */
int tto_surrogate_trace(tto_surrogate* s, int32_t B, float* h, float* y, float* t, float* dy, float* dh);

/* Append B exact pairs (device genomes [B][k_max], device fitness [B] from
 * tto_evaluate_batch) to the replay ring; non-finite fitness is kept without a
 * target and skipped by the loss.  Asynchronous. */
int tto_surrogate_add(tto_surrogate* s, const int32_t* topo, int32_t B, const float* fitness,
                      void* stream);

/* Run `steps` training steps (minibatch forward, backward, Adam).  If loss is
 * not NULL, synchronises the stream and stores the mean squared error of the
 * last minibatch before its update.  Errors: TTO_E_ARG if the ring is empty. */
int tto_surrogate_train(tto_surrogate* s, int32_t steps, float* loss, void* stream);

/* Loss and gradient without an update on B exact pairs (device genomes
 * [B][k_max], device fitness [B]; non-finite fitness is skipped): features,
 * forward, standardised targets as in training, backward.  Writes the mean
 * squared error to *loss and the packed gradient (host float [n_params]) to
 * grad.  Synchronises the stream. */
int tto_surrogate_grad(tto_surrogate* s, const int32_t* topo, int32_t B, const float* fitness,
                       float* loss, float* grad, void* stream);

/* Ranking of the screened step (rank_by). */
#define TTO_SCREEN_SCORE 0     /* by predicted score */
#define TTO_SCREEN_CELL_GAIN 1 /* empty cells first, then by predicted gain over the cell's elite */

/* One surrogate-screened MapElites iteration: propose n_propose candidates
 * (as tto_mapelites_propose; n_propose <= 2^30), score them, and evaluate
 * exactly the n_exact ranked first.  TTO_SCREEN_SCORE ranks by predicted
 * score; TTO_SCREEN_CELL_GAIN ranks the proposals whose descriptors map to an
 * empty cell first, by predicted score, then the others by predicted
 * improvement over their cell's elite, score - log1p(-fitness_elite).  Ties go
 * by proposal index.  Either way a proposal that islands the grid or equals
 * its cell's elite slot for slot ranks last, and a proposal whose genome
 * repeats the one ranked just before it moves behind all others (repeats fill
 * the batch only when too few others remain).  While the replay ring is empty
 * every proposal that does not island the grid scores 0.  The evaluated
 * candidates are inserted into the archive and appended to the replay ring,
 * then train_steps training steps run.  topo_out / fitness_out / score_out
 * (device, optional, [n_exact]) receive the evaluated genomes, their exact
 * fitness and their predicted score (+inf for a skipped elite copy).
 * Asynchronous. */
int tto_mapelites_step_screened(tto_archive* a, tto_surrogate* s, uint64_t seed, uint64_t iteration,
                                int32_t n_propose, int32_t n_exact, int32_t rank_by,
                                const tto_mut_params* mp, const tto_eval_opts* opts,
                                int32_t train_steps, int32_t* topo_out, float* fitness_out,
                                float* score_out, void* stream);

/* Thread-local message of the last failing call ("" if none). */
const char* tto_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* TTO_H */
