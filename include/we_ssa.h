/*
 * we_ssa.h -- C ABI of the GB300 (sm_103a) weighted-ensemble Gillespie-SSA library.
 *
 * The library runs the data-parallel hot path of the weighted-ensemble (WE) method for
 * stochastic chemical kinetics of Donovan, Sedgewick, Faeder & Zuckerman (arXiv:1303.5986):
 * many weighted walkers ("trajectory segments") are propagated with Gillespie's direct SSA
 * for one interval tau (Sec. II.A), then binned and split or merged inside each bin so that
 * every occupied bin holds M_targ walkers while the total weight is kept (Sec. II.B and its WE
 * algorithm listing).  Optional steady-state recycling ("feedback", Sec. II.B.2) moves walkers
 * that reach a target set B back to a source state and records the weight that arrived, whose
 * rate is the flux with MFPT = 1/flux (Eq. "mfpt").
 *
 * Conventions shared by every entry point:
 *   - Every function returns a we_status (0 = WE_OK, negative = error) and never throws,
 *     aborts or traps; the message of the last failure on the calling thread is returned by
 *     we_last_error().
 *   - Host inputs are borrowed for the duration of the call and copied; handles are owned by
 *     the library and released by the matching *_destroy.
 *   - Device work is issued on the cudaStream_t passed as `stream` (NULL = the legacy default
 *     stream).  Entry points that return data to the host synchronise that stream; the others
 *     only enqueue work.
 *   - Device memory of an ensemble is either carved from a caller-owned device buffer
 *     (`workspace`, e.g. a PyTorch tensor) or, when workspace is NULL, allocated by the library.
 *   - Device-side failures (step cap, count overflow) are reported through a per-run status
 *     word that the host reads back (we_ensemble_get WE_OUT_STATUS, or the return of a
 *     synchronising call).  Every device wait in the library is bounded.
 *   - Species counts are int32 and never exceed WE_MAX_COUNT; times, propensities and weights
 *     are IEEE double.
 */
#ifndef WE_SSA_H
#define WE_SSA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t we_status;
#define WE_OK 0
#define WE_EINVAL (-1)         /* an argument is invalid (message in we_last_error) */
#define WE_ENOMEM (-2)         /* host or device allocation failed, or workspace too small */
#define WE_ECUDA (-3)          /* a CUDA runtime call failed */
#define WE_EOVERFLOW (-4)      /* a species count would pass WE_MAX_COUNT, or walkers passed capacity */
#define WE_ESTEPCAP (-5)       /* a walker needed more than max_steps events in one interval */
#define WE_ETIMEOUT (-6)       /* a bounded device wait gave up */
#define WE_ENOTSUPPORTED (-7)  /* the request is valid but not implemented for these sizes */

/* Largest count a species may reach.  Products of three counts then fit in int64, which keeps
 * every combinatorial propensity factor exact. */
#define WE_MAX_COUNT 2097151

/* Events one walker may fire in one interval when the configuration sets no cap of its own;
 * past it the walker stops with WE_ESTEPCAP, so every SSA loop is bounded. */
#define WE_DEFAULT_MAX_STEPS (1ll << 26)

/* Rate laws (Sec. III): mass action with combinatorial factors C(x, m) per reactant taken m
 * times (the convention that puts the Schloegl model's stable states at X=82 and X=563,
 * Sec. III.B.3), or Hill repression c/(1 + (y/K)^n) of a zeroth-order production reaction
 * (the epigenetic switch, Sec. III.C.1), evaluated as (c K^n)/(K^n + y^n). */
#define WE_MASS_ACTION 0
#define WE_HILL_REPRESSION 1

/* Feedback modes of we_run_config.feedback. */
#define WE_FEEDBACK_RECYCLE 1
#define WE_FEEDBACK_ABSORB 2
#define WE_FEEDBACK_ENDPOINT 3

/* Target-set clause operators: x[species] >= threshold, x[species] <= threshold. */
#define WE_OP_GE 0
#define WE_OP_LE 1

/* Thread-to-walker mapping of the SSA kernel. */
#define WE_MAP_AUTO 0          /* let the autotuner pick */
#define WE_MAP_THREAD 1        /* one thread per walker, propensity tree in registers */
#define WE_MAP_WARP 2          /* one warp per walker, propensity tree in shared memory
                                  (any network up to 16,384 reactions) */
#define WE_MAP_THREAD_TABLE 3  /* one thread per walker, propensity tree looked up by count
                                  (networks whose propensities all read one species) */

/* Kernels of the grouping-by-bin and split/merge step (we_ensemble_set_resample_kernel). */
#define WE_RESAMPLE_AUTO 0        /* ONE_LAUNCH for grids of up to 256 bins that fit, else CHAIN */
#define WE_RESAMPLE_CHAIN 1       /* per-run scan, grid-wide grouping, one warp per occupied bin
                                     (three launches; any size) */
#define WE_RESAMPLE_ONE_LAUNCH 2  /* one launch, blocks of 512 threads, the run's walker lists in
                                     shared memory */

const char *we_status_string(we_status s);
/* Message of the last failing call on this thread ("" if none).  Valid until the next call. */
const char *we_last_error(void);
/* Fault injection for tests: the nth device allocation the library makes from now on fails as
 * if the device were out of memory (its caller then returns WE_ENOMEM and frees what it had
 * allocated); 0 disarms.  Allocations: a library-owned ensemble workspace (1), an MLP (4), an
 * MLP training or gradient call (1).  Process-wide. */
we_status we_debug_fail_allocation(int32_t nth);
/* Library version as MAJOR*10000 + MINOR*100 + PATCH. */
int32_t we_version(void);

/* ------------------------------------------------------------------------------------------
 * Reaction network (Sec. II.A; models of Sec. III).
 *
 * n_species S >= 1, n_reactions M >= 1.  Reactants and products are CSR lists over reactions:
 * reaction j has reactant entries [reac_ptr[j], reac_ptr[j+1]) of (species, multiplicity 1..3)
 * and product entries likewise (multiplicity >= 0); repeated species are summed; the total
 * reactant order of a reaction is at most 3.  rate is n_param_sets x M row-major (c_j of each
 * parameter set; runs of a batch pick a set).  rate_law (M, NULL = all mass action);
 * hill_species / hill_n (M, n in 1..3) and hill_K (hill_K_rows x M, hill_K_rows = 1 or
 * n_param_sets) are read for WE_HILL_REPRESSION reactions only, which must have no dynamic
 * reactant; the regulator count y is the state's entry for hill_species.  Rate constants must
 * be finite and >= 0; K finite and > 0.  fixed_count (S, NULL = none): -1 for a
 * dynamic species, otherwise the constant count of a species held fixed (A and B of the
 * Schloegl model); fixed reactants are folded into the rate constant, c_eff = c * prod C(n, m),
 * and fixed species are never changed by a reaction.
 * Errors: WE_EINVAL on any malformed input; WE_ENOMEM.
 * ------------------------------------------------------------------------------------------ */
typedef struct we_network we_network;
we_status we_network_create(int32_t n_species, int32_t n_reactions,
                            const int32_t *reac_ptr, const int32_t *reac_species,
                            const int32_t *reac_mult, const int32_t *prod_ptr,
                            const int32_t *prod_species, const int32_t *prod_mult,
                            int32_t n_param_sets, const double *rate, const int32_t *rate_law,
                            const int32_t *hill_species, int32_t hill_K_rows, const double *hill_K,
                            const int32_t *hill_n, const int32_t *fixed_count, we_network **out);
void we_network_destroy(we_network *net);
/* Effective (folded) rate constant of reaction j in parameter set p; for Hill reactions
 * c*K^n.  Host-side query for tests. */
we_status we_network_keff(const we_network *net, int32_t p, int32_t j, double *out);
/* Number of reactions whose propensity may change when reaction j fires (dependency-graph
 * out-degree, j itself included when affected). */
we_status we_network_dep_degree(const we_network *net, int32_t j, int32_t *out);

/* ------------------------------------------------------------------------------------------
 * Bin maps (Sec. II.B: non-overlapping bins, regular 1-D or 2-D grids).
 *
 * Grid: ndim in 1..4 dimensions; dimension d bins species[d] with n_bins[d] bins given by
 * n_bins[d]+1 ascending edges (concatenated over dimensions in `edges`).  Bin k of a dimension
 * is [edge_k, edge_{k+1}); counts below the first edge fall in bin 0 and counts at or above the
 * last edge in the last bin (give a last edge of +INFINITY for an overflow bin).  The flat bin
 * index is row-major, last dimension fastest.  Errors: WE_EINVAL (non-ascending edges, NaN,
 * more than 65536 bins in total).
 * ------------------------------------------------------------------------------------------ */
typedef struct we_binmap we_binmap;
we_status we_binmap_grid(int32_t ndim, const int32_t *species, const int32_t *n_bins,
                         const double *edges, we_binmap **out);
void we_binmap_destroy(we_binmap *bm);
int32_t we_binmap_n_bins(const we_binmap *bm);

/* ------------------------------------------------------------------------------------------
 * Learned progress coordinate.  WE is unbiased under any binning (Sec. II.B), and choosing bins
 * automatically is the open problem named in Sec. IV.B; these entry points fit a small MLP
 * z(x) = w3 . silu(W2 silu(W1 phi + b1) + b2) + b3, phi_s = log1p(x_s) over every species, so that
 * sigmoid(z) estimates the probability of reaching the target set (labels come from the
 * library's own SSA runs), and bin walkers by intervals of z.
 *
 * we_mlp_create: n_in = number of species, hidden <= 64; params (host, FP32) in the layout
 *   W1[hidden][n_in], b1[hidden], W2[hidden][hidden], b2[hidden], w3[hidden], b3.
 * we_mlp_train: `steps` Adam steps (beta 0.9/0.999, eps 1e-8) on consecutive batches of the
 *   device arrays states (n x n_in int32, sample-major) and labels (n float in [0,1]) with the
 *   batch-mean BCE-with-logits loss; loss_per_step (host, steps floats, may be NULL).
 * we_mlp_gradient: the batch-mean loss and its gradient (device, n_params floats) over all n
 *   samples, without changing the weights (for gradient checks).
 * we_mlp_forward: z (device, n floats) of n states (device, n x n_in int32) from the FP32
 *   weights on the CUDA cores (bf16 = 0) or in the inference form (bf16 = 1): weights rounded
 *   to BF16, the 64 x 64 layer on the tensor cores (tcgen05, FP32 accumulator, the FP32
 *   activations split into three BF16 parts), the same z as a learned bin map made from this
 *   MLP computes, bit for bit.
 * Training is FP32 with sums in sample order (deterministic).  Errors: WE_EINVAL, WE_ENOMEM,
 * WE_ECUDA; WE_ENOTSUPPORTED when the inference form's shared memory (57 KB + 2 hidden
 * (n_in + 1) bytes + biases) passes 227 KB.
 * ------------------------------------------------------------------------------------------ */
typedef struct we_mlp we_mlp;
we_status we_mlp_create(int32_t n_in, int32_t hidden, const float *params, we_mlp **out);
void we_mlp_destroy(we_mlp *mlp);
int32_t we_mlp_n_params(const we_mlp *mlp);
we_status we_mlp_get_params(const we_mlp *mlp, float *dst, size_t dst_floats);
we_status we_mlp_train(we_mlp *mlp, const int32_t *states, const float *labels, int32_t n,
                       int32_t steps, int32_t batch, float lr, float *loss_per_step, void *stream);
we_status we_mlp_gradient(const we_mlp *mlp, const int32_t *states, const float *labels, int32_t n,
                          float *grad, float *loss, void *stream);
we_status we_mlp_forward(const we_mlp *mlp, const int32_t *states, int32_t n, int32_t bf16, float *z,
                         void *stream);
/* we_mlp_create_init: a new MLP with the library's own initial weights: W1, W2 and w3 uniform
 *   in [-1/sqrt(fan_in), 1/sqrt(fan_in)) from a splitmix64 stream started at `seed` (in that
 *   order, row-major), zero biases.
 * we_mlp_coordinate_edges: n_bins equal intervals of the learned coordinate for bin placement:
 *   z of the n given states (device, n x n_in int32) in the inference form (bf16 = 1, the z a
 *   learned bin map computes), then lo = the floor(lo_q (n - 1))-th smallest z (0-based) and
 *   hi = the largest, both found on the device by radix selection, and edges[i] =
 *   fl32(lo + (hi - lo) i / n_bins) in double for i = 0..n_bins (hi = lo + 1 when hi <= lo).
 *   edges: n_bins + 1 floats, host or device.  Allocates its scratch; synchronises the stream.
 *   Errors: WE_EINVAL, WE_ENOMEM, WE_ECUDA, WE_ENOTSUPPORTED (as we_mlp_forward). */
we_status we_mlp_create_init(int32_t n_in, int32_t hidden, uint64_t seed, we_mlp **out);
we_status we_mlp_coordinate_edges(const we_mlp *mlp, const int32_t *states, int32_t n, int32_t n_bins,
                                  double lo_q, float *edges, void *stream);
/* Bin map on the learned coordinate: a snapshot of the MLP's weights rounded to BF16, with
 * n_bins intervals [edges[k], edges[k+1]) of z (values outside fall in the end bins).  Binning
 * runs in a kernel of its own after the SSA kernel, in tiles of 128 walkers, in the inference
 * form of we_mlp_forward with bf16 = 1. */
we_status we_binmap_learned(const we_mlp *mlp, int32_t n_bins, const float *edges, we_binmap **out);

/* ------------------------------------------------------------------------------------------
 * Run configuration (the arguments of the WE procedure, Sec. II.B: tau, M_targ, the grid,
 * the initial state, plus the recycling target of Sec. II.B.2).  A configuration describes
 * n_runs independent WE runs executed together (a batch: replicas or a parameter sweep).
 * ------------------------------------------------------------------------------------------ */
typedef struct {
  double tau;                      /* WE interval (> 0) */
  int32_t m_targ;                  /* walkers per occupied bin after resampling (>= 1) */
  int32_t n_runs;                  /* independent runs in the batch (>= 1) */
  uint64_t seed;                   /* Philox key: word 0 = low 32 bits, word 1 = high 32 bits + run id */
  const uint32_t *run_ids;         /* n_runs run ids (NULL: 0..n_runs-1) */
  const int32_t *param_set;        /* n_runs parameter-set indices (NULL: run % n_param_sets) */
  int32_t n_init;                  /* walkers per run at the start (>= 1, <= capacity) */
  const int32_t *init_states;      /* n_runs x n_init x S species counts, walker-major */
  const double *init_weights;      /* n_runs x n_init weights */
  int32_t first_iter;              /* index of the first WE iteration (resume) */
  int32_t capacity;                /* walker slots per run (0: max(m_targ * n_bins, n_init)) */
  int32_t record_iters;            /* iterations of observables kept on the device (>= 1) */
  int32_t feedback;                /* 0: none.  WE_FEEDBACK_RECYCLE (1): a walker that enters
                                      the target set is put back in the recycle state at once
                                      and its weight counted as flux (Sec. II.B.2).
                                      WE_FEEDBACK_ABSORB (2): the target set is absorbing --
                                      a walker stops at the event that enters it and stays
                                      there, and the time of that first passage is kept per
                                      walker (WE_OUT_FPT): the brute-force transition-time runs
                                      of Sec. II.C; needs resample = 0.
                                      WE_FEEDBACK_ENDPOINT (3): the target set is checked at the
                                      end of each interval only (the protocol of checking at a
                                      prescribed time step, Sec. IV): a walker found in it is
                                      put in the recycle state, its weight counted as flux, and
                                      binned there; a walker that enters and leaves within one
                                      interval is not counted, which biases the MFPT up */
  int32_t n_clauses;               /* target set B = AND of clauses (1..4 when feedback) */
  int32_t tgt_species[4];
  int32_t tgt_op[4];               /* WE_OP_GE / WE_OP_LE */
  const int32_t *tgt_threshold;    /* n_runs x n_clauses */
  const int32_t *recycle_state;    /* n_runs x S (NULL: the run's first initial walker) */
  int64_t max_steps;               /* events per walker per interval before WE_ESTEPCAP
                                      (<=0: WE_DEFAULT_MAX_STEPS) */
  int32_t hist_species;            /* species of the weighted histogram */
  int32_t hist_len;                /* histogram entries (0: none); the last one collects x >= hist_len-1 */
  int32_t resample;                /* 1: weighted ensemble; 0: plain SSA propagation */
  int32_t mapping;                 /* WE_MAP_AUTO / WE_MAP_THREAD / WE_MAP_WARP */
  int32_t block_threads;           /* threads per block of the SSA kernel (0: auto).  Thread
                                      mappings: 128 = one event warp fed by three draw warps
                                      per 32 walkers (default); 32, 64, 96 = every thread
                                      makes its own draws */
  int32_t reweight_period;         /* 0: off.  > 0: steady-state reweighting (Sec. II.B.2,
                                      Eq. "ss") after the split/merge of iterations period-1,
                                      2 period-1, ... (iteration indices counted from 0 for
                                      the run, so a resumed run keeps the schedule): the rates
                                      k_ij = F_ij / W_j
                                      from the weight F_ij that moved from bin j to bin i over
                                      all intervals so far (W_j = sum_i F_ij), the balance
                                      equations solved on the largest strongly connected set
                                      of bins with W_j > 0 (elimination of Grassmann, Taksar
                                      and Heyman, which keeps every weight's relative
                                      accuracy), and the walkers of each of its bins that
                                      holds any rescaled to the solved bin weights (their
                                      total kept); the outcome per iteration is WE_OUT_RW.
                                      Needs resample = 1 and at most 1024 bins; adds
                                      16 * n_bins^2 bytes per run to the workspace */
  const int32_t *n_init_per_run;   /* n_runs initial walker counts, each 1..n_init (NULL: n_init
                                      for every run); run r uses the first n_init_per_run[r]
                                      walkers of its n_init rows of init_states/init_weights */
} we_run_config;

/* ------------------------------------------------------------------------------------------
 * Ensemble: the walkers of every run of a batch, resident in device memory as
 * structure-of-arrays (counts int32[S][runs*capacity], weights double[runs*capacity]).
 *
 * we_ensemble_workspace_bytes: device bytes an ensemble needs for (net, bins, cfg).
 * we_ensemble_create: validates, compiles the device tables and uploads the initial walkers.
 *   workspace: caller-owned device buffer of at least workspace_bytes (256-byte aligned), or
 *   NULL to let the library allocate.  The workspace must outlive the ensemble.
 * Errors: WE_EINVAL, WE_ENOMEM (also when workspace_bytes is too small), WE_ECUDA.
 * ------------------------------------------------------------------------------------------ */
typedef struct we_ensemble we_ensemble;
we_status we_ensemble_workspace_bytes(const we_network *net, const we_binmap *bins,
                                      const we_run_config *cfg, size_t *bytes);
we_status we_ensemble_create(const we_network *net, const we_binmap *bins,
                             const we_run_config *cfg, void *workspace, size_t workspace_bytes,
                             void *stream, we_ensemble **out);
we_status we_ensemble_destroy(we_ensemble *ens);

/* One SSA interval of length tau for every live walker (Sec. II.A; the "propagate dynamics"
 * step of the WE algorithm), with in-interval recycling when feedback is on, followed by bin
 * assignment and the observables of the interval.  Enqueue only. */
we_status we_ensemble_propagate(we_ensemble *ens, void *stream);
/* Split/merge of every occupied bin of every run (Sec. II.B): afterwards each occupied bin
 * holds m_targ walkers and each bin keeps its total weight.  Advances the iteration counter.
 * Enqueue only. */
we_status we_ensemble_resample(we_ensemble *ens, void *stream);
/* Which kernels carry out the grouping by bin and the split/merge of we_ensemble_resample
 * (Sec. II.B); every choice gives the same walkers, weights, parents and observables.
 * kind: WE_RESAMPLE_AUTO (default), WE_RESAMPLE_CHAIN, WE_RESAMPLE_ONE_LAUNCH.  blocks_per_run
 * (0..32, 0: about one bin per two warps, at most 16, and at most two blocks per SM over all
 * runs) applies to
 * ONE_LAUNCH: each block of a run groups the run's walkers itself and splits/merges the bins
 * whose task index is its own modulo blocks_per_run.  ONE_LAUNCH needs 24 n_bins + 16 capacity
 * bytes of shared memory per block (within the device's opt-in limit) and at most 8 species.
 * Call between iterations; synchronises the device and drops the captured iteration graphs.
 * Errors: WE_EINVAL (NULL ensemble, unknown kind, blocks_per_run out of range, ONE_LAUNCH that
 * does not fit, a propagate without its resample pending). */
we_status we_ensemble_set_resample_kernel(we_ensemble *ens, int32_t kind, int32_t blocks_per_run);
/* n_iters full WE iterations (propagate + resample), replayed from a CUDA graph captured on
 * the first call.  Enqueue only.  Errors: WE_EOVERFLOW if record_iters would be exceeded. */
we_status we_ensemble_step(we_ensemble *ens, int32_t n_iters, void *stream);
/* Kernel launches of one WE iteration: the kernel nodes of the iteration graph that
 * we_ensemble_step replays (captured here if it does not exist yet; nothing runs).
 * Errors: WE_EINVAL (NULL argument, a propagate without its resample pending), WE_ECUDA. */
we_status we_ensemble_iteration_kernels(we_ensemble *ens, int32_t *n_kernels);
/* The same n_iters iterations as we_ensemble_step, with the device time of every iteration's
 * SSA kernel measured by CUDA events recorded on `stream` on either side of it; synchronises
 * the stream and writes n_iters durations in milliseconds to propagate_ms (host array).  The
 * events come from a per-device pool that the library creates on first need and keeps for the
 * life of the process (2 per iteration), so nothing is created or destroyed while the launches
 * run; timed calls on one device must not overlap in time.  n_iters = 0 only captures the
 * timed graph (nothing runs), so that a later timed call launches at once. */
we_status we_ensemble_step_timed(we_ensemble *ens, int32_t n_iters, void *stream,
                                 float *propagate_ms);
/* we_ensemble_step_timed with only every `every`-th iteration (0, every, 2 every, ...) timed
 * and the others replayed from the plain graph: ceil(n_iters / every) durations are written.
 * The event-record nodes cost the timed iterations a few microseconds each; sampling keeps the
 * timed run close to we_ensemble_step's. */
we_status we_ensemble_step_timed_every(we_ensemble *ens, int32_t n_iters, int32_t every, void *stream,
                                       float *propagate_ms);

/* Checkpoint of an ensemble between iterations: every run's live walkers (counts and weights,
 * in slot order), the next iteration index, and, with steady-state reweighting on, the
 * accumulated transfers and the bin layout of the last split/merge.  Synchronises the stream.
 * dst (host) may be NULL to query the size (*needed).  The walkers and the counter-based
 * random numbers are the whole state of the dynamics, so a resumed ensemble continues exactly
 * as the original would have.  Errors: WE_EINVAL (between propagate and resample, or dst too
 * small), WE_ECUDA. */
we_status we_ensemble_checkpoint(we_ensemble *ens, void *dst, size_t dst_bytes, size_t *needed,
                                 void *stream);
/* A new ensemble continuing from a checkpoint: cfg gives everything but the walkers, their
 * per-run counts and the first iteration, which come from the checkpoint (cfg's n_init,
 * init_states, init_weights, n_init_per_run and first_iter are ignored; give recycle_state
 * explicitly for feedback runs -- its default, the first initial walker, would be the
 * checkpoint's).  The checkpoint must have cfg's run count and the network's species count;
 * reweighting data is restored when cfg reweights over the same bins (and is otherwise
 * refused).  Device memory is allocated by the library.  Errors: WE_EINVAL (malformed or
 * mismatched checkpoint), and those of we_ensemble_create. */
we_status we_ensemble_resume(const we_network *net, const we_binmap *bins, const we_run_config *cfg,
                             const void *checkpoint, size_t checkpoint_bytes, void *stream,
                             we_ensemble **out);
/* Synchronise the stream and return the first non-OK device status of any run (or WE_OK). */
we_status we_ensemble_sync(we_ensemble *ens, void *stream);

/* Outputs.  `what` selects an array; `run` selects a run (or -1 for all runs, concatenated).
 * dst may be host or device memory (copied with cudaMemcpyDefault after synchronising the
 * stream); dst == NULL only returns the byte count in *needed.  Layouts:
 *   WE_OUT_COUNTS    int32[runs]                    live walkers per run
 *   WE_OUT_STATES    int32[n_live x S]              walker-major counts of one run (run = -1:
 *                                                   of all runs, concatenated in run order)
 *   WE_OUT_WEIGHTS   double[n_live]
 *   WE_OUT_PARENT    int32[n_live]                  slot before the last resampling
 *   WE_OUT_FLUX      double[iters x runs]           recycled weight per interval
 *   WE_OUT_TOTAL_W   double[iters x runs]           sum of weights after resampling
 *   WE_OUT_NWALKERS  int32[iters x runs]            walkers after resampling
 *   WE_OUT_EVENTS    int64[iters x runs]            SSA events fired per interval
 *   WE_OUT_HIST      double[iters x runs x hist_len] weighted histogram after propagation
 *   WE_OUT_STATUS    int32[runs]                    first device status of each run
 *   WE_OUT_ITER      int32[1]                       next iteration index
 *   WE_OUT_RECORDED  int32[1]                       iterations of observables recorded
 *   WE_OUT_TLAST     double[n_prev]                 time of each walker's last event in the
 *                                                   last propagated interval (0 if none), by
 *                                                   the slot it held then (before resampling)
 *   WE_OUT_Z         float[n_prev]                  learned coordinate of each walker at the end
 *                                                   of the last interval (learned bin maps)
 *   WE_OUT_NREC      int32[n_prev]                  recycles of each walker in the last interval
 *   WE_OUT_RW        int32[iters x runs]            steady-state reweighting per iteration: 1 done,
 *                                                   -1 attempted and skipped, 0 not scheduled
 *   WE_OUT_NEAR_TAU  int32[iters x runs]            walkers whose interval ended near tau: the
 *                                                   last fired event or the first draw past tau
 *                                                   within 2^-40 tau of tau.  The waiting times
 *                                                   are computed to ~1e-14 relative (float-float
 *                                                   logarithm), so such a stop decision may differ
 *                                                   from one taken in other arithmetic; 0 means no
 *                                                   walker was that close
 *   WE_OUT_FPT       double[n_live]                 absorbing runs: each walker's first-passage
 *                                                   time into the target set, counted from the
 *                                                   run's start (iteration 0): fl(fl(i tau) + t)
 *                                                   for an entrance at time t of interval i, or
 *                                                   fl(i tau) for a walker found inside at the
 *                                                   start of interval i; -1 if not (yet) entered
 * Per-iteration arrays hold the recorded iterations in order. */
#define WE_OUT_COUNTS 1
#define WE_OUT_STATES 2
#define WE_OUT_WEIGHTS 3
#define WE_OUT_PARENT 4
#define WE_OUT_FLUX 5
#define WE_OUT_TOTAL_W 6
#define WE_OUT_NWALKERS 7
#define WE_OUT_EVENTS 8
#define WE_OUT_HIST 9
#define WE_OUT_STATUS 10
#define WE_OUT_ITER 11
#define WE_OUT_RECORDED 12
#define WE_OUT_TLAST 13
#define WE_OUT_Z 14
#define WE_OUT_NREC 15
#define WE_OUT_RW 16
#define WE_OUT_FPT 17
#define WE_OUT_NEAR_TAU 18
we_status we_ensemble_get(we_ensemble *ens, int32_t what, int32_t run, void *dst,
                          size_t dst_bytes, size_t *needed, void *stream);

/* Maximum-likelihood transition time of a brute-force campaign (Sec. II.C, Eq. "mld"), per run
 * of an absorbing ensemble (feedback = WE_FEEDBACK_ABSORB): the run's N live walkers are N
 * independent SSA runs of length T from the initial state; the n of them whose first-passage
 * time t_i (WE_OUT_FPT) lies in [0, T] transitioned, the others are censored at T.  Under an
 * exponential law of transition times the likelihood is maximal at
 *     mu = (sum_i t_i + (N - n) T) / n,    with standard error sigma = mu / sqrt(n)
 * (the printed factor (1 - n/N) on T is read as (N/n - 1): only this form reproduces the
 * paper's own brute-force figures of Sec. III.C).  T <= 0 takes the time simulated so far,
 * (next iteration index) x tau; a larger T than that is refused (WE_EINVAL).  Writes runs x 5 doubles (N, n, sum t_i, mu, sigma; mu and
 * sigma are +inf when n = 0) to dst (host or device, dst_bytes >= 40 runs); the sums run on
 * the device in slot order; synchronises the stream.  Errors: WE_EINVAL (not an absorbing
 * ensemble, dst too small, between propagate and resample), WE_ECUDA. */
we_status we_ensemble_fpt_mle(we_ensemble *ens, double T, void *dst, size_t dst_bytes, void *stream);

/* Whole WE procedure in one call (Sec. II.B): create an ensemble in library-owned memory,
 * run cfg->record_iters iterations, synchronise, and return the ensemble for we_ensemble_get.
 * Host inputs, host or device outputs. */
we_status we_run(const we_network *net, const we_binmap *bins, const we_run_config *cfg,
                 void *stream, we_ensemble **out);

/* ------------------------------------------------------------------------------------------
 * Split/merge without allocation.  The paper has no counterpart: this is a service for callers
 * that may not allocate device memory -- for instance a host framework whose caching allocator
 * already holds all of the GPU's memory, or a loop in which a cudaMalloc (which can synchronise
 * the device and can fail under memory pressure) is not allowed after set-up.
 *
 * It applies the same per-bin split/merge as we_ensemble_resample to one run given as plain
 * device arrays: n walkers with their bins (int32, 0..n_bins-1) and weights (double); `iter`,
 * `seed` and `run_id` key the merge draws exactly as in an ensemble.  Outputs (device memory,
 * capacity entries): out_weights and out_parent (input slot of each new walker), in the order
 * the ensemble uses; out_count[0] receives the new walker count, or a negative we_status
 * (WE_EINVAL for a bin out of range, WE_EOVERFLOW when capacity is too small).
 *
 * Working memory is one array of about 1.4 MB in device global memory, part of the library
 * image, that every GPU loading the library keeps until the process exits.  Limits: n and
 * capacity at most WE_STATIC_MAX_WALKERS, n_bins at most WE_STATIC_MAX_BINS (larger sizes
 * return WE_EINVAL); capacity >= n.  The first call on each device looks up the array's device
 * address (cudaGetSymbolAddress), so make that first call before any stream capture.  Every
 * call shares the array: calls whose GPU work can overlap (other streams, other threads) race
 * and give wrong results; order them on one stream.  Enqueue only; the call allocates nothing.
 * ------------------------------------------------------------------------------------------ */
#define WE_STATIC_MAX_WALKERS 65536
#define WE_STATIC_MAX_BINS 4096
we_status we_resample_static(int32_t n, const int32_t *bins, const double *weights,
                             int32_t n_bins, int32_t m_targ, int32_t iter, uint64_t seed,
                             uint32_t run_id, int32_t capacity, double *out_weights,
                             int32_t *out_parent, int32_t *out_count, void *stream);

/* ------------------------------------------------------------------------------------------
 * Measured denominators for the kernels' rooflines (not part of the method).
 *
 * we_measure_alu_peaks: whole-GPU throughput of FP64 fused multiply-adds, 32-bit integer
 *   multiply-adds and 32-bit integer ALU operations (xor, add), in lane operations per second,
 *   each from one CUDA-event-timed launch of independent chains on every SM after a warm-up
 *   launch.  Allocates 64 bytes of device memory for the duration of the call; synchronises the
 *   stream.  Errors: WE_EINVAL (NULL output), WE_ECUDA.
 * we_measure_graph_floor: the launch-latency floor of one WE iteration: milliseconds per replay
 *   of a CUDA graph of `kernels` (1..64) empty launches of one block per SM, replayed n_replays
 *   times back to back.  Synchronises the stream.  Errors: WE_EINVAL, WE_ECUDA.
 * ------------------------------------------------------------------------------------------ */
we_status we_measure_alu_peaks(void *stream, double *fp64_fma_per_s, double *imad_per_s,
                               double *ialu_per_s);
we_status we_measure_graph_floor(int32_t kernels, int32_t n_replays, void *stream, double *ms_per_replay);

/* Autotuner: time the SSA kernel mappings and block sizes on a short probe of this
 * configuration and return the fastest (mapping, block_threads).  Results are cached per
 * (device name, S, M, walker slots, initial walkers) for the life of the process; the cache
 * can be saved to and merged from a text file (one entry per line: device S M walker_slots
 * n_init mapping block_threads) and cleared.  Errors of the file calls: WE_EINVAL (unreadable
 * or unwritable file, malformed line; entries before a malformed line are kept). */
we_status we_autotune(const we_network *net, const we_binmap *bins, const we_run_config *cfg,
                      void *stream, int32_t *mapping, int32_t *block_threads);
we_status we_autotune_cache_save(const char *path);
we_status we_autotune_cache_load(const char *path);
void we_autotune_cache_clear(void);

#ifdef __cplusplus
}
#endif
#endif
