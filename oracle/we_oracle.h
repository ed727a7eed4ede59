/*
 * we_oracle.h -- plain, slow, single-threaded CPU oracle for the weighted-ensemble (WE)
 * Gillespie-SSA hot path of Donovan, Sedgewick, Faeder & Zuckerman, "Efficient stochastic
 * simulation of chemical kinetics networks using a weighted ensemble of trajectories"
 * (arXiv:1303.5986).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or calls this code;
 * only the test suite, the package smoke check and the benchmark's CPU-baseline leg do.  It
 * shares no source with the CUDA path: every rule below is restated from the paper and written
 * out independently.
 *
 * What it computes (each function cites the passage it follows):
 *   - Philox-4x32-10 counter-based random numbers (Salmon, Moraes, Dror & Shaw, SC'11),
 *     used because the paper's SSA draws (Sec. II.A) must be reproducible per walker;
 *   - mass-action propensities with combinatorial factors (the Schloegl model, Eq. "schlogl",
 *     whose bistable modes at X=82/563 fix this convention, Sec. III.B.3) and Hill-repression
 *     propensities (epigenetic switch, Sec. III.C.1);
 *   - Gillespie's direct SSA for one WE interval tau (Sec. II.A, and the WE algorithm of
 *     Sec. II.B), with steady-state recycling ("feedback", Sec. II.B.2, Eq. "mfpt");
 *   - static grid bins, split (replicate) and merge (prune) per bin (Sec. II.B and its WE
 *     algorithm listing), and the per-iteration observables the paper reads off: bin-free
 *     weighted histograms of a species (Sec. II.B.1) and the recycled flux (Eq. "mfpt").
 *
 * Points the paper leaves open are fixed by one reading each; every reading is stated beside
 * the code that implements it (in this header or in we_oracle.c).
 */
#ifndef WE_ORACLE_H
#define WE_ORACLE_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_EOVERFLOW = -4, ORC_ESTEPCAP = -5 };
enum { ORC_MASS_ACTION = 0, ORC_HILL_REPRESSION = 1 };
enum { ORC_OP_GE = 0, ORC_OP_LE = 1 };
/* Largest species count a walker may hold; products of up to three counts then fit in int64. */
#define ORC_MAX_COUNT 2097151
/* Events one walker may fire in one interval when no cap is configured (then ORC_ESTEPCAP). */
#define ORC_DEFAULT_MAX_STEPS (1ll << 26)

typedef struct {
  int32_t n_species, n_reactions;
  const int32_t *reac_ptr, *reac_species, *reac_mult;   /* CSR over reactions, n_reactions+1 */
  const int32_t *prod_ptr, *prod_species, *prod_mult;
  const double *rate;                                    /* c_j, n_reactions */
  const int32_t *rate_law;                               /* ORC_MASS_ACTION / ORC_HILL_REPRESSION, may be NULL */
  const int32_t *hill_species;                           /* regulator species per reaction, may be NULL */
  const double *hill_K;                                  /* per reaction, may be NULL */
  const int32_t *hill_n;                                 /* per reaction, may be NULL */
  const int32_t *fixed_count;                            /* per species: -1 dynamic, >=0 held constant; may be NULL */
} orc_network_in;

typedef struct orc_net orc_net;

typedef struct {
  double tau;
  int32_t m_targ, n_iters, first_iter;
  uint64_t seed;
  uint32_t run_id;
  int32_t n_init;                    /* initial walkers */
  const int32_t *init_states;        /* n_init x S, walker-major */
  const double *init_weights;        /* n_init */
  /* grid bin map: up to 4 dims; dim d has n_bins[d] bins given by n_bins[d]+1 ascending edges */
  int32_t bin_ndim;
  int32_t bin_species[4];
  int32_t bin_nbins[4];
  const double *bin_edges;           /* concatenated */
  /* optional per-walker bin override (learned bins are assigned outside and passed per call) */
  int32_t feedback;                  /* 0: none; 1: recycle walkers entering the target set
                                        (Sec. II.B.2); 2: absorb them -- a walker stops at its
                                        first entrance and stays there (the brute-force
                                        transition-time runs of Sec. II.C; resample = 0 only);
                                        3: check the target set at the end of each interval
                                        only and recycle a walker found in it (B checked at a
                                        prescribed time step, Sec. IV) */
  int32_t n_clauses;                 /* target set = AND of clauses  x[species] op threshold */
  int32_t tgt_species[4], tgt_op[4], tgt_threshold[4];
  const int32_t *recycle_state;      /* S */
  int64_t max_steps;                 /* per walker per interval; <=0: ORC_DEFAULT_MAX_STEPS */
  int32_t capacity;                  /* walker slots */
  int32_t hist_species, hist_len;    /* weighted histogram of one species, last entry = overflow */
  int32_t resample;                  /* 0: plain propagation (no split/merge) */
  int32_t reweight_period;           /* >0: steady-state reweighting (Eq. "ss") after the
                                        resampling of iterations period-1, 2 period-1, ... */
} orc_we_config;

typedef struct {
  /* per iteration (n_iters entries each) */
  double *flux_weight;               /* recycled weight during the interval */
  double *total_weight;              /* sum of weights after resampling */
  int32_t *n_walkers;                /* walkers after resampling */
  int64_t *events;                   /* SSA events fired during the interval */
  double *hist;                      /* n_iters x hist_len, before resampling; may be NULL */
  /* final ensemble (capacity entries) */
  int32_t *states;                   /* capacity x S */
  double *weights;
  int32_t *parent;                   /* slot of the parent in the previous interval */
  double *t_last;                    /* capacity: last event time of each walker in the last
                                        interval, by slot before resampling (may be NULL) */
  int32_t n_final;
  int32_t status;
  double *first_passage;             /* capacity, may be NULL; plain runs (resample = 0) with
                                        feedback = 2: time from the run's start (iteration 0)
                                        at which the walker of each slot first entered the
                                        target set, fl(fl(iter * tau) + t) for an entrance at
                                        time t of interval iter (fl(iter * tau) for a walker
                                        found inside at the start of an interval); -1 if it
                                        has not entered */
  int32_t *reweighted;               /* per iteration: 1 reweighted, -1 attempted and skipped,
                                        0 not a reweighting iteration (may be NULL) */
} orc_we_out;

/* Philox-4x32-10 block function: out = philox(ctr, key). */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
/* Uniform in (0,1) from two 32-bit words: m = hi<<20 | lo>>12 (52 bits), u = (2m+1)/2^53 (exact). */
double orc_u01(uint32_t hi, uint32_t lo);

int orc_net_create(const orc_network_in *in, orc_net **out);
void orc_net_destroy(orc_net *net);
int32_t orc_net_n_species(const orc_net *net);
int32_t orc_net_n_reactions(const orc_net *net);
/* Effective rate constant after folding held-constant species. */
double orc_net_keff(const orc_net *net, int32_t j);
/* a[j] for every reaction at state x. */
void orc_propensities(const orc_net *net, const int32_t *x, double *a);
/* Canonical total propensity: pairwise tree over leaves padded to a power of two. */
double orc_tree_total(int32_t n, const double *a);
/* Reaction selected by a tree descent on target in [0, total). */
int32_t orc_tree_select(int32_t n, const double *a, double target);

/* One walker for one interval; returns status.  *n_rec = recycles (feedback 2: 1 if the walker
 * entered the target set in this interval), *n_ev = events fired, *t_last = time of the last
 * event fired in the interval (0 if none; may be NULL). */
int orc_propagate(const orc_net *net, const orc_we_config *cfg, int32_t iter, int32_t slot,
                  int32_t *x, int64_t *n_ev, int32_t *n_rec, double *t_last);
int32_t orc_bin_of(const orc_we_config *cfg, const int32_t *x);

/* Split/merge of one ensemble, given every walker's bin.  Inputs are n walkers (states S wide).
 * Writes the resampled ensemble to out_states/out_weights/out_parent and returns its size,
 * or a negative status. */
int32_t orc_resample(int32_t n, int32_t n_species, const int32_t *states, const double *weights,
                     const int32_t *bins, int32_t n_bins, int32_t m_targ, int32_t iter,
                     uint64_t seed, uint32_t run_id, int32_t capacity,
                     int32_t *out_states, double *out_weights, int32_t *out_parent);

/* Steady-state reweighting (Sec. II.B.2, Eq. "ss").  F[e * n_bins + b] holds the weight that
 * moved from bin b (start of an interval) to bin e (its end), summed over the intervals seen;
 * cb[b] the current weight of bin b.  Writes fac[b] = the factor for the walkers of bin b
 * (0: leave them as they are) and returns 1, or returns -1 when no reweighting is possible. */
int32_t orc_rw_solve(int32_t n_bins, const double *F, const double *cb, double *fac);

/* The whole WE run of the paper's algorithm listing (Sec. II.B). */
int orc_we_run(const orc_net *net, const orc_we_config *cfg, orc_we_out *out);

/* CPU baseline, not part of the oracle's definition: the same SSA with a dependency graph
 * (only the propensities a fired reaction can change are recomputed, with their tree paths),
 * for a CPU throughput figure that is not the oracle's full recomputation.  Same results as
 * orc_propagate / orc_we_run (no steady-state reweighting). */
typedef struct orc_dg orc_dg;
int orc_dg_create(const orc_net *net, orc_dg **out);
void orc_dg_destroy(orc_dg *g);
int orc_propagate_dg(const orc_dg *g, const orc_we_config *cfg, int32_t iter, int32_t slot,
                     int32_t *x, int64_t *n_ev, int32_t *n_rec, double *t_last);
int orc_we_run_dg(const orc_dg *g, const orc_we_config *cfg, orc_we_out *out);

#ifdef __cplusplus
}
#endif
#endif
