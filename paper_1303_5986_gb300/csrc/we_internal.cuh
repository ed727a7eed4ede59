// we_internal.cuh -- device-side data layout and kernel parameters shared by the library's
// host code and kernels.  Not part of the public ABI (include/we_ssa.h is).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace we {

constexpr int kMaxClauses = 4;
constexpr int kMaxBinDims = 4;
constexpr int kMaxReactantSlots = 3;
constexpr int kThreadMaxLeaves = 16;     // thread-per-walker kernel: propensity tree in registers
constexpr int kThreadMaxSpecies = 32;    // thread-per-walker kernel: counts staged in shared memory
constexpr int32_t kMaxCount = 2097151;   // same bound as WE_MAX_COUNT

// Per-reaction description used by every SSA kernel (int32 words, 16 per reaction).
//   n_reac: dynamic reactant slots (0..3); sp[k], m[k]: species and multiplicity;
//   law: 0 mass action, 1 Hill repression; hsp, hn: regulator species and Hill exponent;
//   d_begin/d_end: range of this reaction's net changes in the delta arrays.
struct RxnMeta {
  int32_t n_reac;
  int32_t sp[kMaxReactantSlots];
  int32_t m[kMaxReactantSlots];
  int32_t law;
  int32_t hsp;
  int32_t hn;
  int32_t d_begin;
  int32_t d_end;
  int32_t pad[4];
};
static_assert(sizeof(RxnMeta) == 64, "RxnMeta is 64 bytes");

// Device view of a compiled network (all pointers into the ensemble workspace).
struct NetView {
  int32_t S, M, P, log2P;      // P = leaves of the canonical tree (power of two >= M)
  int32_t n_param_sets;
  int32_t n_delta;             // total net-change entries
  const RxnMeta *meta;         // P entries (padding reactions: n_reac = 0, keff = 0)
  const double *keff;          // n_param_sets x P (mass action: folded c; Hill: c*K^n)
  const double *hill_Kn;       // n_param_sets x P
  const int32_t *d_sp;         // n_delta
  const int32_t *d_val;        // n_delta
  // dependency graph: reactions whose propensity reads a species changed by j (CSR over P)
  const int32_t *dep_ptr;      // P + 1
  const int32_t *dep_idx;
  // Per-reaction event records for the warp-per-walker kernel (null for the other mappings):
  // everything one event reads from global memory, at a fixed stride so that it is fetched in
  // one round trip.  Record j, in 16-byte units:
  //   [0]                      (n_changes, n_dependents, d_begin, dep_begin)
  //   [1, 1 + (wrec_chg+1)/2)  the first wrec_chg net changes as int2 (species, change);
  //                            unused entries have species -1
  //   then wrec_dep entries of 32 bytes, one per dependent reaction i (dep_idx order):
  //     int4 (i | packed << 20, sp0, sp1, sp2), double2 (keff, Kn) of parameter set 0;
  //     packed = n_reac | hill << 2 | hn << 3 | m0 << 5 | m1 << 7 | m2 << 9 (sp0 = hsp for a
  //     Hill term); unused entries have word 0 = -1.
  // Changes and dependents past these counts are read from d_sp/d_val and dep_idx/meta.
  const int4 *wrec;
  int32_t wrec_stride, wrec_chg, wrec_dep;
};

// Learned progress coordinate: z = w3 . silu(W2 silu(W1 phi + b1) + b2) + b3 with
// phi_s = log1p(x_s) for every species, weights in BF16 (rounded from FP32 master weights),
// arithmetic in FP32.
struct MlpView {
  int32_t n_in, hidden;
  const uint16_t *w1;          // hidden x n_in, BF16 bits
  const uint16_t *w2;          // hidden x hidden
  const uint16_t *w3;          // hidden
  const float *b1, *b2, *b3;   // hidden, hidden, 1
};

struct BinView {
  int32_t ndim;
  int32_t n_bins;
  int32_t species[kMaxBinDims];
  int32_t nb[kMaxBinDims];
  int32_t edge_off[kMaxBinDims];
  // Dimensions whose inner edges e_1 .. e_{nb-1} are integers e_1 + (k - 1) h (ustep = h > 0):
  // the bin of a count comes from one division instead of a search of the edges in memory.
  int32_t ufirst[kMaxBinDims], ustep[kMaxBinDims];
  const double *edges;
  int32_t learned;             // 1: bins are intervals of the learned coordinate z
  MlpView mlp;
  const float *zedges;         // n_bins + 1 ascending edges on z
  float *zout;                 // per walker slot: z of the last interval (may be null)
};

// Ensemble state on the device.  Global slot g = run * cap + w.
struct EnsView {
  int32_t R, cap, S;
  int32_t m_targ;
  int32_t record_iters;
  int32_t first_iter;
  int32_t hist_species, hist_len;
  int32_t feedback, n_clauses;  // feedback inside the interval: 0 none, 1 recycle, 2 absorb
  int32_t end_check;           // 1: the target set is checked at the interval's end only
  int32_t tgt_species[kMaxClauses];
  int32_t tgt_op[kMaxClauses];
  int64_t max_steps;
  double tau;
  uint64_t seed;
  // per-run constants
  const uint32_t *run_id;      // R
  const int32_t *param_set;    // R
  const int32_t *tgt_thr;      // R x n_clauses
  const int32_t *recycle;      // R x S
  // walker arrays, double-buffered by iteration parity
  int32_t *x[2];               // S x (R*cap)
  double *w[2];                // R*cap
  int32_t *parent[2];          // R*cap
  int32_t *bin;                // R*cap  bin of each walker after propagation
  int32_t *nrec;               // R*cap  recycles of each walker in the last interval
  double *tlast;               // R*cap  time of each walker's last event in the last interval
  double *fpt;                 // R*cap  absorbing runs: first-passage time from the run's start
                               //        (-1: none yet); null unless feedback = 2
  // per-run bookkeeping
  int32_t *count;              // R      live walkers
  int32_t *prev_count;         // R      walkers propagated in the last interval
  int32_t *run_off;            // R + 1  exclusive prefix of count
  int32_t *status;             // R
  int32_t *iter;               // 1      current iteration index (absolute)
  int32_t *bin_count;          // R x n_bins
  int32_t *n_tasks;            // R
  int4 *tasks;                 // R x n_bins: (bin, in_offset, count, out_offset)
  int32_t *cursor;             // R x n_bins: next free position of each bin while grouping
  int32_t *sorted_slot;        // R*cap   walkers grouped by bin (scratch)
  double *sorted_w;            // R*cap
  int32_t *alive;              // R*cap
  const unsigned long long *div_magic;   // [m_targ + 1]: floor((2^64 - 1) / c) for c >= 2
  // observables, record_iters x R (x hist_len)
  double *obs_flux;
  double *obs_totw;
  int32_t *obs_nw;
  unsigned long long *obs_events;
  double *obs_hist;
  int32_t *obs_near;           // walkers whose interval ended within 2^-40 tau of an event
};

// Tables of the waiting-time logarithm (see neg_log_u01), each value as an unevaluated sum
// of two floats (hi, lo): cb[j] = (1/c_j, -log(c_j / 2)) side by side, so that a draw fetches
// both with one 16-byte shared-memory load; n_ln2[i] = i ln 2.
struct LogTables {
  float4 cb[128];
  float2 n_ln2[64];
};

// State-indexed propensity tables for networks whose propensities all depend on one species:
// row x (x < len) holds [1/a0, tree node 1 (= a0), node 2, ..., node 2P-1] at that count.
// Fixed-point clock of the table kernels: integer units of tau / 2^kClockBits.
constexpr int kClockBits = 62;
constexpr unsigned long long kClockTau = 1ull << kClockBits;

// State-indexed table: per parameter set, len x lenB rows of P 64-bit words, row x * lenB + y
// for count x of `species` and count y of `species2` (lenB = 1, y = 0 for one species):
//   word 0      float-float (2^62 / tau) / a0 (hi in the low half; 0 when a0 = 0)
//   words 1..   the P-1 breakpoints b_i on the 52-bit uniform index (see k_build_table)
struct TableView {
  const unsigned long long *rows;
  int32_t len;                 // counts of `species` covered; larger counts are evaluated directly
  int32_t lenB;                // counts of `species2` covered (1 without a second species)
  int32_t species;             // the species the propensities read (-1: no tables)
  int32_t species2;            // the second one (-1: one-species table)
  int32_t smem_rows;           // rows a block of the warp-specialised kernel stages in shared memory
  double clock_scale;          // 2^62 / tau, for rows evaluated on the fly
};

// Steady-state reweighting (Sec. II.B.2, Eq. "ss"): per run, the weight moved from bin b to
// bin e summed over the intervals so far (F, nb x nb, row e), the solve's scratch (M, n x n
// over the bins solved for), per-bin vectors and the per-iteration outcome.
struct RwView {
  int32_t period;              // 0: off; else reweight after every period-th iteration
  int32_t nb;                  // bins
  int32_t start_known;         // 1: the first interval's start bins are known (resumed ensemble)
  double *F;                   // R x nb x nb
  double *M;                   // R x nb x nb
  double *W, *cb, *x, *fac;    // R x nb each
  int32_t *act;                // R x nb: the bins solved for, ascending
  int32_t *iscr;               // R x 6 nb: scratch of the strongly-connected-set search
  int32_t *obs;                // record_iters x R: 1 reweighted, -1 skipped, 0 not scheduled
};

// Every device allocation of the library goes through here, so that a test can make the n-th
// one fail as if the device were out of memory (we_debug_fail_allocation).
cudaError_t device_alloc(void **p, size_t bytes);

struct PropagateParams {
  NetView net;
  BinView bins;
  EnsView ens;
  TableView tab;
  const LogTables *logt;
  int32_t resample;            // 1: WE; 0: plain SSA (bookkeeping of parents is identity)
  RwView rw;
};

}  // namespace we
