// we_host.cu -- host side of the C ABI declared in include/we_ssa.h: validation, network
// compilation (constant folding, net changes, dependency graph), device workspace layout,
// kernel launches and CUDA-graph replay of whole WE iterations.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/we_ssa.h"
#include "we_internal.cuh"
#include "we_exact.cuh"
#include "we_mlp.cuh"

namespace we {
cudaError_t launch_propagate_thread(const PropagateParams &prm, int block, bool table, cudaStream_t st);
cudaError_t launch_propagate_ws(const PropagateParams &prm, bool table, cudaStream_t st);
cudaError_t launch_propagate_warp(const PropagateParams &prm, int block, cudaStream_t st);
cudaError_t launch_init_log_tables(LogTables *T, cudaStream_t st);
cudaError_t launch_build_table(const NetView &N, const int32_t *base, int species, int species2, int len,
                               int lenB, double clock_scale, unsigned long long *rows, cudaStream_t st);
size_t propagate_warp_smem(const NetView &N, int block);
cudaError_t launch_resample_chain(const PropagateParams &prm, cudaStream_t st);
cudaError_t launch_gather_finalize(const PropagateParams &prm, cudaStream_t st);
size_t resample_run_smem(const EnsView &E, int n_bins);
cudaError_t resample_run_prepare();
cudaError_t launch_resample_run(const PropagateParams &prm, int blocks_per_run, cudaStream_t st);
cudaError_t launch_fpt_mle(const EnsView &E, double T, double *out, cudaStream_t st);
cudaError_t launch_pack_states(const EnsView &E, int r, int32_t *out, cudaStream_t st);
cudaError_t launch_learned_bins(const PropagateParams &prm, cudaStream_t st);
size_t learned_bins_smem(int n_in, int H);
cudaError_t launch_rw_flux(const PropagateParams &prm, cudaStream_t st);
cudaError_t launch_rw_solve_apply(const PropagateParams &prm, cudaStream_t st);
}  // namespace we

using namespace we;

// ------------------------------------------------------------------------------------------
// errors
// ------------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static we_status fail(we_status code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

static we_status cuda_fail(cudaError_t e, const char *what) {
  return fail(WE_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define WE_CUDA_TRY(call)                                   \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);     \
  } while (0)

extern "C" const char *we_status_string(we_status s) {
  switch (s) {
    case WE_OK: return "WE_OK";
    case WE_EINVAL: return "WE_EINVAL";
    case WE_ENOMEM: return "WE_ENOMEM";
    case WE_ECUDA: return "WE_ECUDA";
    case WE_EOVERFLOW: return "WE_EOVERFLOW";
    case WE_ESTEPCAP: return "WE_ESTEPCAP";
    case WE_ETIMEOUT: return "WE_ETIMEOUT";
    case WE_ENOTSUPPORTED: return "WE_ENOTSUPPORTED";
    default: return "WE_UNKNOWN";
  }
}

extern "C" const char *we_last_error(void) { return g_last_error.c_str(); }

// Fault injection for tests: the n-th device allocation from now on fails (0: none).
static std::atomic<int> g_fail_alloc{0};

extern "C" we_status we_debug_fail_allocation(int32_t nth) {
  if (nth < 0) return fail(WE_EINVAL, "nth must be >= 0");
  g_fail_alloc.store(nth);
  return WE_OK;
}

namespace we {
cudaError_t device_alloc(void **p, size_t bytes) {
  *p = nullptr;
  int n = g_fail_alloc.load();
  while (n > 0) {
    if (g_fail_alloc.compare_exchange_weak(n, n - 1)) {
      if (n == 1) return cudaErrorMemoryAllocation;        // the armed allocation
      break;
    }
  }
  return cudaMalloc(p, bytes);
}
}  // namespace we
extern "C" int32_t we_version(void) { return 100; }

// ------------------------------------------------------------------------------------------
// network compilation
// ------------------------------------------------------------------------------------------
struct we_network {
  int32_t S = 0, M = 0, P = 1, log2P = 0, nps = 1;
  std::vector<RxnMeta> meta;        // P
  std::vector<double> keff, Kn;     // nps x P
  std::vector<int32_t> d_sp, d_val;
  std::vector<int32_t> dep_ptr, dep_idx;
  std::vector<int32_t> fixed;       // S
  int32_t table_species = -1;       // the species every propensity reads (-1: no tables) ...
  int32_t table_species2 = -1;      // ... and a second one (two-species tables; -1: one species)
};

static long long binom_small_h(long long x, int m) {
  return m == 1 ? x : (m == 2 ? x * (x - 1) / 2 : x * (x - 1) * (x - 2) / 6);
}

extern "C" we_status we_network_create(int32_t S, int32_t M, const int32_t *reac_ptr,
                                       const int32_t *reac_species, const int32_t *reac_mult,
                                       const int32_t *prod_ptr, const int32_t *prod_species,
                                       const int32_t *prod_mult, int32_t nps, const double *rate,
                                       const int32_t *rate_law, const int32_t *hill_species,
                                       int32_t hill_K_rows, const double *hill_K,
                                       const int32_t *hill_n, const int32_t *fixed_count,
                                       we_network **out) {
  if (!out) return fail(WE_EINVAL, "out is NULL");
  *out = nullptr;
  if (S < 1 || M < 1) return fail(WE_EINVAL, "need n_species >= 1 and n_reactions >= 1");
  if (nps < 1) return fail(WE_EINVAL, "n_param_sets must be >= 1");
  if (!reac_ptr || !prod_ptr || !rate) return fail(WE_EINVAL, "reac_ptr, prod_ptr and rate are required");
  if (reac_ptr[0] != 0 || prod_ptr[0] != 0) return fail(WE_EINVAL, "CSR pointers must start at 0");
  for (int j = 0; j < M; ++j)
    if (reac_ptr[j + 1] < reac_ptr[j] || prod_ptr[j + 1] < prod_ptr[j])
      return fail(WE_EINVAL, "CSR pointers must be non-decreasing (reaction %d)", j);
  if ((reac_ptr[M] > 0 && (!reac_species || !reac_mult)) || (prod_ptr[M] > 0 && (!prod_species || !prod_mult)))
    return fail(WE_EINVAL, "species/multiplicity arrays are required");
  bool any_hill = false;
  if (rate_law)
    for (int j = 0; j < M; ++j) {
      if (rate_law[j] != WE_MASS_ACTION && rate_law[j] != WE_HILL_REPRESSION)
        return fail(WE_EINVAL, "reaction %d: unknown rate law %d", j, rate_law[j]);
      any_hill |= rate_law[j] == WE_HILL_REPRESSION;
    }
  if (any_hill && (!hill_species || !hill_K || !hill_n || (hill_K_rows != 1 && hill_K_rows != nps)))
    return fail(WE_EINVAL, "Hill reactions need hill_species, hill_n and hill_K with 1 or n_param_sets rows");
  std::vector<int32_t> fixed(S, -1);
  if (fixed_count)
    for (int s = 0; s < S; ++s) {
      if (fixed_count[s] < -1 || fixed_count[s] > WE_MAX_COUNT)
        return fail(WE_EINVAL, "fixed_count[%d] out of range", s);
      fixed[s] = fixed_count[s];
    }
  for (int i = 0; i < nps * M; ++i)
    if (!(rate[i] >= 0.0) || std::isinf(rate[i])) return fail(WE_EINVAL, "rate[%d] must be finite and >= 0", i);

  we_network *n = new (std::nothrow) we_network();
  if (!n) return fail(WE_ENOMEM, "host allocation");
  n->S = S; n->M = M; n->nps = nps; n->fixed = fixed;
  int P = 1, L = 0;
  while (P < M) { P <<= 1; ++L; }
  n->P = P; n->log2P = L;
  n->meta.assign(P, RxnMeta{});
  n->keff.assign((size_t)nps * P, 0.0);
  n->Kn.assign((size_t)nps * P, 0.0);
  std::vector<std::vector<int32_t>> reads(M);       // dynamic species each propensity reads
  std::vector<std::vector<int32_t>> changes(M);     // dynamic species each reaction changes
  std::vector<long long> rm(S), net(S);
  for (int j = 0; j < M; ++j) {
    std::fill(rm.begin(), rm.end(), 0);
    std::fill(net.begin(), net.end(), 0);
    int order = 0;
    for (int e = reac_ptr[j]; e < reac_ptr[j + 1]; ++e) {
      const int s = reac_species[e], m = reac_mult[e];
      if (s < 0 || s >= S || m < 1 || m > 3) { delete n; return fail(WE_EINVAL, "reaction %d: bad reactant entry", j); }
      rm[s] += m; net[s] -= m; order += m;
    }
    for (int e = prod_ptr[j]; e < prod_ptr[j + 1]; ++e) {
      const int s = prod_species[e], m = prod_mult[e];
      if (s < 0 || s >= S || m < 0) { delete n; return fail(WE_EINVAL, "reaction %d: bad product entry", j); }
      net[s] += m;
    }
    if (order > 3) { delete n; return fail(WE_EINVAL, "reaction %d: reactant order %d > 3", j, order); }
    const int law = rate_law ? rate_law[j] : WE_MASS_ACTION;
    RxnMeta &mt = n->meta[j];
    mt.law = law;
    // held-constant reactants fold into the rate constant, ascending species order
    std::vector<double> fold(nps);
    for (int p = 0; p < nps; ++p) fold[p] = rate[(size_t)p * M + j];
    int nr = 0;
    for (int s = 0; s < S; ++s) {
      if (rm[s] == 0) continue;
      if (fixed[s] >= 0) {
        const double f = (double)binom_small_h(fixed[s], (int)rm[s]);
        for (int p = 0; p < nps; ++p) fold[p] = fold[p] * f;
      } else {
        mt.sp[nr] = s; mt.m[nr] = (int)rm[s]; ++nr;
        reads[j].push_back(s);
      }
    }
    mt.n_reac = nr;
    if (law == WE_HILL_REPRESSION) {
      const int hs = hill_species[j], hn = hill_n[j];
      if (nr != 0) { delete n; return fail(WE_EINVAL, "Hill reaction %d must have no dynamic reactant", j); }
      if (hs < 0 || hs >= S || hn < 1 || hn > 3) { delete n; return fail(WE_EINVAL, "Hill reaction %d: bad species or exponent", j); }
      mt.hsp = hs; mt.hn = hn;
      if (fixed[hs] < 0) reads[j].push_back(hs);
      for (int p = 0; p < nps; ++p) {
        const double K = hill_K[(size_t)(hill_K_rows == 1 ? 0 : p) * M + j];
        if (!(K > 0.0) || std::isinf(K)) { delete n; return fail(WE_EINVAL, "Hill reaction %d: K must be finite and > 0", j); }
        double Kn = K;
        for (int q = 1; q < hn; ++q) Kn = Kn * K;
        n->Kn[(size_t)p * P + j] = Kn;
        n->keff[(size_t)p * P + j] = fold[p] * Kn;
      }
    } else {
      for (int p = 0; p < nps; ++p) n->keff[(size_t)p * P + j] = fold[p];
    }
    mt.d_begin = (int32_t)n->d_sp.size();
    for (int s = 0; s < S; ++s) {
      if (fixed[s] >= 0 || net[s] == 0) continue;
      n->d_sp.push_back(s);
      n->d_val.push_back((int32_t)net[s]);
      changes[j].push_back(s);
    }
    mt.d_end = (int32_t)n->d_sp.size();
  }
  for (int j = M; j < P; ++j) { n->meta[j].d_begin = n->meta[j].d_end = (int32_t)n->d_sp.size(); }
  // dependency graph: i depends on j when i reads a species that j changes
  std::vector<std::vector<int32_t>> readers(S);
  for (int i = 0; i < M; ++i)
    for (int s : reads[i]) readers[s].push_back(i);
  n->dep_ptr.assign(P + 1, 0);
  for (int j = 0; j < P; ++j) {
    std::set<int32_t> d;
    if (j < M)
      for (int s : changes[j])
        for (int i : readers[s]) d.insert(i);
    n->dep_ptr[j] = (int32_t)n->dep_idx.size();
    n->dep_idx.insert(n->dep_idx.end(), d.begin(), d.end());
  }
  n->dep_ptr[P] = (int32_t)n->dep_idx.size();
  // State-indexed tables apply when one or two dynamic species are the only ones any
  // propensity reads and any reaction changes.
  std::set<int32_t> touched;
  for (int j = 0; j < M; ++j) {
    touched.insert(reads[j].begin(), reads[j].end());
    touched.insert(changes[j].begin(), changes[j].end());
  }
  if (touched.size() == 1 || touched.size() == 2) {
    n->table_species = *touched.begin();
    if (touched.size() == 2) n->table_species2 = *touched.rbegin();
  }
  *out = n;
  return WE_OK;
}

extern "C" void we_network_destroy(we_network *n) { delete n; }

extern "C" we_status we_network_keff(const we_network *n, int32_t p, int32_t j, double *out) {
  if (!n || !out || p < 0 || p >= n->nps || j < 0 || j >= n->M) return fail(WE_EINVAL, "bad arguments");
  *out = n->keff[(size_t)p * n->P + j];
  return WE_OK;
}

extern "C" we_status we_network_dep_degree(const we_network *n, int32_t j, int32_t *out) {
  if (!n || !out || j < 0 || j >= n->M) return fail(WE_EINVAL, "bad arguments");
  *out = n->dep_ptr[j + 1] - n->dep_ptr[j];
  return WE_OK;
}

// ------------------------------------------------------------------------------------------
// bin maps
// ------------------------------------------------------------------------------------------
struct we_binmap {
  int32_t ndim = 0, n_bins = 1;
  int32_t species[kMaxBinDims] = {0, 0, 0, 0};
  int32_t nb[kMaxBinDims] = {1, 1, 1, 1};
  int32_t edge_off[kMaxBinDims] = {0, 0, 0, 0};
  std::vector<double> edges;
  bool learned = false;
  we_learned_bins lb;
};

extern "C" we_status we_binmap_learned(const we_mlp *mlp, int32_t n_bins, const float *edges, we_binmap **out) {
  if (!out) return fail(WE_EINVAL, "out is NULL");
  *out = nullptr;
  we_binmap *b = new (std::nothrow) we_binmap();
  if (!b) return fail(WE_ENOMEM, "host allocation");
  we_status st = make_learned_snapshot(mlp, n_bins, edges, &b->lb);
  if (st) { delete b; return fail(st, "learned bin map: need an MLP, 1..65536 bins and ascending edges"); }
  b->learned = true;
  b->n_bins = n_bins;
  b->edges.assign(1, 0.0);
  *out = b;
  return WE_OK;
}

extern "C" we_status we_binmap_grid(int32_t ndim, const int32_t *species, const int32_t *n_bins,
                                    const double *edges, we_binmap **out) {
  if (!out) return fail(WE_EINVAL, "out is NULL");
  *out = nullptr;
  if (ndim < 1 || ndim > kMaxBinDims || !species || !n_bins || !edges)
    return fail(WE_EINVAL, "ndim must be 1..%d with species, n_bins and edges given", kMaxBinDims);
  we_binmap *b = new (std::nothrow) we_binmap();
  if (!b) return fail(WE_ENOMEM, "host allocation");
  b->ndim = ndim;
  long long total = 1;
  int off = 0;
  for (int d = 0; d < ndim; ++d) {
    if (n_bins[d] < 1 || species[d] < 0) { delete b; return fail(WE_EINVAL, "dimension %d: bad species or bin count", d); }
    b->species[d] = species[d];
    b->nb[d] = n_bins[d];
    b->edge_off[d] = off;
    for (int k = 0; k <= n_bins[d]; ++k) {
      const double e = edges[off + k];
      if (std::isnan(e)) { delete b; return fail(WE_EINVAL, "dimension %d: NaN edge", d); }
      if (k > 0 && !(e > edges[off + k - 1])) { delete b; return fail(WE_EINVAL, "dimension %d: edges must ascend", d); }
      b->edges.push_back(e);
    }
    off += n_bins[d] + 1;
    total *= n_bins[d];
    if (total > 65536) { delete b; return fail(WE_EINVAL, "more than 65536 bins"); }
  }
  b->n_bins = (int32_t)total;
  *out = b;
  return WE_OK;
}

// Inner edges e_1 .. e_{nb-1} of one grid dimension that are integers in arithmetic progression
// (e_k = e_1 + (k - 1) h, h a positive integer; any h for nb = 2): first = e_1, step = h, and
// the device bins a count by division.  Otherwise step = 0 (the device searches the edges).
// Limits keep count - e_1 within 32 bits for every count.
static void uniform_inner_edges(const double *e, int nb, int32_t *first, int32_t *step) {
  *first = 0;
  *step = 0;
  if (nb < 2) return;
  const double lim = 1073741824.0;                         // 2^30
  auto is_int = [&](double v) { return std::isfinite(v) && std::fabs(v) <= lim && v == std::floor(v); };
  if (!is_int(e[1])) return;
  long long h = 1;
  if (nb >= 3) {
    if (!is_int(e[2])) return;
    h = (long long)e[2] - (long long)e[1];
    if (h < 1 || h > (long long)lim) return;
  }
  for (int k = 1; k <= nb - 1; ++k)
    if (!is_int(e[k]) || (long long)e[k] != (long long)e[1] + (long long)(k - 1) * h) return;
  *first = (int32_t)e[1];
  *step = (int32_t)h;
}

extern "C" void we_binmap_destroy(we_binmap *b) { delete b; }
extern "C" int32_t we_binmap_n_bins(const we_binmap *b) { return b ? b->n_bins : 0; }

// ------------------------------------------------------------------------------------------
// ensemble: workspace layout
// ------------------------------------------------------------------------------------------
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  }
};

struct Offsets {
  size_t meta, keff, Kn, d_sp, d_val, dep_ptr, dep_idx, edges;
  size_t run_id, param_set, tgt_thr, recycle;
  size_t x0, x1, w0, w1, p0, p1, bin, nrec, tlast, fpt, mle;
  size_t count, prev_count, run_off, status, iter, bin_count, n_tasks, tasks, cursor, sorted_slot, sorted_w, alive, div_magic;
  size_t flux, totw, nw, events, hist, pack, near;
  size_t logt, table, base;
  size_t lw1, lw2, lw3, lb, lz, zout;
  size_t wrec;
  size_t rw_F, rw_M, rw_vec, rw_act, rw_iscr, rw_obs;
  int32_t table_len, table_lenB, wrec_stride;
  size_t total;
};

// Counts covered by the state-indexed table: `len` values of the first species (and `lenB` of
// the second for two-species tables), at most 64 MB over all parameter sets.  0: no table.
static int table_len_for(const we_network *n, int *lenB_out = nullptr) {
  if (lenB_out) *lenB_out = 1;
  if (n->table_species < 0 || n->P > kThreadMaxLeaves || n->S > kThreadMaxSpecies) return 0;
  const size_t budget = 64u << 20, row = (size_t)n->P * 8;
  if (n->table_species2 < 0) {
    int len = 4096;
    while (len > 256 && (size_t)n->nps * len * row > budget) len >>= 1;
    return len;
  }
  int L = 256;
  while (L > 32 && (size_t)n->nps * L * L * row > budget) L >>= 1;
  if ((size_t)n->nps * L * L * row > budget) return 0;
  if (lenB_out) *lenB_out = L;
  return L;
}

static int choose_mapping(const we_network *n, const we_run_config *c) {
  if (c->mapping == WE_MAP_THREAD || c->mapping == WE_MAP_WARP || c->mapping == WE_MAP_THREAD_TABLE)
    return c->mapping;
  if (table_len_for(n) > 0) return WE_MAP_THREAD_TABLE;
  return (n->P <= kThreadMaxLeaves && n->S <= kThreadMaxSpecies) ? WE_MAP_THREAD : WE_MAP_WARP;
}

// Event records of the warp-per-walker kernel (layout documented at NetView::wrec).
struct WarpRecords {
  int32_t stride = 0, chg = 0, dep = 0;     // in 16-byte units; entries kept per record
  std::vector<int32_t> words;               // P x stride x 4
};

static WarpRecords warp_records(const we_network *n) {
  WarpRecords W;
  const int P = n->P;
  int maxc = 0, maxd = 0;
  for (int j = 0; j < P; ++j) {
    maxc = std::max(maxc, n->meta[j].d_end - n->meta[j].d_begin);
    maxd = std::max(maxd, n->dep_ptr[j + 1] - n->dep_ptr[j]);
  }
  W.chg = std::min(maxc, 32);
  W.dep = std::min(maxd, 96);
  W.stride = 1 + (W.chg + 1) / 2 + 2 * W.dep;
  W.words.assign((size_t)P * W.stride * 4, 0);
  for (int j = 0; j < P; ++j) {
    int32_t *r = W.words.data() + (size_t)j * W.stride * 4;
    const RxnMeta &mt = n->meta[j];
    const int nd = n->dep_ptr[j + 1] - n->dep_ptr[j];
    r[0] = mt.d_end - mt.d_begin; r[1] = nd; r[2] = mt.d_begin; r[3] = n->dep_ptr[j];
    int32_t *c = r + 4;
    for (int q = 0; q < W.chg; ++q) {
      const bool have = q < mt.d_end - mt.d_begin;
      c[2 * q] = have ? n->d_sp[mt.d_begin + q] : -1;
      c[2 * q + 1] = have ? n->d_val[mt.d_begin + q] : 0;
    }
    int32_t *d = r + 4 * (1 + (W.chg + 1) / 2);
    for (int q = 0; q < W.dep; ++q) {
      int32_t *e = d + 8 * q;
      if (q >= nd) { e[0] = -1; continue; }
      const int i = n->dep_idx[n->dep_ptr[j] + q];
      const RxnMeta &mi = n->meta[i];
      const int hill = mi.law == WE_HILL_REPRESSION ? 1 : 0;
      const int packed = (mi.n_reac & 3) | hill << 2 | (mi.hn & 3) << 3 | (mi.m[0] & 3) << 5 |
                         (mi.m[1] & 3) << 7 | (mi.m[2] & 3) << 9;
      e[0] = i | packed << 20;
      e[1] = hill ? mi.hsp : mi.sp[0];
      e[2] = mi.sp[1];
      e[3] = mi.sp[2];
      const double kd[2] = {n->keff[i], n->Kn[i]};
      std::memcpy(e + 4, kd, 16);
    }
  }
  return W;
}

static Offsets layout(const we_network *n, const we_binmap *b, const we_run_config *c, int cap) {
  Layout L;
  Offsets o{};
  o.table_len = table_len_for(n, &o.table_lenB);
  o.logt = L.take(sizeof(LogTables));
  if (b->learned) {
    const we_learned_bins &lb = b->lb;
    o.lw1 = L.take(2 * lb.w1.size());
    o.lw2 = L.take(2 * lb.w2.size());
    o.lw3 = L.take(2 * lb.w3.size());
    o.lb = L.take(4 * (2 * (size_t)lb.H + 1));
    o.lz = L.take(4 * lb.zedges.size());
    o.zout = L.take(4 * (size_t)c->n_runs * (size_t)cap);
  }
  o.table = L.take((size_t)n->nps * o.table_len * o.table_lenB * n->P * 8);
  o.base = L.take(4 * (size_t)n->S);
  const size_t R = c->n_runs, RC = R * cap, rec = c->record_iters;
  o.meta = L.take(sizeof(RxnMeta) * n->P);
  o.keff = L.take(8 * n->keff.size());
  o.Kn = L.take(8 * n->Kn.size());
  o.d_sp = L.take(4 * (n->d_sp.size() + 1));
  o.d_val = L.take(4 * (n->d_val.size() + 1));
  o.dep_ptr = L.take(4 * n->dep_ptr.size());
  o.dep_idx = L.take(4 * (n->dep_idx.size() + 1));
  if (choose_mapping(n, c) == WE_MAP_WARP) {
    int maxc = 0, maxd = 0;
    for (int j = 0; j < n->P; ++j) {
      maxc = std::max(maxc, n->meta[j].d_end - n->meta[j].d_begin);
      maxd = std::max(maxd, n->dep_ptr[j + 1] - n->dep_ptr[j]);
    }
    o.wrec_stride = 1 + (std::min(maxc, 32) + 1) / 2 + 2 * std::min(maxd, 96);
    o.wrec = L.take(16 * (size_t)n->P * o.wrec_stride);
  }
  o.edges = L.take(8 * b->edges.size());
  o.run_id = L.take(4 * R);
  o.param_set = L.take(4 * R);
  o.tgt_thr = L.take(4 * R * (c->n_clauses > 0 ? c->n_clauses : 1));
  o.recycle = L.take(4 * R * n->S);
  o.x0 = L.take(4 * RC * n->S);
  o.x1 = L.take(4 * RC * n->S);
  o.w0 = L.take(8 * RC);
  o.w1 = L.take(8 * RC);
  o.p0 = L.take(4 * RC);
  o.p1 = L.take(4 * RC);
  o.bin = L.take(4 * RC);
  o.nrec = L.take(4 * RC);
  o.tlast = L.take(8 * RC);
  o.fpt = c->feedback == WE_FEEDBACK_ABSORB ? L.take(8 * RC) : 0;
  o.mle = c->feedback == WE_FEEDBACK_ABSORB ? L.take(8 * 5 * R) : 0;
  o.count = L.take(4 * R);
  o.prev_count = L.take(4 * R);
  o.run_off = L.take(4 * (R + 1));
  o.status = L.take(4 * R);
  o.iter = L.take(4);
  o.bin_count = L.take(4 * R * b->n_bins);
  o.n_tasks = L.take(4 * R);
  o.tasks = L.take(16 * R * b->n_bins);
  o.cursor = L.take(4 * R * b->n_bins);
  o.sorted_slot = L.take(4 * RC);
  o.sorted_w = L.take(8 * RC);
  o.alive = L.take(4 * RC);
  o.div_magic = L.take(8 * ((size_t)c->m_targ + 1));
  o.flux = L.take(8 * rec * R);
  o.totw = L.take(8 * rec * R);
  o.nw = L.take(4 * rec * R);
  o.events = L.take(8 * rec * R);
  o.hist = L.take(8 * rec * R * (c->hist_len > 0 ? c->hist_len : 1));
  o.near = L.take(4 * rec * R);
  o.pack = L.take(4 * (size_t)R * cap * n->S);
  if (c->reweight_period > 0) {
    const size_t nb = b->n_bins;
    o.rw_F = L.take(8 * R * nb * nb);
    o.rw_M = L.take(8 * R * nb * nb);
    o.rw_vec = L.take(8 * 4 * R * nb);
    o.rw_act = L.take(4 * R * nb);
    o.rw_iscr = L.take(24 * R * nb);
    o.rw_obs = L.take(4 * rec * R);
  }
  o.total = L.off;
  return o;
}

struct we_ensemble {
  we_run_config cfg{};
  int32_t S = 0, cap = 0, n_bins = 0;
  int32_t mapping = WE_MAP_THREAD, block = 128;
  int32_t resample_kernel = WE_RESAMPLE_AUTO, resample_blocks = 0;
  int32_t graph_kernels = 0;        // kernel nodes of the captured iteration graph
  void *ws = nullptr;
  bool owns_ws = false;
  Offsets off{};
  PropagateParams prm{};
  int32_t iters_enqueued = 0;       // iterations recorded so far (host view)
  bool phase_propagated = false;
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t timed_graph = nullptr, timed_graph2 = nullptr;   // two instances, alternated
  cudaGraph_t timed_graph_src = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  cudaGraphNode_t ev_node_start = nullptr, ev_node_end = nullptr;
  cudaStream_t cap_stream = nullptr;
};

static we_status check_config(const we_network *n, const we_binmap *b, const we_run_config *c, int *cap_out) {
  if (!n || !b || !c) return fail(WE_EINVAL, "network, bins and config are required");
  if (!(c->tau > 0.0) || std::isinf(c->tau)) return fail(WE_EINVAL, "tau must be finite and > 0");
  if (c->m_targ < 1) return fail(WE_EINVAL, "m_targ must be >= 1");
  if (c->n_runs < 1) return fail(WE_EINVAL, "n_runs must be >= 1");
  if (c->n_init < 1 || !c->init_states || !c->init_weights) return fail(WE_EINVAL, "need n_init >= 1 initial walkers with states and weights");
  if (c->record_iters < 1) return fail(WE_EINVAL, "record_iters must be >= 1");
  if (c->first_iter < 0) return fail(WE_EINVAL, "first_iter must be >= 0");
  for (int d = 0; d < b->ndim; ++d)
    if (b->species[d] >= n->S) return fail(WE_EINVAL, "bin dimension %d names species %d >= S", d, b->species[d]);
  if (b->learned && b->lb.n_in != n->S)
    return fail(WE_EINVAL, "learned bin map reads %d species, the network has %d", b->lb.n_in, n->S);
  if (b->learned && learned_bins_smem(b->lb.n_in, b->lb.H) > 227 * 1024)
    return fail(WE_ENOTSUPPORTED, "learned bin map: %d inputs x %d hidden do not fit the binning kernel's shared memory",
                b->lb.n_in, b->lb.H);
  long long cap = c->capacity > 0 ? c->capacity : std::max<long long>((long long)c->m_targ * b->n_bins, c->n_init);
  if (cap < c->n_init) return fail(WE_EINVAL, "capacity %lld < n_init %d", cap, c->n_init);
  if (cap * c->n_runs > (1ll << 30)) return fail(WE_EINVAL, "runs x capacity too large");
  if (c->feedback < 0 || c->feedback > WE_FEEDBACK_ENDPOINT)
    return fail(WE_EINVAL, "feedback must be 0, WE_FEEDBACK_RECYCLE, WE_FEEDBACK_ABSORB or WE_FEEDBACK_ENDPOINT");
  if (c->feedback == WE_FEEDBACK_ABSORB && c->resample)
    return fail(WE_EINVAL, "an absorbing target (brute-force runs) needs resample = 0");
  if (c->feedback) {
    if (c->n_clauses < 1 || c->n_clauses > kMaxClauses || !c->tgt_threshold) return fail(WE_EINVAL, "feedback needs 1..4 target clauses with thresholds");
    for (int k = 0; k < c->n_clauses; ++k) {
      if (c->tgt_species[k] < 0 || c->tgt_species[k] >= n->S) return fail(WE_EINVAL, "target clause %d: bad species", k);
      if (c->tgt_op[k] != WE_OP_GE && c->tgt_op[k] != WE_OP_LE) return fail(WE_EINVAL, "target clause %d: bad operator", k);
    }
  }
  if (c->hist_len < 0 || (c->hist_len > 0 && (c->hist_species < 0 || c->hist_species >= n->S)))
    return fail(WE_EINVAL, "bad histogram species/length");
  if (c->reweight_period < 0) return fail(WE_EINVAL, "reweight_period must be >= 0");
  if (c->n_init_per_run)
    for (int r = 0; r < c->n_runs; ++r)
      if (c->n_init_per_run[r] < 1 || c->n_init_per_run[r] > c->n_init)
        return fail(WE_EINVAL, "run %d: n_init_per_run must be 1..n_init", r);
  if (c->reweight_period > 0 && (!c->resample || b->n_bins > 1024))
    return fail(WE_EINVAL, "steady-state reweighting needs resample = 1 and at most 1024 bins");
  if (c->param_set)
    for (int r = 0; r < c->n_runs; ++r)
      if (c->param_set[r] < 0 || c->param_set[r] >= n->nps) return fail(WE_EINVAL, "run %d: parameter set out of range", r);
  for (long long i = 0; i < (long long)c->n_runs * c->n_init * n->S; ++i) {
    const int v = c->init_states[i];
    if (v < 0 || v > WE_MAX_COUNT) return fail(WE_EINVAL, "initial count %lld out of range", i);
  }
  for (long long i = 0; i < (long long)c->n_runs * c->n_init; ++i)
    if (!(c->init_weights[i] >= 0.0) || std::isinf(c->init_weights[i])) return fail(WE_EINVAL, "initial weight %lld must be finite and >= 0", i);
  *cap_out = (int)cap;
  return WE_OK;
}

extern "C" we_status we_ensemble_workspace_bytes(const we_network *n, const we_binmap *b,
                                                 const we_run_config *c, size_t *bytes) {
  if (!bytes) return fail(WE_EINVAL, "bytes is NULL");
  int cap = 0;
  we_status st = check_config(n, b, c, &cap);
  if (st) return st;
  *bytes = layout(n, b, c, cap).total;
  return WE_OK;
}

template <typename T>
static T *at(void *base, size_t off) { return reinterpret_cast<T *>(static_cast<char *>(base) + off); }




extern "C" we_status we_ensemble_create(const we_network *n, const we_binmap *b,
                                        const we_run_config *c, void *workspace,
                                        size_t workspace_bytes, void *stream, we_ensemble **out) {
  if (!out) return fail(WE_EINVAL, "out is NULL");
  *out = nullptr;
  int cap = 0;
  we_status st = check_config(n, b, c, &cap);
  if (st) return st;
  const int mapping = choose_mapping(n, c);
  const bool thread_map = mapping == WE_MAP_THREAD || mapping == WE_MAP_THREAD_TABLE;
  if (thread_map && (n->P > kThreadMaxLeaves || n->S > kThreadMaxSpecies))
    return fail(WE_ENOTSUPPORTED, "thread mapping needs <= %d reactions and <= %d species", kThreadMaxLeaves, kThreadMaxSpecies);
  if (mapping == WE_MAP_THREAD_TABLE && table_len_for(n) == 0)
    return fail(WE_ENOTSUPPORTED, "table mapping needs every propensity to read one species only");
  const int block = c->block_threads > 0 ? c->block_threads : (thread_map ? 128 : 32);
  if (thread_map && block != 32 && block != 64 && block != 96 && block != 128)
    return fail(WE_EINVAL, "thread mapping supports block_threads of 32, 64, 96 or 128");
  if (mapping == WE_MAP_WARP && 12ull * (n->P < 4 ? 4 : n->P) + 4ull * n->S + sizeof(LogTables) + 16 > 227ull * 1024)
    return fail(WE_ENOTSUPPORTED, "warp mapping keeps the walker's tree in shared memory: at most 16,384 reactions");
  Offsets o = layout(n, b, c, cap);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void *ws = workspace;
  bool owns = false;
  if (ws) {
    if (workspace_bytes < o.total) return fail(WE_ENOMEM, "workspace of %zu bytes < %zu needed", workspace_bytes, o.total);
    if (reinterpret_cast<uintptr_t>(ws) % 256) return fail(WE_EINVAL, "workspace must be 256-byte aligned");
  } else {
    cudaError_t e = device_alloc(&ws, o.total);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(WE_ENOMEM, "cudaMalloc(%zu): %s", o.total, cudaGetErrorString(e)); }
    owns = true;
  }
  we_ensemble *E = new (std::nothrow) we_ensemble();
  if (!E) { if (owns) cudaFree(ws); return fail(WE_ENOMEM, "host allocation"); }
  E->cfg = *c;
  E->cfg.capacity = cap;
  E->S = n->S; E->cap = cap; E->n_bins = b->n_bins;
  E->mapping = mapping; E->block = block;
  E->ws = ws; E->owns_ws = owns; E->off = o;
  auto cleanup = [&](we_status code) { if (owns) cudaFree(ws); delete E; return code; };

  const int R = c->n_runs, S = n->S;
  const size_t RC = (size_t)R * cap;
  // host images of everything uploaded
  std::vector<int32_t> run_id(R), pset(R), thr(R * (c->n_clauses > 0 ? c->n_clauses : 1), 0), rec((size_t)R * S);
  for (int r = 0; r < R; ++r) {
    run_id[r] = c->run_ids ? (int32_t)c->run_ids[r] : r;
    pset[r] = c->param_set ? c->param_set[r] : r % n->nps;
    for (int k = 0; k < c->n_clauses && c->feedback; ++k) thr[r * c->n_clauses + k] = c->tgt_threshold[r * c->n_clauses + k];
    for (int sp = 0; sp < S; ++sp)
      rec[(size_t)r * S + sp] = c->recycle_state ? c->recycle_state[(size_t)r * S + sp] : c->init_states[(size_t)r * c->n_init * S + sp];
  }
  if (c->feedback == WE_FEEDBACK_RECYCLE || c->feedback == WE_FEEDBACK_ENDPOINT)
    for (int r = 0; r < R; ++r) {
      bool in = true;
      for (int k = 0; k < c->n_clauses; ++k) {
        const int v = rec[(size_t)r * S + c->tgt_species[k]];
        in = in && (c->tgt_op[k] == WE_OP_GE ? v >= thr[r * c->n_clauses + k] : v <= thr[r * c->n_clauses + k]);
      }
      if (in) return cleanup(fail(WE_EINVAL, "run %d: the recycle state lies inside the target set", r));
    }
  const int par0 = c->first_iter & 1;
  std::vector<int32_t> xh((size_t)S * RC, 0), ph(RC, -1), cnt(R, c->n_init), roff(R + 1);
  std::vector<double> wh(RC, 0.0);
  if (c->n_init_per_run)
    for (int r = 0; r < R; ++r) cnt[r] = c->n_init_per_run[r];
  for (int r = 0; r < R; ++r)
    for (int w = 0; w < cnt[r]; ++w) {
      const size_t g = (size_t)r * cap + w;
      for (int sp = 0; sp < S; ++sp) xh[(size_t)sp * RC + g] = c->init_states[((size_t)r * c->n_init + w) * S + sp];
      wh[g] = c->init_weights[(size_t)r * c->n_init + w];
    }
  roff[0] = 0;
  for (int r = 0; r < R; ++r) roff[r + 1] = roff[r] + cnt[r];
  int32_t it0 = c->first_iter;
  auto up = [&](size_t offs, const void *src, size_t bytes) -> cudaError_t {
    if (!bytes) return cudaSuccess;
    return cudaMemcpyAsync(at<char>(ws, offs), src, bytes, cudaMemcpyHostToDevice, s);
  };
  std::vector<unsigned long long> magic((size_t)c->m_targ + 1, 0ull);   // lives past the copies
  for (int k = 2; k <= c->m_targ; ++k) magic[k] = ex_div_magic((unsigned)k);
  cudaError_t e = cudaSuccess;
  e = e ? e : cudaMemsetAsync(ws, 0, o.total, s);
  e = e ? e : up(o.div_magic, magic.data(), 8 * magic.size());
  e = e ? e : up(o.meta, n->meta.data(), sizeof(RxnMeta) * n->P);
  e = e ? e : up(o.keff, n->keff.data(), 8 * n->keff.size());
  e = e ? e : up(o.Kn, n->Kn.data(), 8 * n->Kn.size());
  e = e ? e : up(o.d_sp, n->d_sp.data(), 4 * n->d_sp.size());
  e = e ? e : up(o.d_val, n->d_val.data(), 4 * n->d_val.size());
  e = e ? e : up(o.dep_ptr, n->dep_ptr.data(), 4 * n->dep_ptr.size());
  e = e ? e : up(o.dep_idx, n->dep_idx.data(), 4 * n->dep_idx.size());
  WarpRecords wrec;                                                       // lives past the copies
  if (mapping == WE_MAP_WARP) {
    wrec = warp_records(n);
    if (wrec.stride != o.wrec_stride) return cleanup(fail(WE_EINVAL, "event record layout mismatch"));
    e = e ? e : up(o.wrec, wrec.words.data(), 4 * wrec.words.size());
  }
  e = e ? e : up(o.edges, b->edges.data(), 8 * b->edges.size());
  e = e ? e : up(o.run_id, run_id.data(), 4 * R);
  e = e ? e : up(o.param_set, pset.data(), 4 * R);
  e = e ? e : up(o.tgt_thr, thr.data(), 4 * thr.size());
  e = e ? e : up(o.recycle, rec.data(), 4 * rec.size());
  e = e ? e : up(par0 ? o.x1 : o.x0, xh.data(), 4 * xh.size());
  e = e ? e : up(par0 ? o.w1 : o.w0, wh.data(), 8 * wh.size());
  e = e ? e : up(par0 ? o.p1 : o.p0, ph.data(), 4 * ph.size());
  e = e ? e : up(o.count, cnt.data(), 4 * R);
  e = e ? e : up(o.prev_count, cnt.data(), 4 * R);
  e = e ? e : up(o.run_off, roff.data(), 4 * (R + 1));
  e = e ? e : up(o.iter, &it0, 4);
  std::vector<double> fpt0(c->feedback == WE_FEEDBACK_ABSORB ? RC : 0, -1.0);   // no first passage yet
  e = e ? e : up(o.fpt, fpt0.data(), 8 * fpt0.size());
  std::vector<int32_t> base(S, 0);
  for (int sp = 0; sp < S; ++sp) base[sp] = n->fixed[sp] >= 0 ? n->fixed[sp] : 0;
  e = e ? e : up(o.base, base.data(), 4 * S);
  if (b->learned) {
    const we_learned_bins &lb = b->lb;
    std::vector<float> bias(lb.b1);
    bias.insert(bias.end(), lb.b2.begin(), lb.b2.end());
    bias.push_back(lb.b3[0]);
    e = e ? e : up(o.lw1, lb.w1.data(), 2 * lb.w1.size());
    e = e ? e : up(o.lw2, lb.w2.data(), 2 * lb.w2.size());
    e = e ? e : up(o.lw3, lb.w3.data(), 2 * lb.w3.size());
    e = e ? e : up(o.lb, bias.data(), 4 * bias.size());
    e = e ? e : up(o.lz, lb.zedges.data(), 4 * lb.zedges.size());
  }
  e = e ? e : launch_init_log_tables(at<LogTables>(ws, o.logt), s);
  e = e ? e : resample_run_prepare();
  if (e) { cudaGetLastError(); return cleanup(cuda_fail(e, "ensemble upload")); }

  NetView &N = E->prm.net;
  N.S = S; N.M = n->M; N.P = n->P; N.log2P = n->log2P; N.n_param_sets = n->nps;
  N.n_delta = (int32_t)n->d_sp.size();
  N.meta = at<RxnMeta>(ws, o.meta);
  N.keff = at<double>(ws, o.keff);
  N.hill_Kn = at<double>(ws, o.Kn);
  N.d_sp = at<int32_t>(ws, o.d_sp);
  N.d_val = at<int32_t>(ws, o.d_val);
  N.dep_ptr = at<int32_t>(ws, o.dep_ptr);
  N.dep_idx = at<int32_t>(ws, o.dep_idx);
  if (mapping == WE_MAP_WARP) {
    N.wrec = at<int4>(ws, o.wrec);
    N.wrec_stride = wrec.stride; N.wrec_chg = wrec.chg; N.wrec_dep = wrec.dep;
  }
  BinView &Bv = E->prm.bins;
  Bv.ndim = b->ndim; Bv.n_bins = b->n_bins;
  for (int d = 0; d < kMaxBinDims; ++d) {
    Bv.species[d] = b->species[d]; Bv.nb[d] = b->nb[d]; Bv.edge_off[d] = b->edge_off[d];
    Bv.ufirst[d] = 0; Bv.ustep[d] = 0;
    if (d < b->ndim) uniform_inner_edges(b->edges.data() + b->edge_off[d], b->nb[d], &Bv.ufirst[d], &Bv.ustep[d]);
  }
  Bv.edges = at<double>(ws, o.edges);
  Bv.learned = b->learned ? 1 : 0;
  if (b->learned) {
    Bv.mlp.n_in = b->lb.n_in;
    Bv.mlp.hidden = b->lb.H;
    Bv.mlp.w1 = at<uint16_t>(ws, o.lw1);
    Bv.mlp.w2 = at<uint16_t>(ws, o.lw2);
    Bv.mlp.w3 = at<uint16_t>(ws, o.lw3);
    Bv.mlp.b1 = at<float>(ws, o.lb);
    Bv.mlp.b2 = at<float>(ws, o.lb) + b->lb.H;
    Bv.mlp.b3 = at<float>(ws, o.lb) + 2 * b->lb.H;
    Bv.zedges = at<float>(ws, o.lz);
    Bv.zout = at<float>(ws, o.zout);
  }
  EnsView &V = E->prm.ens;
  V.R = R; V.cap = cap; V.S = S; V.m_targ = c->m_targ; V.record_iters = c->record_iters;
  V.first_iter = c->first_iter; V.hist_species = c->hist_species; V.hist_len = c->hist_len;
  // the kernels see the end-of-interval check as no feedback inside the interval
  V.feedback = c->feedback == WE_FEEDBACK_ENDPOINT ? 0 : c->feedback;
  V.end_check = c->feedback == WE_FEEDBACK_ENDPOINT ? 1 : 0;
  V.n_clauses = c->feedback ? c->n_clauses : 0;
  for (int k = 0; k < kMaxClauses; ++k) { V.tgt_species[k] = c->tgt_species[k]; V.tgt_op[k] = c->tgt_op[k]; }
  V.max_steps = c->max_steps > 0 ? c->max_steps : WE_DEFAULT_MAX_STEPS;
  V.tau = c->tau; V.seed = c->seed;
  V.run_id = at<uint32_t>(ws, o.run_id);
  V.param_set = at<int32_t>(ws, o.param_set);
  V.tgt_thr = at<int32_t>(ws, o.tgt_thr);
  V.recycle = at<int32_t>(ws, o.recycle);
  V.x[0] = at<int32_t>(ws, o.x0); V.x[1] = at<int32_t>(ws, o.x1);
  V.w[0] = at<double>(ws, o.w0); V.w[1] = at<double>(ws, o.w1);
  V.parent[0] = at<int32_t>(ws, o.p0); V.parent[1] = at<int32_t>(ws, o.p1);
  V.bin = at<int32_t>(ws, o.bin); V.nrec = at<int32_t>(ws, o.nrec); V.tlast = at<double>(ws, o.tlast);
  V.fpt = c->feedback == WE_FEEDBACK_ABSORB ? at<double>(ws, o.fpt) : nullptr;
  V.count = at<int32_t>(ws, o.count); V.prev_count = at<int32_t>(ws, o.prev_count);
  V.run_off = at<int32_t>(ws, o.run_off);
  V.status = at<int32_t>(ws, o.status); V.iter = at<int32_t>(ws, o.iter);
  V.bin_count = at<int32_t>(ws, o.bin_count); V.n_tasks = at<int32_t>(ws, o.n_tasks);
  V.tasks = at<int4>(ws, o.tasks); V.cursor = at<int32_t>(ws, o.cursor);
  V.sorted_slot = at<int32_t>(ws, o.sorted_slot);
  V.sorted_w = at<double>(ws, o.sorted_w); V.alive = at<int32_t>(ws, o.alive);
  V.div_magic = at<unsigned long long>(ws, o.div_magic);
  V.obs_flux = at<double>(ws, o.flux); V.obs_totw = at<double>(ws, o.totw);
  V.obs_nw = at<int32_t>(ws, o.nw); V.obs_events = at<unsigned long long>(ws, o.events);
  V.obs_hist = at<double>(ws, o.hist);
  V.obs_near = at<int32_t>(ws, o.near);
  E->prm.resample = c->resample ? 1 : 0;
  E->prm.logt = at<LogTables>(ws, o.logt);
  if (c->reweight_period > 0) {
    RwView &rw = E->prm.rw;
    const size_t nbR = (size_t)b->n_bins * R;
    rw.period = c->reweight_period;
    rw.nb = b->n_bins;
    rw.F = at<double>(ws, o.rw_F);
    rw.M = at<double>(ws, o.rw_M);
    rw.W = at<double>(ws, o.rw_vec);
    rw.cb = rw.W + nbR; rw.x = rw.cb + nbR; rw.fac = rw.x + nbR;
    rw.act = at<int32_t>(ws, o.rw_act);
    rw.iscr = at<int32_t>(ws, o.rw_iscr);
    rw.obs = at<int32_t>(ws, o.rw_obs);
  }
  E->prm.tab.species = -1;
  E->prm.tab.species2 = -1;
  E->prm.tab.lenB = 1;
  E->prm.tab.smem_rows = 0;
  if (mapping == WE_MAP_THREAD_TABLE) {
    E->prm.tab.rows = at<unsigned long long>(ws, o.table);
    E->prm.tab.len = o.table_len;
    E->prm.tab.lenB = o.table_lenB;
    E->prm.tab.species = n->table_species;
    E->prm.tab.species2 = n->table_species2;
    E->prm.tab.clock_scale = std::ldexp(1.0 / c->tau, kClockBits);   // 2^62 / tau
    e = launch_build_table(N, at<int32_t>(ws, o.base), n->table_species, n->table_species2,
                           o.table_len, o.table_lenB,
                           E->prm.tab.clock_scale, at<unsigned long long>(ws, o.table), s);
  }
  e = e ? e : cudaStreamSynchronize(s);
  if (e) { cudaGetLastError(); return cleanup(cuda_fail(e, "ensemble set-up")); }
  *out = E;
  return WE_OK;
}

extern "C" we_status we_ensemble_destroy(we_ensemble *E) {
  if (!E) return WE_OK;
  if (E->graph) cudaGraphExecDestroy(E->graph);
  if (E->timed_graph) cudaGraphExecDestroy(E->timed_graph);
  if (E->timed_graph2) cudaGraphExecDestroy(E->timed_graph2);
  if (E->timed_graph_src) cudaGraphDestroy(E->timed_graph_src);
  if (E->ev_a) cudaEventDestroy(E->ev_a);
  if (E->ev_b) cudaEventDestroy(E->ev_b);
  if (E->cap_stream) cudaStreamDestroy(E->cap_stream);
  if (E->owns_ws) cudaFree(E->ws);
  delete E;
  return WE_OK;
}

// Thread mappings: 128-thread blocks run the warp-specialised kernel (one event warp and three
// draw warps per 32 walkers); 32/64/96-thread blocks run the plain kernel in which each thread
// makes its own draws.
static cudaError_t enqueue_ssa(we_ensemble *E, cudaStream_t s) {
  if (E->mapping == WE_MAP_WARP) return launch_propagate_warp(E->prm, E->block, s);
  const bool table = E->mapping == WE_MAP_THREAD_TABLE;
  if (E->block == 128) return launch_propagate_ws(E->prm, table, s);
  return launch_propagate_thread(E->prm, E->block, table, s);
}

static cudaError_t enqueue_propagate(we_ensemble *E, cudaStream_t s) {
  cudaError_t e = enqueue_ssa(E, s);
  if (!e && E->prm.bins.learned) e = launch_learned_bins(E->prm, s);
  return e;
}

// Grids of up to this many bins whose runs fit in shared memory take the one-launch split/merge.
constexpr int kOneLaunchAutoMaxBins = 256;

static bool resample_in_one_launch(const we_ensemble *E) {
  if (E->resample_kernel == WE_RESAMPLE_CHAIN) return false;
  if (!resample_run_smem(E->prm.ens, E->n_bins)) return false;
  return E->resample_kernel == WE_RESAMPLE_ONE_LAUNCH || E->n_bins <= kOneLaunchAutoMaxBins;
}

static cudaError_t enqueue_resample(we_ensemble *E, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const bool rw = E->prm.resample && E->prm.rw.period > 0;
  if (rw) e = launch_rw_flux(E->prm, s);           // before the split/merge replaces its tasks
  if (!e && E->prm.resample)
    e = resample_in_one_launch(E) ? launch_resample_run(E->prm, E->resample_blocks, s)
                                  : launch_resample_chain(E->prm, s);
  if (!e) e = launch_gather_finalize(E->prm, s);
  if (!e && rw) e = launch_rw_solve_apply(E->prm, s);
  return e;
}

extern "C" we_status we_ensemble_propagate(we_ensemble *E, void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  if (E->phase_propagated) return fail(WE_EINVAL, "propagate called twice without resample");
  if (E->iters_enqueued >= E->cfg.record_iters) return fail(WE_EOVERFLOW, "record_iters (%d) exhausted", E->cfg.record_iters);
  cudaError_t e = enqueue_propagate(E, static_cast<cudaStream_t>(stream));
  if (e) return cuda_fail(e, "propagate launch");
  E->phase_propagated = true;
  return WE_OK;
}

extern "C" we_status we_ensemble_resample(we_ensemble *E, void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  if (!E->phase_propagated) return fail(WE_EINVAL, "resample called before propagate");
  cudaError_t e = enqueue_resample(E, static_cast<cudaStream_t>(stream));
  if (e) return cuda_fail(e, "resample launch");
  E->phase_propagated = false;
  E->iters_enqueued += 1;
  return WE_OK;
}

static void drop_graphs(we_ensemble *E) {
  if (E->graph) cudaGraphExecDestroy(E->graph);
  if (E->timed_graph) cudaGraphExecDestroy(E->timed_graph);
  if (E->timed_graph2) cudaGraphExecDestroy(E->timed_graph2);
  if (E->timed_graph_src) cudaGraphDestroy(E->timed_graph_src);
  E->graph = E->timed_graph = E->timed_graph2 = nullptr;
  E->timed_graph_src = nullptr;
  E->ev_node_start = E->ev_node_end = nullptr;
}

extern "C" we_status we_ensemble_set_resample_kernel(we_ensemble *E, int32_t kind, int32_t blocks_per_run) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  if (kind < WE_RESAMPLE_AUTO || kind > WE_RESAMPLE_ONE_LAUNCH) return fail(WE_EINVAL, "unknown resample kernel %d", kind);
  if (blocks_per_run < 0 || blocks_per_run > 32) return fail(WE_EINVAL, "blocks_per_run must be 0..32");
  if (kind == WE_RESAMPLE_ONE_LAUNCH && !resample_run_smem(E->prm.ens, E->n_bins))
    return fail(WE_EINVAL, "the one-launch split/merge needs the runs' walker lists in shared memory "
                           "(24 n_bins + 16 capacity bytes) and at most 8 species");
  if (E->phase_propagated) return fail(WE_EINVAL, "set the resample kernel between iterations");
  WE_CUDA_TRY(cudaDeviceSynchronize());                  // no replay of the old graphs in flight
  drop_graphs(E);
  E->resample_kernel = kind;
  E->resample_blocks = blocks_per_run;
  return WE_OK;
}

// The iteration graph (propagate + resample), captured once per ensemble.
static we_status build_graph(we_ensemble *E) {
  if (!E->cap_stream) WE_CUDA_TRY(cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking));
  WE_CUDA_TRY(cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t e1 = enqueue_propagate(E, E->cap_stream);
  cudaError_t e2 = e1 ? e1 : enqueue_resample(E, E->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e3 = cudaStreamEndCapture(E->cap_stream, &g);
  if (e2 || e3) { if (g) cudaGraphDestroy(g); cudaGetLastError(); return cuda_fail(e2 ? e2 : e3, "graph capture"); }
  size_t n_nodes = 0;
  cudaError_t e4 = cudaGraphGetNodes(g, nullptr, &n_nodes);
  std::vector<cudaGraphNode_t> nodes(n_nodes);
  if (!e4 && n_nodes) e4 = cudaGraphGetNodes(g, nodes.data(), &n_nodes);
  int32_t n_kernels = 0;
  for (size_t i = 0; !e4 && i < n_nodes; ++i) {
    cudaGraphNodeType t;
    e4 = cudaGraphNodeGetType(nodes[i], &t);
    if (!e4 && t == cudaGraphNodeTypeKernel) ++n_kernels;
  }
  if (!e4) e4 = cudaGraphInstantiate(&E->graph, g, 0);
  cudaGraphDestroy(g);
  if (e4) { E->graph = nullptr; return cuda_fail(e4, "graph instantiate"); }
  E->graph_kernels = n_kernels;
  return WE_OK;
}

extern "C" we_status we_ensemble_iteration_kernels(we_ensemble *E, int32_t *n_kernels) {
  if (!E || !n_kernels) return fail(WE_EINVAL, "ensemble and n_kernels are required");
  if (E->phase_propagated) return fail(WE_EINVAL, "a propagate without its resample is pending");
  if (!E->graph) {
    we_status st = build_graph(E);
    if (st) return st;
  }
  *n_kernels = E->graph_kernels;
  return WE_OK;
}

extern "C" we_status we_ensemble_step(we_ensemble *E, int32_t n_iters, void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  if (n_iters < 0) return fail(WE_EINVAL, "n_iters must be >= 0");
  if (E->phase_propagated) return fail(WE_EINVAL, "step called between propagate and resample");
  if (E->iters_enqueued + n_iters > E->cfg.record_iters)
    return fail(WE_EOVERFLOW, "%d more iterations would exceed record_iters (%d)", n_iters, E->cfg.record_iters);
  if (n_iters == 0) return WE_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!E->graph) {
    we_status st = build_graph(E);
    if (st) return st;
  }
  for (int i = 0; i < n_iters; ++i) WE_CUDA_TRY(cudaGraphLaunch(E->graph, s));
  E->iters_enqueued += n_iters;
  return WE_OK;
}

// Events for timed replays, per device: grown on demand, kept for the life of the process.
// Calls that overlap in time on one device must not share them; timed replays of different
// ensembles are meant to run one after another (they synchronise before returning).
static std::mutex g_ev_mu;
static std::vector<cudaEvent_t> g_ev_pool[256];

static we_status timing_events(size_t n, cudaEvent_t **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) { cudaGetLastError(); return fail(WE_ECUDA, "current device"); }
  std::lock_guard<std::mutex> lk(g_ev_mu);
  std::vector<cudaEvent_t> &pool = g_ev_pool[dev];
  while (pool.size() < n) {
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return fail(WE_ECUDA, "event creation"); }
    pool.push_back(e);
  }
  *out = pool.data();
  return WE_OK;
}

// Timed replay: the same iteration graph, captured with an event-record node on each side of
// the SSA kernel; before every replay the two nodes are pointed at that iteration's events.
static we_status build_timed_graph(we_ensemble *E) {
  if (!E->cap_stream) WE_CUDA_TRY(cudaStreamCreateWithFlags(&E->cap_stream, cudaStreamNonBlocking));
  // the placeholder events stay alive with the graph: its event-record nodes refer to them
  if (!E->ev_a) WE_CUDA_TRY(cudaEventCreate(&E->ev_a));
  if (!E->ev_b) WE_CUDA_TRY(cudaEventCreate(&E->ev_b));
  cudaEvent_t ea = E->ev_a, eb = E->ev_b;
  WE_CUDA_TRY(cudaStreamBeginCapture(E->cap_stream, cudaStreamCaptureModeThreadLocal));
  // External records become event-record nodes of the graph (a plain record inside a capture
  // only orders streams).
  cudaError_t e1 = cudaEventRecordWithFlags(ea, E->cap_stream, cudaEventRecordExternal);
  e1 = e1 ? e1 : enqueue_propagate(E, E->cap_stream);
  e1 = e1 ? e1 : cudaEventRecordWithFlags(eb, E->cap_stream, cudaEventRecordExternal);
  e1 = e1 ? e1 : enqueue_resample(E, E->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(E->cap_stream, &g);
  if (e1 || e2) { if (g) cudaGraphDestroy(g); cudaGetLastError(); return cuda_fail(e1 ? e1 : e2, "timed graph capture"); }
  size_t n = 0;
  cudaGraphGetNodes(g, nullptr, &n);
  std::vector<cudaGraphNode_t> nodes(n);
  cudaGraphGetNodes(g, nodes.data(), &n);
  for (auto nd : nodes) {
    cudaGraphNodeType t;
    cudaGraphNodeGetType(nd, &t);
    if (t != cudaGraphNodeTypeEventRecord) continue;
    size_t nd_deps = 0;
    cudaGraphNodeGetDependencies(nd, nullptr, nullptr, &nd_deps);
    if (nd_deps == 0) E->ev_node_start = nd; else E->ev_node_end = nd;
  }
  if (!E->ev_node_start || !E->ev_node_end) {
    cudaGraphDestroy(g);
    return fail(WE_ECUDA, "timed graph: event-record nodes not found in the capture");
  }
  // two executable instances, launched alternately: retargeting the event nodes of one while
  // the other runs keeps the host from waiting on the launch in flight
  cudaError_t e3 = cudaGraphInstantiate(&E->timed_graph, g, 0);
  e3 = e3 ? e3 : cudaGraphInstantiate(&E->timed_graph2, g, 0);
  if (e3) {
    if (E->timed_graph) cudaGraphExecDestroy(E->timed_graph);
    cudaGraphDestroy(g);
    E->timed_graph = E->timed_graph2 = nullptr;
    return cuda_fail(e3, "timed graph instantiate");
  }
  // the event-record node handles used to retarget the executable graph belong to this graph,
  // so it lives as long as the ensemble
  E->timed_graph_src = g;
  return WE_OK;
}

extern "C" we_status we_ensemble_step_timed_every(we_ensemble *E, int32_t n_iters, int32_t every, void *stream,
                                                 float *propagate_ms) {
  if (!E || !propagate_ms) return fail(WE_EINVAL, "ensemble and propagate_ms are required");
  if (n_iters < 0) return fail(WE_EINVAL, "n_iters must be >= 0");
  if (every < 1) return fail(WE_EINVAL, "every must be >= 1");
  if (E->phase_propagated) return fail(WE_EINVAL, "step called between propagate and resample");
  if (E->iters_enqueued + n_iters > E->cfg.record_iters)
    return fail(WE_EOVERFLOW, "%d more iterations would exceed record_iters (%d)", n_iters, E->cfg.record_iters);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (!E->timed_graph) {                                 // n_iters = 0: capture only
    we_status st = build_timed_graph(E);
    if (st) return st;
  }
  if (every > 1 && !E->graph) {
    we_status st = build_graph(E);
    if (st) return st;
  }
  if (n_iters == 0) return WE_OK;
  const int n_timed = (n_iters + every - 1) / every;
  // per-iteration events from a process-wide pool (per device), created once and reused, so
  // that no event is created or destroyed between the launches being timed
  cudaEvent_t *ev = nullptr;
  {
    we_status st = timing_events(2 * (size_t)n_timed, &ev);
    if (st) return st;
  }
  for (int i = 0; i < n_iters; ++i) {
    cudaError_t e;
    if (i % every == 0) {
      const int k = i / every;
      cudaGraphExec_t gx = (k & 1) ? E->timed_graph2 : E->timed_graph;
      e = cudaGraphExecEventRecordNodeSetEvent(gx, E->ev_node_start, ev[2 * k]);
      e = e ? e : cudaGraphExecEventRecordNodeSetEvent(gx, E->ev_node_end, ev[2 * k + 1]);
      e = e ? e : cudaGraphLaunch(gx, s);
    } else {
      e = cudaGraphLaunch(E->graph, s);
    }
    if (e) { cudaGetLastError(); return cuda_fail(e, "timed graph launch"); }
  }
  E->iters_enqueued += n_iters;
  cudaError_t e = cudaStreamSynchronize(s);
  for (int k = 0; k < n_timed && !e; ++k) e = cudaEventElapsedTime(&propagate_ms[k], ev[2 * k], ev[2 * k + 1]);
  // point the nodes back at the ensemble's own events
  for (cudaGraphExec_t gx : {E->timed_graph, E->timed_graph2}) {
    cudaGraphExecEventRecordNodeSetEvent(gx, E->ev_node_start, E->ev_a);
    cudaGraphExecEventRecordNodeSetEvent(gx, E->ev_node_end, E->ev_b);
  }
  if (e) return cuda_fail(e, "event timing");
  return WE_OK;
}

extern "C" we_status we_ensemble_step_timed(we_ensemble *E, int32_t n_iters, void *stream, float *propagate_ms) {
  return we_ensemble_step_timed_every(E, n_iters, 1, stream, propagate_ms);
}

extern "C" we_status we_ensemble_sync(we_ensemble *E, void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WE_CUDA_TRY(cudaStreamSynchronize(s));
  std::vector<int32_t> st(E->cfg.n_runs);
  WE_CUDA_TRY(cudaMemcpy(st.data(), E->prm.ens.status, 4 * st.size(), cudaMemcpyDeviceToHost));
  for (int r = 0; r < E->cfg.n_runs; ++r)
    if (st[r]) return fail(st[r], "run %d reported %s on the device", r, we_status_string(st[r]));
  return WE_OK;
}

// ------------------------------------------------------------------------------------------
// checkpoint / resume
// ------------------------------------------------------------------------------------------
// Byte layout: int32 header[8] = {magic, version, runs, species, next iteration, bins of the
// reweighting data (0: none), m_targ, 0}; int32 counts[runs]; per run: int32 states[count x S]
// (walker-major) then double weights[count]; with reweighting data: int32 n_tasks[runs],
// int4 tasks[runs x bins], double transfers[runs x bins x bins].
constexpr int32_t kCkptMagic = 0x31434557;   // "WEC1"
constexpr int32_t kCkptVersion = 1;

extern "C" we_status we_ensemble_checkpoint(we_ensemble *E, void *dst, size_t dst_bytes, size_t *needed,
                                            void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  if (E->phase_propagated) return fail(WE_EINVAL, "checkpoint called between propagate and resample");
  if (E->cfg.feedback == WE_FEEDBACK_ABSORB)
    return fail(WE_ENOTSUPPORTED, "checkpoints do not carry the first-passage times of an absorbing ensemble");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  WE_CUDA_TRY(cudaStreamSynchronize(s));
  const int R = E->cfg.n_runs, S = E->S;
  const EnsView &V = E->prm.ens;
  const RwView &rw = E->prm.rw;
  std::vector<int32_t> cnt(R);
  int32_t iter = 0;
  WE_CUDA_TRY(cudaMemcpy(cnt.data(), V.count, 4 * (size_t)R, cudaMemcpyDeviceToHost));
  WE_CUDA_TRY(cudaMemcpy(&iter, V.iter, 4, cudaMemcpyDeviceToHost));
  const int nb = rw.period > 0 ? rw.nb : 0;
  size_t bytes = 32 + 4 * (size_t)R;
  for (int r = 0; r < R; ++r) bytes += (size_t)cnt[r] * (4 * (size_t)S + 8);
  if (nb) bytes += 4 * (size_t)R + 16 * (size_t)R * nb + 8 * (size_t)R * nb * nb;
  if (needed) *needed = bytes;
  if (!dst) return WE_OK;
  if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small (%zu < %zu)", dst_bytes, bytes);
  char *o = static_cast<char *>(dst);
  const int32_t hdr[8] = {kCkptMagic, kCkptVersion, R, S, iter, nb, E->cfg.m_targ, 0};
  std::memcpy(o, hdr, 32); o += 32;
  std::memcpy(o, cnt.data(), 4 * (size_t)R); o += 4 * (size_t)R;
  for (int r = 0; r < R; ++r) {
    const size_t ns = (size_t)cnt[r] * S * 4, nw = (size_t)cnt[r] * 8;
    size_t got = 0;
    we_status st = we_ensemble_get(E, WE_OUT_STATES, r, o, ns, &got, stream);
    if (st) return st;
    o += ns;
    st = we_ensemble_get(E, WE_OUT_WEIGHTS, r, o, nw, &got, stream);
    if (st) return st;
    o += nw;
  }
  if (nb) {
    WE_CUDA_TRY(cudaMemcpy(o, V.n_tasks, 4 * (size_t)R, cudaMemcpyDeviceToHost)); o += 4 * (size_t)R;
    WE_CUDA_TRY(cudaMemcpy(o, V.tasks, 16 * (size_t)R * nb, cudaMemcpyDeviceToHost)); o += 16 * (size_t)R * nb;
    WE_CUDA_TRY(cudaMemcpy(o, rw.F, 8 * (size_t)R * nb * nb, cudaMemcpyDeviceToHost)); o += 8 * (size_t)R * nb * nb;
  }
  return WE_OK;
}

extern "C" we_status we_ensemble_resume(const we_network *n, const we_binmap *b, const we_run_config *c,
                                        const void *ckpt, size_t bytes, void *stream, we_ensemble **out) {
  if (!out) return fail(WE_EINVAL, "out is NULL");
  *out = nullptr;
  if (!n || !b || !c || !ckpt) return fail(WE_EINVAL, "network, bins, config and checkpoint are required");
  const char *p = static_cast<const char *>(ckpt);
  if (bytes < 32) return fail(WE_EINVAL, "checkpoint too short");
  int32_t hdr[8];
  std::memcpy(hdr, p, 32);
  const int R = hdr[2], S = hdr[3], nb = hdr[5];
  if (hdr[0] != kCkptMagic || hdr[1] != kCkptVersion) return fail(WE_EINVAL, "not a checkpoint of this version");
  if (R != c->n_runs || S != n->S) return fail(WE_EINVAL, "checkpoint has %d runs x %d species, expected %d x %d", R, S, c->n_runs, n->S);
  if (hdr[4] < 0 || hdr[6] < 1) return fail(WE_EINVAL, "checkpoint header is inconsistent");
  const bool rw_cfg = c->reweight_period > 0;
  if (nb != 0 && (!rw_cfg || nb != b->n_bins)) return fail(WE_EINVAL, "checkpoint's reweighting data does not match the configuration");
  size_t need = 32 + 4 * (size_t)R;
  if (bytes < need) return fail(WE_EINVAL, "checkpoint too short");
  std::vector<int32_t> cnt(R);
  std::memcpy(cnt.data(), p + 32, 4 * (size_t)R);
  int mx = 1;
  for (int r = 0; r < R; ++r) {
    if (cnt[r] < 1) return fail(WE_EINVAL, "checkpoint run %d has no walkers", r);
    mx = std::max(mx, cnt[r]);
    need += (size_t)cnt[r] * (4 * (size_t)S + 8);
  }
  if (nb) need += 4 * (size_t)R + 16 * (size_t)R * nb + 8 * (size_t)R * nb * nb;
  if (bytes < need) return fail(WE_EINVAL, "checkpoint too short (%zu < %zu)", bytes, need);
  std::vector<int32_t> xs((size_t)R * mx * S, 0);
  std::vector<double> ws((size_t)R * mx, 0.0);
  const char *q = p + 32 + 4 * (size_t)R;
  for (int r = 0; r < R; ++r) {
    std::memcpy(xs.data() + (size_t)r * mx * S, q, (size_t)cnt[r] * S * 4); q += (size_t)cnt[r] * S * 4;
    std::memcpy(ws.data() + (size_t)r * mx, q, (size_t)cnt[r] * 8); q += (size_t)cnt[r] * 8;
  }
  we_run_config c2 = *c;
  c2.n_init = mx;
  c2.init_states = xs.data();
  c2.init_weights = ws.data();
  c2.n_init_per_run = cnt.data();
  c2.first_iter = hdr[4];
  we_ensemble *E = nullptr;
  we_status st = we_ensemble_create(n, b, &c2, nullptr, 0, stream, &E);
  if (st) return st;
  E->cfg.n_init_per_run = nullptr;       // the host arrays above do not outlive this call
  E->cfg.init_states = nullptr;
  E->cfg.init_weights = nullptr;
  if (nb) {
    const EnsView &V = E->prm.ens;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaMemcpyAsync(V.n_tasks, q, 4 * (size_t)R, cudaMemcpyHostToDevice, s); q += 4 * (size_t)R;
    e = e ? e : cudaMemcpyAsync(V.tasks, q, 16 * (size_t)R * nb, cudaMemcpyHostToDevice, s); q += 16 * (size_t)R * nb;
    e = e ? e : cudaMemcpyAsync(E->prm.rw.F, q, 8 * (size_t)R * nb * nb, cudaMemcpyHostToDevice, s);
    e = e ? e : cudaStreamSynchronize(s);
    if (e) { cudaGetLastError(); we_ensemble_destroy(E); return cuda_fail(e, "checkpoint upload"); }
    E->prm.rw.start_known = 1;
  }
  *out = E;
  return WE_OK;
}

extern "C" we_status we_ensemble_get(we_ensemble *E, int32_t what, int32_t run, void *dst,
                                     size_t dst_bytes, size_t *needed, void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const EnsView &V = E->prm.ens;
  const int R = E->cfg.n_runs;
  if (run < -1 || run >= R) return fail(WE_EINVAL, "run %d out of range", run);
  WE_CUDA_TRY(cudaStreamSynchronize(s));
  int32_t iter = 0;
  WE_CUDA_TRY(cudaMemcpy(&iter, V.iter, 4, cudaMemcpyDeviceToHost));
  const int rec = std::min(E->iters_enqueued, E->cfg.record_iters);
  const int par = iter & 1;
  std::vector<int32_t> counts(R);
  WE_CUDA_TRY(cudaMemcpy(counts.data(), V.count, 4 * R, cudaMemcpyDeviceToHost));
  auto per_walker = [&](const void *base, size_t elem) -> we_status {
    if (run < 0) return fail(WE_EINVAL, "walker arrays need a single run");
    const size_t bytes = elem * counts[run];
    if (needed) *needed = bytes;
    if (!dst) return WE_OK;
    if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small (%zu < %zu)", dst_bytes, bytes);
    if (bytes) WE_CUDA_TRY(cudaMemcpy(dst, static_cast<const char *>(base) + elem * (size_t)run * E->cap, bytes, cudaMemcpyDefault));
    return WE_OK;
  };
  auto per_iter = [&](const void *base, size_t elem_per_run) -> we_status {
    const size_t rows = rec;
    const size_t bytes = run < 0 ? rows * R * elem_per_run : rows * elem_per_run;
    if (needed) *needed = bytes;
    if (!dst) return WE_OK;
    if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small (%zu < %zu)", dst_bytes, bytes);
    if (!bytes) return WE_OK;
    if (run < 0) WE_CUDA_TRY(cudaMemcpy(dst, base, bytes, cudaMemcpyDefault));
    else WE_CUDA_TRY(cudaMemcpy2D(dst, elem_per_run, static_cast<const char *>(base) + (size_t)run * elem_per_run,
                                  (size_t)R * elem_per_run, elem_per_run, rows, cudaMemcpyDefault));
    return WE_OK;
  };
  auto scalar = [&](const void *src, size_t bytes) -> we_status {
    if (needed) *needed = bytes;
    if (!dst) return WE_OK;
    if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small");
    WE_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
    return WE_OK;
  };
  switch (what) {
    case WE_OUT_COUNTS: {
      if (run >= 0) return scalar(&counts[run], 4);
      return scalar(counts.data(), 4 * R);
    }
    case WE_OUT_STATES: {
      size_t live = 0;
      if (run < 0) for (int r = 0; r < R; ++r) live += (size_t)counts[r];
      else live = (size_t)counts[run];
      const size_t bytes = (size_t)4 * live * E->S;
      if (needed) *needed = bytes;
      if (!dst) return WE_OK;
      if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small (%zu < %zu)", dst_bytes, bytes);
      if (!bytes) return WE_OK;
      int32_t *pack = at<int32_t>(E->ws, E->off.pack);
      cudaError_t e = launch_pack_states(V, run, pack, s);
      if (e) return cuda_fail(e, "pack states");
      WE_CUDA_TRY(cudaStreamSynchronize(s));
      WE_CUDA_TRY(cudaMemcpy(dst, pack, bytes, cudaMemcpyDefault));
      return WE_OK;
    }
    case WE_OUT_WEIGHTS: return per_walker(V.w[par], 8);
    case WE_OUT_PARENT: return per_walker(V.parent[par], 4);
    case WE_OUT_FLUX: return per_iter(V.obs_flux, 8);
    case WE_OUT_TOTAL_W: return per_iter(V.obs_totw, 8);
    case WE_OUT_NWALKERS: return per_iter(V.obs_nw, 4);
    case WE_OUT_EVENTS: return per_iter(V.obs_events, 8);
    case WE_OUT_HIST: return per_iter(V.obs_hist, 8 * (size_t)(E->cfg.hist_len > 0 ? E->cfg.hist_len : 1));
    case WE_OUT_STATUS: {
      std::vector<int32_t> st(R);
      WE_CUDA_TRY(cudaMemcpy(st.data(), V.status, 4 * R, cudaMemcpyDeviceToHost));
      if (run >= 0) return scalar(&st[run], 4);
      return scalar(st.data(), 4 * R);
    }
    case WE_OUT_TLAST: {
      if (run < 0) return fail(WE_EINVAL, "walker arrays need a single run");
      int32_t pc = 0;
      WE_CUDA_TRY(cudaMemcpy(&pc, V.prev_count + run, 4, cudaMemcpyDeviceToHost));
      const size_t bytes = (size_t)8 * pc;
      if (needed) *needed = bytes;
      if (!dst) return WE_OK;
      if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small (%zu < %zu)", dst_bytes, bytes);
      if (bytes) WE_CUDA_TRY(cudaMemcpy(dst, V.tlast + (size_t)run * E->cap, bytes, cudaMemcpyDefault));
      return WE_OK;
    }
    case WE_OUT_Z:
    case WE_OUT_NREC: {
      if (run < 0) return fail(WE_EINVAL, "walker arrays need a single run");
      if (what == WE_OUT_Z && !E->prm.bins.learned) return fail(WE_EINVAL, "WE_OUT_Z needs a learned bin map");
      int32_t pc = 0;
      WE_CUDA_TRY(cudaMemcpy(&pc, V.prev_count + run, 4, cudaMemcpyDeviceToHost));
      const size_t bytes = (size_t)4 * pc;
      if (needed) *needed = bytes;
      if (!dst) return WE_OK;
      if (dst_bytes < bytes) return fail(WE_EINVAL, "dst too small (%zu < %zu)", dst_bytes, bytes);
      const void *src = what == WE_OUT_Z ? (const void *)(E->prm.bins.zout + (size_t)run * E->cap)
                                         : (const void *)(V.nrec + (size_t)run * E->cap);
      if (bytes) WE_CUDA_TRY(cudaMemcpy(dst, src, bytes, cudaMemcpyDefault));
      return WE_OK;
    }
    case WE_OUT_RW: {
      if (E->prm.rw.period <= 0) return fail(WE_EINVAL, "WE_OUT_RW needs reweight_period > 0");
      return per_iter(E->prm.rw.obs, 4);
    }
    case WE_OUT_NEAR_TAU: return per_iter(V.obs_near, 4);
    case WE_OUT_FPT: {
      if (!V.fpt) return fail(WE_EINVAL, "WE_OUT_FPT needs feedback = WE_FEEDBACK_ABSORB");
      return per_walker(V.fpt, 8);
    }
    case WE_OUT_ITER: return scalar(&iter, 4);
    case WE_OUT_RECORDED: { int32_t v = rec; return scalar(&v, 4); }
    default: return fail(WE_EINVAL, "unknown output selector %d", what);
  }
}

extern "C" we_status we_ensemble_fpt_mle(we_ensemble *E, double T, void *dst, size_t dst_bytes, void *stream) {
  if (!E) return fail(WE_EINVAL, "ensemble is NULL");
  if (!E->prm.ens.fpt) return fail(WE_EINVAL, "the MLE needs an absorbing ensemble (feedback = WE_FEEDBACK_ABSORB)");
  if (E->phase_propagated) return fail(WE_EINVAL, "fpt_mle called between propagate and resample");
  const int R = E->cfg.n_runs;
  if (!dst || dst_bytes < (size_t)R * 5 * sizeof(double)) return fail(WE_EINVAL, "dst must hold runs x 5 doubles");
  if (std::isnan(T) || std::isinf(T)) return fail(WE_EINVAL, "T must be finite");
  const double simulated = (double)(E->cfg.first_iter + E->iters_enqueued) * E->cfg.tau;
  if (T > simulated * (1.0 + 1e-12))
    return fail(WE_EINVAL, "T = %g is past the %g simulated so far: runs that did not pass were not followed to T",
                T, simulated);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double *res = at<double>(E->ws, E->off.mle);
  cudaError_t e = launch_fpt_mle(E->prm.ens, T, res, s);
  if (e) return cuda_fail(e, "fpt_mle launch");
  WE_CUDA_TRY(cudaStreamSynchronize(s));
  WE_CUDA_TRY(cudaMemcpy(dst, res, (size_t)R * 5 * sizeof(double), cudaMemcpyDefault));
  return WE_OK;
}

extern "C" we_status we_run(const we_network *n, const we_binmap *b, const we_run_config *c,
                            void *stream, we_ensemble **out) {
  if (!out) return fail(WE_EINVAL, "out is NULL");
  *out = nullptr;
  we_ensemble *E = nullptr;
  we_status st = we_ensemble_create(n, b, c, nullptr, 0, stream, &E);
  if (st) return st;
  st = we_ensemble_step(E, c->record_iters, stream);
  if (!st) st = we_ensemble_sync(E, stream);
  if (st && st != WE_ESTEPCAP && st != WE_EOVERFLOW) { we_ensemble_destroy(E); return st; }
  *out = E;
  return st;
}

// ------------------------------------------------------------------------------------------
// autotuner: time every supported (mapping, block) on a short probe, cache per shape
// ------------------------------------------------------------------------------------------
static std::mutex g_tune_mu;
// (device name, S, M, walker slots, initial walkers) -> (mapping, block_threads)
using TuneKey = std::tuple<std::string, int, int, int, int>;
static std::map<TuneKey, std::pair<int, int>> g_tune_cache;

static std::string device_name() {
  int dev = 0;
  cudaDeviceProp pr;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&pr, dev) != cudaSuccess) {
    cudaGetLastError();
    return "unknown";
  }
  std::string nm(pr.name);
  for (auto &ch : nm) if (ch == ' ' || ch == '\t' || ch == '\n') ch = '_';
  return nm;
}

// One line per entry: device S M walker_slots n_init mapping block_threads
extern "C" we_status we_autotune_cache_save(const char *path) {
  if (!path) return fail(WE_EINVAL, "path is NULL");
  std::lock_guard<std::mutex> lk(g_tune_mu);
  FILE *f = std::fopen(path, "w");
  if (!f) return fail(WE_EINVAL, "cannot write %s", path);
  for (const auto &kv : g_tune_cache)
    std::fprintf(f, "%s %d %d %d %d %d %d\n", std::get<0>(kv.first).c_str(), std::get<1>(kv.first),
                 std::get<2>(kv.first), std::get<3>(kv.first), std::get<4>(kv.first), kv.second.first, kv.second.second);
  const bool ok = std::fclose(f) == 0;
  return ok ? WE_OK : fail(WE_EINVAL, "cannot write %s", path);
}

extern "C" we_status we_autotune_cache_load(const char *path) {
  if (!path) return fail(WE_EINVAL, "path is NULL");
  FILE *f = std::fopen(path, "r");
  if (!f) return fail(WE_EINVAL, "cannot read %s", path);
  std::lock_guard<std::mutex> lk(g_tune_mu);
  char name[256];
  int S, M, W, n0, map, bt, line = 0;
  we_status st = WE_OK;
  for (;;) {
    const int got = std::fscanf(f, "%255s %d %d %d %d %d %d", name, &S, &M, &W, &n0, &map, &bt);
    if (got == EOF) break;
    ++line;
    if (got != 7 || S < 1 || M < 1 || W < 1 || n0 < 1 ||
        (map != WE_MAP_THREAD && map != WE_MAP_WARP && map != WE_MAP_THREAD_TABLE) || bt < 32 || bt > 1024) {
      st = fail(WE_EINVAL, "%s: line %d is not a tuning entry", path, line);
      break;
    }
    g_tune_cache[TuneKey(name, S, M, W, n0)] = {map, bt};
  }
  std::fclose(f);
  return st;
}

extern "C" void we_autotune_cache_clear(void) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune_cache.clear();
}

extern "C" we_status we_autotune(const we_network *n, const we_binmap *b, const we_run_config *c,
                                 void *stream, int32_t *mapping, int32_t *block_threads) {
  if (!mapping || !block_threads) return fail(WE_EINVAL, "outputs are NULL");
  int cap = 0;
  we_status st = check_config(n, b, c, &cap);
  if (st) return st;
  const TuneKey key(device_name(), n->S, n->M, c->n_runs * cap, c->n_init);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) { *mapping = it->second.first; *block_threads = it->second.second; return WE_OK; }
  }
  std::vector<std::pair<int, int>> cands;
  if (table_len_for(n) > 0)
    for (int bt : {32, 64, 128}) cands.push_back({WE_MAP_THREAD_TABLE, bt});
  if (n->P <= kThreadMaxLeaves && n->S <= kThreadMaxSpecies)
    for (int bt : {32, 64, 128}) cands.push_back({WE_MAP_THREAD, bt});
  cands.push_back({WE_MAP_WARP, 32});
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float best = 1e30f;
  std::pair<int, int> pick = cands.front();
  cudaEvent_t e0, e1;
  WE_CUDA_TRY(cudaEventCreate(&e0));
  WE_CUDA_TRY(cudaEventCreate(&e1));
  for (auto cd : cands) {
    we_run_config cc = *c;
    cc.mapping = cd.first; cc.block_threads = cd.second; cc.record_iters = 4;
    we_ensemble *E = nullptr;
    if (we_ensemble_create(n, b, &cc, nullptr, 0, stream, &E) != WE_OK) continue;
    bool ok = we_ensemble_step(E, 1, stream) == WE_OK && cudaStreamSynchronize(s) == cudaSuccess;
    cudaEventRecord(e0, s);
    ok = ok && we_ensemble_step(E, 3, stream) == WE_OK;
    cudaEventRecord(e1, s);
    ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
    float ms = 0;
    if (ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess && ms < best) { best = ms; pick = cd; }
    we_ensemble_destroy(E);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaGetLastError();
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = pick;
  }
  *mapping = pick.first;
  *block_threads = pick.second;
  return WE_OK;
}
