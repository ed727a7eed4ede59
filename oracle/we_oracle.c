/*
 * we_oracle.c -- plain CPU oracle for the weighted-ensemble Gillespie-SSA hot path of
 * arXiv:1303.5986.  TEST INFRASTRUCTURE ONLY: the product library never links or calls it.
 *
 * Written to be read against the paper, not to be fast: propensities are recomputed in full
 * after every event, the canonical propensity tree is rebuilt from the leaves every time it is
 * needed, and every bin is searched linearly.  Floating point is IEEE double throughout; build
 * with -ffp-contract=off so that no multiply-add is fused (the rounding of every operation is
 * part of the definition below).
 */
#include "we_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------------
 * Philox-4x32-10 (Salmon, Moraes, Dror & Shaw, "Parallel random numbers: as easy as 1, 2, 3",
 * SC'11).  One round multiplies counter words 0 and 2 by the two Philox multipliers, keeps
 * the 64-bit products' halves, and mixes the high halves with the other two counter words and
 * the key; the key is bumped by the two Weyl constants between rounds.  Ten rounds.
 * ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;
  const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)mul0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)mul1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += weyl0;
    k1 += weyl1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

double orc_u01(uint32_t hi, uint32_t lo) {
  uint64_t m = ((uint64_t)hi << 20) | (uint64_t)(lo >> 12);   /* 52 random bits */
  return (double)(2u * m + 1u) * 0x1p-53;                      /* exact, in (0, 1) */
}

/* Key of a run: word 0 = low half of the seed, word 1 = high half plus the run id (mod 2^32). */
static void run_key(uint64_t seed, uint32_t run_id, uint32_t key[2]) {
  key[0] = (uint32_t)seed;
  key[1] = (uint32_t)(seed >> 32) + run_id;
}

/* ------------------------------------------------------------------------------------------
 * Network.  Mass action with combinatorial factors: a reactant taken m times contributes
 * C(x, m) = x(x-1).../m!; this is the convention under which the Schloegl model (Sec. III.B.1,
 * Eq. "schlogl") has its stable states at X=82 and X=563 and barrier at X=256 (Sec. III.B.3).
 * Species held constant (A and B in the Schloegl model) are folded into the rate constant.
 * Hill repression (Sec. III.C.1): a = c / (1 + (y/K)^n), written as c K^n / (K^n + y^n).
 * ------------------------------------------------------------------------------------------ */
struct orc_net {
  int32_t S, M;
  int32_t *n_reac;      /* dynamic reactant entries per reaction (<= 3) */
  int32_t *reac_sp;     /* M x 3 */
  int32_t *reac_m;      /* M x 3 */
  double *keff;         /* mass action: folded rate constant; Hill: c * K^n (folded) */
  int32_t *law;
  int32_t *hill_sp;
  int32_t *hill_n;
  double *hill_Kn;      /* K^n */
  int32_t *d_ptr, *d_sp, *d_val;   /* net change of dynamic species per reaction */
};

static int64_t binom_small(int64_t x, int32_t m) {
  if (m == 1) return x;
  if (m == 2) return x * (x - 1) / 2;
  return x * (x - 1) * (x - 2) / 6;
}

void orc_net_destroy(orc_net *n) {
  if (!n) return;
  free(n->n_reac); free(n->reac_sp); free(n->reac_m); free(n->keff); free(n->law);
  free(n->hill_sp); free(n->hill_n); free(n->hill_Kn); free(n->d_ptr); free(n->d_sp); free(n->d_val);
  free(n);
}

int orc_net_create(const orc_network_in *in, orc_net **out) {
  *out = NULL;
  if (!in || in->n_species < 1 || in->n_reactions < 1) return ORC_EINVAL;
  const int32_t S = in->n_species, M = in->n_reactions;
  if (!in->reac_ptr || !in->prod_ptr || !in->rate) return ORC_EINVAL;
  orc_net *n = (orc_net *)calloc(1, sizeof(orc_net));
  if (!n) return ORC_ENOMEM;
  n->S = S; n->M = M;
  n->n_reac = calloc(M, sizeof(int32_t)); n->reac_sp = calloc(3 * (size_t)M, sizeof(int32_t));
  n->reac_m = calloc(3 * (size_t)M, sizeof(int32_t)); n->keff = calloc(M, sizeof(double));
  n->law = calloc(M, sizeof(int32_t)); n->hill_sp = calloc(M, sizeof(int32_t));
  n->hill_n = calloc(M, sizeof(int32_t)); n->hill_Kn = calloc(M, sizeof(double));
  n->d_ptr = calloc((size_t)M + 1, sizeof(int32_t));
  n->d_sp = calloc((size_t)M * S, sizeof(int32_t)); n->d_val = calloc((size_t)M * S, sizeof(int32_t));
  int64_t *reac_mult = calloc(S, sizeof(int64_t)), *net = calloc(S, sizeof(int64_t));
  if (!n->n_reac || !n->reac_sp || !n->reac_m || !n->keff || !n->law || !n->hill_sp || !n->hill_n ||
      !n->hill_Kn || !n->d_ptr || !n->d_sp || !n->d_val || !reac_mult || !net) {
    free(reac_mult); free(net); orc_net_destroy(n); return ORC_ENOMEM;
  }
  int rc = ORC_OK;
  int32_t nd = 0;
  for (int32_t j = 0; j < M && rc == ORC_OK; ++j) {
    memset(reac_mult, 0, sizeof(int64_t) * S);
    memset(net, 0, sizeof(int64_t) * S);
    int32_t order = 0;
    for (int32_t e = in->reac_ptr[j]; e < in->reac_ptr[j + 1]; ++e) {
      int32_t s = in->reac_species[e], m = in->reac_mult[e];
      if (s < 0 || s >= S || m < 1 || m > 3) { rc = ORC_EINVAL; break; }
      reac_mult[s] += m; net[s] -= m; order += m;
    }
    for (int32_t e = in->prod_ptr[j]; e < in->prod_ptr[j + 1] && rc == ORC_OK; ++e) {
      int32_t s = in->prod_species[e], m = in->prod_mult[e];
      if (s < 0 || s >= S || m < 0) { rc = ORC_EINVAL; break; }
      net[s] += m;
    }
    if (rc != ORC_OK) break;
    if (order > 3) { rc = ORC_EINVAL; break; }
    double c = in->rate[j];
    if (!(c >= 0.0) || isinf(c)) { rc = ORC_EINVAL; break; }
    int32_t law = in->rate_law ? in->rate_law[j] : ORC_MASS_ACTION;
    if (law != ORC_MASS_ACTION && law != ORC_HILL_REPRESSION) { rc = ORC_EINVAL; break; }
    /* fold held-constant reactants, ascending species order */
    double k = c;
    int32_t nr = 0;
    for (int32_t s = 0; s < S; ++s) {
      if (reac_mult[s] == 0) continue;
      int32_t fixed = in->fixed_count ? in->fixed_count[s] : -1;
      if (fixed >= 0) {
        k = k * (double)binom_small(fixed, (int32_t)reac_mult[s]);
      } else {
        n->reac_sp[3 * j + nr] = s;
        n->reac_m[3 * j + nr] = (int32_t)reac_mult[s];
        ++nr;
      }
    }
    n->n_reac[j] = nr;
    n->law[j] = law;
    if (law == ORC_HILL_REPRESSION) {
      if (!in->hill_species || !in->hill_K || !in->hill_n || nr != 0) { rc = ORC_EINVAL; break; }
      int32_t hs = in->hill_species[j], hn = in->hill_n[j];
      double K = in->hill_K[j];
      if (hs < 0 || hs >= S || hn < 1 || hn > 3 || !(K > 0.0) || isinf(K)) { rc = ORC_EINVAL; break; }
      double Kn = K;
      for (int32_t p = 1; p < hn; ++p) Kn = Kn * K;
      n->hill_sp[j] = hs; n->hill_n[j] = hn; n->hill_Kn[j] = Kn;
      n->keff[j] = k * Kn;
    } else {
      n->keff[j] = k;
    }
    n->d_ptr[j] = nd;
    for (int32_t s = 0; s < S; ++s) {
      int32_t fixed = in->fixed_count ? in->fixed_count[s] : -1;
      if (fixed >= 0 || net[s] == 0) continue;
      n->d_sp[nd] = s; n->d_val[nd] = (int32_t)net[s]; ++nd;
    }
  }
  n->d_ptr[M] = nd;
  free(reac_mult); free(net);
  if (rc != ORC_OK) { orc_net_destroy(n); return rc; }
  *out = n;
  return ORC_OK;
}

int32_t orc_net_n_species(const orc_net *n) { return n->S; }
int32_t orc_net_n_reactions(const orc_net *n) { return n->M; }
double orc_net_keff(const orc_net *n, int32_t j) { return n->keff[j]; }

static double propensity_of(const orc_net *n, int32_t j, const int32_t *x) {
  if (n->law[j] == ORC_HILL_REPRESSION) {
    int64_t y = x[n->hill_sp[j]];
    int64_t yn = y;
    for (int32_t p = 1; p < n->hill_n[j]; ++p) yn *= y;
    double den = n->hill_Kn[j] + (double)yn;
    return n->keff[j] / den;
  }
  int64_t h = 1;
  for (int32_t r = 0; r < n->n_reac[j]; ++r)
    h *= binom_small(x[n->reac_sp[3 * j + r]], n->reac_m[3 * j + r]);
  return n->keff[j] * (double)h;
}

void orc_propensities(const orc_net *n, const int32_t *x, double *a) {
  for (int32_t j = 0; j < n->M; ++j) a[j] = propensity_of(n, j, x);
}

/* ------------------------------------------------------------------------------------------
 * Canonical total propensity a0 = sum_j a_j (Sec. II.A: the waiting time is exponential with
 * rate a0 and reaction j is chosen with probability a_j/a0).  The sum is fixed to one shape so
 * that every implementation reaches the same double: a complete binary tree over the leaves,
 * padded with +0.0 to a power of two, each node the rounded sum of its two children.
 * ------------------------------------------------------------------------------------------ */
static int32_t pow2_at_least(int32_t n) { int32_t p = 1; while (p < n) p <<= 1; return p; }

static double *build_heap(int32_t n, const double *a, int32_t *P_out) {
  int32_t P = pow2_at_least(n);
  double *node = (double *)calloc(2 * (size_t)P, sizeof(double));
  if (!node) return NULL;
  for (int32_t j = 0; j < n; ++j) node[P + j] = a[j];
  for (int32_t k = P - 1; k >= 1; --k) node[k] = node[2 * k] + node[2 * k + 1];
  *P_out = P;
  return node;
}

double orc_tree_total(int32_t n, const double *a) {
  int32_t P;
  double *node = build_heap(n, a, &P);
  if (!node) return NAN;
  double t = node[1];
  free(node);
  return t;
}

/* Descend from the root: go left while the target lies below the left sum; otherwise subtract
 * the left sum and go right -- unless the right subtree sums to zero, in which case stay left
 * (so a reaction with zero propensity is never chosen, whatever the rounding of the target). */
int32_t orc_tree_select(int32_t n, const double *a, double target) {
  int32_t P;
  double *node = build_heap(n, a, &P);
  if (!node) return -1;
  int32_t k = 1;
  while (k < P) {
    double L = node[2 * k], R = node[2 * k + 1];
    if (R == 0.0) {
      k = 2 * k;
    } else if (target < L) {
      k = 2 * k;
    } else {
      target = target - L;
      k = 2 * k + 1;
    }
  }
  free(node);
  return k - P;
}

/* ------------------------------------------------------------------------------------------
 * Target set B for steady-state recycling (Sec. II.B.2): the conjunction of the clauses.
 * ------------------------------------------------------------------------------------------ */
static int in_target(const orc_we_config *cfg, const int32_t *x) {
  if (cfg->n_clauses < 1) return 0;
  for (int32_t c = 0; c < cfg->n_clauses; ++c) {
    int32_t v = x[cfg->tgt_species[c]];
    if (cfg->tgt_op[c] == ORC_OP_GE) { if (!(v >= cfg->tgt_threshold[c])) return 0; }
    else { if (!(v <= cfg->tgt_threshold[c])) return 0; }
  }
  return 1;
}

/* ------------------------------------------------------------------------------------------
 * Gillespie's direct SSA (Sec. II.A) for one WE interval of length tau (the "propagate dynamics"
 * step of the WE algorithm, Sec. II.B).  Draw d of walker slot w in iteration i uses Philox
 * counter (d, i, w, 0): words 0-1 give u1 (waiting time), words 2-3 give u2 (which reaction).
 * A waiting time that would carry the clock past tau ends the interval; the unused remainder
 * is discarded, which leaves the process exact because the exponential clock is memoryless.
 * With feedback on, a walker that enters B is put back in the recycle state at once and keeps
 * running for the rest of the interval (first passage is detected at the event that crosses).
 * With absorbing feedback (the brute-force runs of Sec. II.C, which record the time of the
 * first transition), a walker stops at the event that enters B and stays there; one that starts
 * the interval inside B fires nothing.  With the end-of-interval check (feedback 3: B checked
 * at a prescribed time step, Sec. IV), only a walker in B when the interval ends is recycled.
 * ------------------------------------------------------------------------------------------ */
int orc_propagate(const orc_net *n, const orc_we_config *cfg, int32_t iter, int32_t slot,
                  int32_t *x, int64_t *n_ev, int32_t *n_rec, double *t_last) {
  const int32_t S = n->S, M = n->M;
  double *a = (double *)malloc(sizeof(double) * M);
  int32_t *xn = (int32_t *)malloc(sizeof(int32_t) * S);
  if (!a || !xn) { free(a); free(xn); return ORC_ENOMEM; }
  uint32_t key[2];
  run_key(cfg->seed, cfg->run_id, key);
  double t = 0.0;
  uint32_t draw = 0;
  int64_t ev = 0;
  int32_t rec = 0;
  int status = ORC_OK;
  orc_propensities(n, x, a);
  for (;;) {
    if (cfg->feedback == 2 && in_target(cfg, x)) break;      /* absorbed: nothing more fires */
    double a0 = orc_tree_total(M, a);
    if (!(a0 > 0.0)) break;                     /* nothing can fire: idle to the end of tau */
    uint32_t ctr[4] = {draw, (uint32_t)iter, (uint32_t)slot, 0u}, r[4];
    ++draw;
    orc_philox4x32_10(ctr, key, r);
    double u1 = orc_u01(r[0], r[1]);
    double u2 = orc_u01(r[2], r[3]);
    double e = -log(u1);
    double dt = e / a0;
    double tn = t + dt;
    if (tn > cfg->tau) break;
    if (ev >= (cfg->max_steps > 0 ? cfg->max_steps : ORC_DEFAULT_MAX_STEPS)) { status = ORC_ESTEPCAP; break; }
    double target = u2 * a0;
    int32_t j = orc_tree_select(M, a, target);
    memcpy(xn, x, sizeof(int32_t) * S);
    int over = 0;
    for (int32_t e2 = n->d_ptr[j]; e2 < n->d_ptr[j + 1]; ++e2) {
      int64_t v = (int64_t)xn[n->d_sp[e2]] + n->d_val[e2];
      if (v > ORC_MAX_COUNT) over = 1;
      xn[n->d_sp[e2]] = (int32_t)v;
    }
    if (over) { status = ORC_EOVERFLOW; break; }
    memcpy(x, xn, sizeof(int32_t) * S);
    ++ev;
    t = tn;
    if ((cfg->feedback == 1 || cfg->feedback == 2) && in_target(cfg, x)) {
      ++rec;
      if (cfg->feedback == 2) break;                          /* first passage: stop here */
      memcpy(x, cfg->recycle_state, sizeof(int32_t) * S);
    }
    orc_propensities(n, x, a);
  }
  free(a); free(xn);
  if (cfg->feedback == 3 && in_target(cfg, x)) {             /* checked at the interval's end */
    ++rec;
    memcpy(x, cfg->recycle_state, sizeof(int32_t) * S);
  }
  *n_ev = ev;
  *n_rec = rec;
  if (t_last) *t_last = t;
  return status;
}

/* Grid bins (Sec. II.B: non-overlapping bins on a regular 1-D or 2-D grid).  Bin k of a
 * dimension is [edge_k, edge_{k+1}); values below the first edge go to bin 0, values at or above
 * the last edge to the last bin (an overflow bin is a last edge at +infinity).  The flat index is
 * row-major with the last dimension fastest. */
int32_t orc_bin_of(const orc_we_config *cfg, const int32_t *x) {
  int32_t flat = 0;
  const double *edges = cfg->bin_edges;
  for (int32_t d = 0; d < cfg->bin_ndim; ++d) {
    int32_t nb = cfg->bin_nbins[d];
    double v = (double)x[cfg->bin_species[d]];
    int32_t idx = 0;
    for (int32_t k = 0; k < nb; ++k)
      if (edges[k] <= v) idx = k;
    flat = flat * nb + idx;
    edges += nb + 1;
  }
  return flat;
}

/* ------------------------------------------------------------------------------------------
 * Split and merge inside each bin (Sec. II.B and its WE algorithm listing).  Bins are taken in
 * ascending order and a bin's walkers in ascending slot order.
 *  - More than M_targ: repeatedly merge the two lowest weights (Sec. II.B); ties go to the
 *    earlier position.  Of the pair (earlier p, later q) p survives with probability
 *    w_p/(w_p+w_q), decided by u < w_p/(w_p+w_q) with u from Philox counter (k, i, bin, 1) where
 *    k counts the merges done in this bin this iteration.  The survivor keeps its position and
 *    takes the pair's summed weight.
 *  - Fewer than M_targ (and at least one): replicate until the bin holds M_targ.  Each walker
 *    starts with one copy; the next copy goes to the walker whose per-copy weight w_i/c_i is
 *    largest (ties to the earlier one).  Every copy carries w_i/c_i, which for a lone walker is
 *    the paper's w/M_targ.  Copies follow their parent.
 * The output is the concatenation over bins; parent[] holds the input slot of each output.
 * ------------------------------------------------------------------------------------------ */
int32_t orc_resample(int32_t n, int32_t S, const int32_t *states, const double *weights,
                     const int32_t *bins, int32_t n_bins, int32_t m_targ, int32_t iter,
                     uint64_t seed, uint32_t run_id, int32_t capacity,
                     int32_t *out_states, double *out_weights, int32_t *out_parent) {
  if (m_targ < 1 || n < 0 || n_bins < 1) return ORC_EINVAL;
  uint32_t key[2];
  run_key(seed, run_id, key);
  int32_t *ls = (int32_t *)malloc(sizeof(int32_t) * (n > 0 ? n : 1));
  double *lw = (double *)malloc(sizeof(double) * (n > 0 ? n : 1));
  int32_t *cp = (int32_t *)malloc(sizeof(int32_t) * (m_targ + 1));
  if (!ls || !lw || !cp) { free(ls); free(lw); free(cp); return ORC_ENOMEM; }
  int32_t out = 0;
  int32_t status = 0;
  for (int32_t b = 0; b < n_bins && status == 0; ++b) {
    int32_t cnt = 0;
    for (int32_t w = 0; w < n; ++w)
      if (bins[w] == b) { ls[cnt] = w; lw[cnt] = weights[w]; ++cnt; }
    if (cnt == 0) continue;
    if (cnt > m_targ) {
      uint32_t k = 0;
      while (cnt > m_targ) {
        int32_t ia = 0;
        for (int32_t i = 1; i < cnt; ++i) if (lw[i] < lw[ia]) ia = i;
        int32_t ib = (ia == 0) ? 1 : 0;
        for (int32_t i = 0; i < cnt; ++i) if (i != ia && lw[i] < lw[ib]) ib = i;
        int32_t p = ia < ib ? ia : ib, q = ia < ib ? ib : ia;
        uint32_t ctr[4] = {k, (uint32_t)iter, (uint32_t)b, 1u}, r[4];
        ++k;
        orc_philox4x32_10(ctr, key, r);
        double u = orc_u01(r[0], r[1]);
        double wsum = lw[p] + lw[q];
        double prob = lw[p] / wsum;
        int32_t gone;
        if (u < prob) { lw[p] = wsum; gone = q; }
        else { lw[q] = wsum; gone = p; }
        for (int32_t i = gone; i + 1 < cnt; ++i) { ls[i] = ls[i + 1]; lw[i] = lw[i + 1]; }
        --cnt;
      }
      for (int32_t i = 0; i < cnt; ++i) {
        if (out >= capacity) { status = ORC_EOVERFLOW; break; }
        memcpy(out_states + (size_t)out * S, states + (size_t)ls[i] * S, sizeof(int32_t) * S);
        out_weights[out] = lw[i]; out_parent[out] = ls[i]; ++out;
      }
    } else {
      for (int32_t i = 0; i < cnt; ++i) cp[i] = 1;
      for (int32_t extra = cnt; extra < m_targ; ++extra) {
        int32_t best = 0;
        double bw = lw[0] / (double)cp[0];
        for (int32_t i = 1; i < cnt; ++i) {
          double v = lw[i] / (double)cp[i];
          if (v > bw) { bw = v; best = i; }
        }
        cp[best] += 1;
      }
      for (int32_t i = 0; i < cnt && status == 0; ++i) {
        double wc = lw[i] / (double)cp[i];
        for (int32_t c = 0; c < cp[i]; ++c) {
          if (out >= capacity) { status = ORC_EOVERFLOW; break; }
          memcpy(out_states + (size_t)out * S, states + (size_t)ls[i] * S, sizeof(int32_t) * S);
          out_weights[out] = wc; out_parent[out] = ls[i]; ++out;
        }
      }
    }
  }
  free(ls); free(lw); free(cp);
  return status ? status : out;
}

/* ------------------------------------------------------------------------------------------
 * Steady-state reweighting (Sec. II.B.2, Eq. "ss").  In steady state the weight flowing into
 * each bin equals the weight flowing out: sum_j (k_ij w_j - k_ji w_i) = 0, with f_ij = k_ij w_j
 * the flux into bin i from bin j.  The rates are estimated from the measured transfers,
 * k_ij = F_ij / W_j, where F_ij is the weight that started an interval in bin j and ended it in
 * bin i, and W_j = sum_i F_ij (ascending i) the weight that started in j, both summed over all
 * intervals so far.  The bins taken are the largest strongly connected component of the
 * observed transfers among the bins with W_j > 0 (so that the estimated chain on them is
 * irreducible and its steady state unique and positive); transfers that leave that set are
 * left out, and bins outside it keep their weights.  The balance equations on that set are
 * solved by the elimination of Grassmann, Taksar and Heyman (GTH): states are removed from the
 * last to the first, each one's exit rates folded into the rates among the remaining states,
 * then the weights are rebuilt from the first state on.  It only adds, multiplies and divides
 * non-negative numbers, so every weight keeps its relative accuracy -- steady-state bin weights
 * in WE span many orders of magnitude, and Gaussian elimination with pivoting leaves the small
 * ones with absolute errors of ~1e-17 that can make them negative.  Bins that hold walkers now take
 * the solved weights, scaled so that their total is unchanged: the walkers of bin i are
 * multiplied by (x_i q) / c_i with q = (sum of their current weights c) / (sum of their x).
 * Nothing is changed when the set has fewer than two bins, an eliminated state has no exit
 * rate left (not possible for an irreducible chain unless rates underflow), or a bin holding
 * walkers gets a solved weight that is not positive.
 * ------------------------------------------------------------------------------------------ */
/* The largest strongly connected component of the observed-transfer graph over the active bins
 * act[0..n) (edge j -> i when i != j and F[i][j] > 0), written ascending to out; returns its
 * size.  Largest by bin count, ties to the component with the lowest bin.  Components found by
 * Kosaraju's two depth-first passes (finish order, then the transposed graph). */
static int32_t largest_scc(int32_t n, const int32_t *act, const double *F, int32_t nb, int32_t *out) {
  int32_t *seen = (int32_t *)calloc(n, sizeof(int32_t));
  int32_t *order = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *nxt = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t *comp = (int32_t *)malloc(sizeof(int32_t) * n);
  int32_t best_size = 0;
  if (!seen || !order || !stk || !nxt || !comp) goto done;
  {
    int32_t no = 0;
    for (int32_t s0 = 0; s0 < n; ++s0) {
      if (seen[s0]) continue;
      int32_t top = 0;
      stk[0] = s0; nxt[0] = 0; seen[s0] = 1;
      while (top >= 0) {
        const int32_t j = stk[top];
        int32_t i = nxt[top];
        while (i < n && (i == j || seen[i] || !(F[(size_t)act[i] * nb + act[j]] > 0.0))) ++i;
        if (i < n) {
          nxt[top] = i + 1;
          seen[i] = 1;
          ++top; stk[top] = i; nxt[top] = 0;
        } else {
          order[no++] = j;
          --top;
        }
      }
    }
    for (int32_t k = 0; k < n; ++k) comp[k] = -1;
    int32_t nc = 0;
    for (int32_t q = n - 1; q >= 0; --q) {
      const int32_t s1 = order[q];
      if (comp[s1] >= 0) continue;
      int32_t top = 0;
      stk[0] = s1; nxt[0] = 0; comp[s1] = nc;
      while (top >= 0) {
        const int32_t j = stk[top];
        int32_t i = nxt[top];                     /* transposed: i -> j exists when F[j][i] > 0 */
        while (i < n && (i == j || comp[i] >= 0 || !(F[(size_t)act[j] * nb + act[i]] > 0.0))) ++i;
        if (i < n) {
          nxt[top] = i + 1;
          comp[i] = nc;
          ++top; stk[top] = i; nxt[top] = 0;
        } else {
          --top;
        }
      }
      ++nc;
    }
    int32_t best = -1, best_min = 0;
    for (int32_t c = 0; c < nc; ++c) {
      int32_t size = 0, mn = n;
      for (int32_t k = 0; k < n; ++k)
        if (comp[k] == c) { ++size; if (k < mn) mn = k; }
      if (size > best_size || (size == best_size && mn < best_min)) { best = c; best_size = size; best_min = mn; }
    }
    int32_t m = 0;
    for (int32_t k = 0; k < n; ++k)
      if (comp[k] == best) out[m++] = act[k];
  }
done:
  free(seen); free(order); free(stk); free(nxt); free(comp);
  return best_size;
}

int32_t orc_rw_solve(int32_t nb, const double *F, const double *cb, double *fac) {
  for (int32_t b = 0; b < nb; ++b) fac[b] = 0.0;
  double *W = (double *)malloc(sizeof(double) * nb);
  int32_t *A = (int32_t *)malloc(sizeof(int32_t) * nb);
  if (!W || !A) { free(W); free(A); return -1; }
  int32_t na = 0;
  for (int32_t b = 0; b < nb; ++b) {
    double s = 0.0;
    for (int32_t e = 0; e < nb; ++e) s = s + F[(size_t)e * nb + b];
    W[b] = s;
    if (s > 0.0) A[na++] = b;
  }
  int32_t result = -1;
  double *M = NULL, *x = NULL;
  int32_t n = na >= 2 ? largest_scc(na, A, F, nb, A) : 0;
  if (n < 2) goto done;
  M = (double *)malloc(sizeof(double) * (size_t)n * n);
  x = (double *)malloc(sizeof(double) * n);
  if (!M || !x) goto done;
  /* R[a][b]: rate from the a-th to the b-th bin of the set, k_ba = F[b][a] / W[a] */
  for (int32_t a = 0; a < n; ++a)
    for (int32_t b = 0; b < n; ++b)
      M[(size_t)a * n + b] = a == b ? 0.0 : F[(size_t)A[b] * nb + A[a]] / W[A[a]];
  /* GTH elimination, last state first: fold state k's exits into the others' rates */
  for (int32_t k = n - 1; k >= 1; --k) {
    double out = 0.0;
    for (int32_t j = 0; j < k; ++j) out = out + M[(size_t)k * n + j];
    if (!(out > 0.0)) goto done;
    for (int32_t i = 0; i < k; ++i) M[(size_t)i * n + k] = M[(size_t)i * n + k] / out;
    for (int32_t i = 0; i < k; ++i)
      for (int32_t j = 0; j < k; ++j)
        if (i != j) M[(size_t)i * n + j] = M[(size_t)i * n + j] + M[(size_t)i * n + k] * M[(size_t)k * n + j];
  }
  x[0] = 1.0;
  for (int32_t k = 1; k < n; ++k) {
    double v = 0.0;
    for (int32_t i = 0; i < k; ++i) v = v + x[i] * M[(size_t)i * n + k];
    x[k] = v;
  }
  {
    double C = 0.0, T = 0.0;
    int32_t held = 0;
    for (int32_t i = 0; i < n; ++i) {
      if (!(cb[A[i]] > 0.0)) continue;
      if (!(x[i] > 0.0) || isinf(x[i])) goto done;
      C = C + cb[A[i]];
      T = T + x[i];
      ++held;
    }
    if (held == 0 || !(T > 0.0) || isinf(T)) goto done;
    const double q = C / T;
    for (int32_t i = 0; i < n; ++i)
      if (cb[A[i]] > 0.0) fac[A[i]] = (x[i] * q) / cb[A[i]];
    result = 1;
  }
done:
  free(W); free(A); free(M); free(x);
  return result;
}

/* ------------------------------------------------------------------------------------------
 * The WE procedure (Sec. II.B, algorithm listing): for each iteration, propagate every walker for
 * tau, record the observables, then split/merge per bin.  Observables per iteration: the
 * recycled weight (its ratio to tau is the flux whose inverse is the MFPT, Eq. "mfpt"), the
 * number of events, a weighted histogram of one species taken after propagation and before
 * resampling (the estimate of P(x, t) of Sec. II.B.1), and the total weight and walker count
 * after resampling.
 * ------------------------------------------------------------------------------------------ */
static int we_run_impl(const orc_net *n, const orc_dg *dg, const orc_we_config *cfg, orc_we_out *out);

int orc_we_run(const orc_net *n, const orc_we_config *cfg, orc_we_out *out) {
  return we_run_impl(n, NULL, cfg, out);
}

static int we_run_impl(const orc_net *n, const orc_dg *dg, const orc_we_config *cfg, orc_we_out *out) {
  const int32_t S = n->S;
  const int32_t cap = cfg->capacity;
  if (cfg->n_init < 1 || cfg->n_init > cap || cfg->m_targ < 1 || !(cfg->tau > 0.0) ||
      cfg->n_iters < 0 || cfg->bin_ndim < 1 || cfg->bin_ndim > 4)
    return out->status = ORC_EINVAL;
  int32_t n_bins = 1;
  for (int32_t d = 0; d < cfg->bin_ndim; ++d) n_bins *= cfg->bin_nbins[d];
  int32_t *st = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap * S);
  int32_t *st2 = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap * S);
  double *w = (double *)malloc(sizeof(double) * cap);
  double *w2 = (double *)malloc(sizeof(double) * cap);
  int32_t *par = (int32_t *)malloc(sizeof(int32_t) * cap);
  int32_t *bins = (int32_t *)malloc(sizeof(int32_t) * cap);
  int32_t *nrec = (int32_t *)malloc(sizeof(int32_t) * cap);
  if (!st || !st2 || !w || !w2 || !par || !bins || !nrec) {
    free(st); free(st2); free(w); free(w2); free(par); free(bins); free(nrec);
    return out->status = ORC_ENOMEM;
  }
  /* steady-state reweighting: start bin of every walker (-1: unknown, the initial walkers),
   * accumulated transfers F, a per-bin accumulator and the current bin weights */
  const int rw = cfg->reweight_period > 0 && cfg->resample;
  int32_t *sbin = (int32_t *)malloc(sizeof(int32_t) * cap);
  double *F = rw ? (double *)calloc((size_t)n_bins * n_bins, sizeof(double)) : NULL;
  double *acc = rw ? (double *)calloc((size_t)n_bins, sizeof(double)) : NULL;
  double *cb = rw ? (double *)calloc((size_t)n_bins, sizeof(double)) : NULL;
  double *fac = rw ? (double *)calloc((size_t)n_bins, sizeof(double)) : NULL;
  int32_t *mark = rw ? (int32_t *)malloc(sizeof(int32_t) * n_bins) : NULL;
  if (!sbin || (rw && (!F || !acc || !cb || !fac || !mark))) {
    free(st); free(st2); free(w); free(w2); free(par); free(bins); free(nrec);
    free(sbin); free(F); free(acc); free(cb); free(fac); free(mark);
    return out->status = ORC_ENOMEM;
  }
  for (int32_t i = 0; i < cap; ++i) sbin[i] = -1;
  for (int32_t b = 0; rw && b < n_bins; ++b) mark[b] = -1;
  int32_t nw = cfg->n_init;
  memcpy(st, cfg->init_states, sizeof(int32_t) * (size_t)nw * S);
  memcpy(w, cfg->init_weights, sizeof(double) * nw);
  for (int32_t i = 0; i < nw; ++i) par[i] = -1;
  if (out->first_passage)
    for (int32_t i = 0; i < cap; ++i) out->first_passage[i] = -1.0;
  const int absorb = cfg->feedback == 2 && !cfg->resample;
  int status = ORC_OK;
  for (int32_t li = 0; li < cfg->n_iters && status == ORC_OK; ++li) {
    int32_t iter = cfg->first_iter + li;
    int64_t events = 0;
    for (int32_t s = 0; s < nw; ++s) {
      int64_t ev = 0;
      double tl = 0.0;
      /* brute-force runs: a walker found inside B at the start of an interval entered it at
       * that time at the latest (only the initial walkers can be found there unrecorded) */
      if (absorb && out->first_passage && out->first_passage[s] < 0.0 && in_target(cfg, st + (size_t)s * S))
        out->first_passage[s] = (double)iter * cfg->tau;
      int32_t rc = dg ? orc_propagate_dg(dg, cfg, iter, s, st + (size_t)s * S, &ev, &nrec[s], &tl)
                      : orc_propagate(n, cfg, iter, s, st + (size_t)s * S, &ev, &nrec[s], &tl);
      if (out->t_last) out->t_last[s] = tl;
      if (absorb && out->first_passage && nrec[s] > 0 && out->first_passage[s] < 0.0)
        out->first_passage[s] = (double)iter * cfg->tau + tl;
      events += ev;
      if (rc != ORC_OK && status == ORC_OK) status = rc;
    }
    double flux = 0.0;
    for (int32_t s = 0; s < nw; ++s) flux = flux + (double)nrec[s] * w[s];
    out->flux_weight[li] = flux;
    out->events[li] = events;
    if (out->hist && cfg->hist_len > 0) {
      double *h = out->hist + (size_t)li * cfg->hist_len;
      for (int32_t k = 0; k < cfg->hist_len; ++k) h[k] = 0.0;
      for (int32_t s = 0; s < nw; ++s) {
        int32_t v = st[(size_t)s * S + cfg->hist_species];
        int32_t idx = v < cfg->hist_len - 1 ? v : cfg->hist_len - 1;
        h[idx] = h[idx] + w[s];
      }
    }
    if (status != ORC_OK) break;
    if (cfg->resample) {
      for (int32_t s = 0; s < nw; ++s) bins[s] = orc_bin_of(cfg, st + (size_t)s * S);
      if (rw) {
        /* transfers of this interval: the walkers of one start bin are consecutive slots in
         * ascending order (the resampling's output order); each (end, start) pair is summed
         * over them from 0, then added to F once */
        int32_t s0 = 0;
        while (s0 < nw) {
          int32_t s1 = s0;
          while (s1 < nw && sbin[s1] == sbin[s0]) ++s1;
          if (sbin[s0] >= 0) {
            const int32_t b = sbin[s0];
            for (int32_t s = s0; s < s1; ++s) {
              if (mark[bins[s]] != s0) { mark[bins[s]] = s0; acc[bins[s]] = 0.0; }
              acc[bins[s]] = acc[bins[s]] + w[s];
            }
            for (int32_t s = s0; s < s1; ++s)
              if (mark[bins[s]] == s0) {
                F[(size_t)bins[s] * n_bins + b] = F[(size_t)bins[s] * n_bins + b] + acc[bins[s]];
                mark[bins[s]] = -1;
              }
          }
          s0 = s1;
        }
      }
      int32_t m = orc_resample(nw, S, st, w, bins, n_bins, cfg->m_targ, iter, cfg->seed,
                               cfg->run_id, cap, st2, w2, par);
      if (m < 0) { status = m; break; }
      nw = m;
      int32_t *ts = st; st = st2; st2 = ts;
      double *tw = w; w = w2; w2 = tw;
      for (int32_t s = 0; s < nw; ++s) sbin[s] = bins[par[s]];
    } else {
      for (int32_t s = 0; s < nw; ++s) par[s] = s;
    }
    double tot = 0.0;
    for (int32_t s = 0; s < nw; ++s) tot = tot + w[s];
    out->total_weight[li] = tot;
    out->n_walkers[li] = nw;
    if (out->reweighted) out->reweighted[li] = 0;
    if (rw && (iter + 1) % cfg->reweight_period == 0) {      /* after iterations period-1, 2 period-1, ... */
      /* current bin weights, each summed over its walkers in ascending slot order */
      for (int32_t b = 0; b < n_bins; ++b) cb[b] = 0.0;
      for (int32_t s = 0; s < nw; ++s) cb[sbin[s]] = cb[sbin[s]] + w[s];
      const int32_t done = orc_rw_solve(n_bins, F, cb, fac);
      if (done == 1)
        for (int32_t s = 0; s < nw; ++s)
          if (fac[sbin[s]] != 0.0) w[s] = w[s] * fac[sbin[s]];
      if (out->reweighted) out->reweighted[li] = done;
    }
  }
  memcpy(out->states, st, sizeof(int32_t) * (size_t)nw * S);
  memcpy(out->weights, w, sizeof(double) * nw);
  memcpy(out->parent, par, sizeof(int32_t) * nw);
  out->n_final = nw;
  out->status = status;
  free(st); free(st2); free(w); free(w2); free(par); free(bins); free(nrec);
  free(sbin); free(F); free(acc); free(cb); free(fac); free(mark);
  return status;
}

/* ==========================================================================================
 * CPU BASELINE, not part of the oracle's definition: the same direct SSA with a dependency
 * graph -- after an event only the propensities that read a changed species are recomputed,
 * and only their paths to the root of the canonical tree -- so that the CPU figure set beside
 * the GPU's is not the oracle's O(M)-per-event strawman.  Every tree node is still the rounded
 * sum of its two children and the descent is the oracle's, so the results are identical to
 * orc_propagate's (checked by a CPU test); only the amount of work differs.
 * ========================================================================================== */
struct orc_dg {
  const orc_net *n;
  int32_t P;                 /* leaves of the canonical tree */
  int32_t *dep_ptr, *dep;    /* reactions whose propensity reads a species that reaction j changes */
};

void orc_dg_destroy(orc_dg *g) {
  if (!g) return;
  free(g->dep_ptr); free(g->dep); free(g);
}

int orc_dg_create(const orc_net *n, orc_dg **out) {
  *out = NULL;
  const int32_t S = n->S, M = n->M;
  orc_dg *g = (orc_dg *)calloc(1, sizeof(orc_dg));
  int32_t *rd_ptr = (int32_t *)calloc((size_t)S + 1, sizeof(int32_t));   /* species -> readers */
  int32_t *mark = (int32_t *)malloc(sizeof(int32_t) * (size_t)M);
  if (!g || !rd_ptr || !mark) { free(g); free(rd_ptr); free(mark); return ORC_ENOMEM; }
  g->n = n;
  g->P = pow2_at_least(M);
  for (int32_t j = 0; j < M; ++j) {
    if (n->law[j] == ORC_HILL_REPRESSION) rd_ptr[n->hill_sp[j] + 1]++;
    else for (int32_t r = 0; r < n->n_reac[j]; ++r) rd_ptr[n->reac_sp[3 * j + r] + 1]++;
  }
  for (int32_t s = 0; s < S; ++s) rd_ptr[s + 1] += rd_ptr[s];
  int32_t *rd = (int32_t *)malloc(sizeof(int32_t) * ((size_t)rd_ptr[S] + 1));
  int32_t *fill = (int32_t *)calloc((size_t)S, sizeof(int32_t));
  if (!rd || !fill) { free(rd); free(fill); free(rd_ptr); free(mark); free(g); return ORC_ENOMEM; }
  for (int32_t j = 0; j < M; ++j) {
    if (n->law[j] == ORC_HILL_REPRESSION) { int32_t s = n->hill_sp[j]; rd[rd_ptr[s] + fill[s]++] = j; }
    else for (int32_t r = 0; r < n->n_reac[j]; ++r) { int32_t s = n->reac_sp[3 * j + r]; rd[rd_ptr[s] + fill[s]++] = j; }
  }
  /* two passes over reactions: count, then fill the deduplicated dependents */
  g->dep_ptr = (int32_t *)calloc((size_t)M + 1, sizeof(int32_t));
  int rc = g->dep_ptr ? ORC_OK : ORC_ENOMEM;
  for (int pass = 0; pass < 2 && rc == ORC_OK; ++pass) {
    for (int32_t i = 0; i < M; ++i) mark[i] = -1;
    int32_t cnt = 0;
    for (int32_t j = 0; j < M; ++j) {
      if (pass == 1) g->dep_ptr[j] = cnt;
      for (int32_t e = n->d_ptr[j]; e < n->d_ptr[j + 1]; ++e) {
        int32_t s = n->d_sp[e];
        for (int32_t q = rd_ptr[s]; q < rd_ptr[s + 1]; ++q)
          if (mark[rd[q]] != j) { mark[rd[q]] = j; if (pass == 1) g->dep[cnt] = rd[q]; ++cnt; }
      }
    }
    if (pass == 0) { g->dep = (int32_t *)malloc(sizeof(int32_t) * ((size_t)cnt + 1)); if (!g->dep) rc = ORC_ENOMEM; }
    else g->dep_ptr[M] = cnt;
  }
  free(rd); free(fill); free(rd_ptr); free(mark);
  if (rc != ORC_OK) { orc_dg_destroy(g); return rc; }
  *out = g;
  return ORC_OK;
}

int orc_propagate_dg(const orc_dg *g, const orc_we_config *cfg, int32_t iter, int32_t slot,
                     int32_t *x, int64_t *n_ev, int32_t *n_rec, double *t_last) {
  const orc_net *n = g->n;
  const int32_t S = n->S, M = n->M, P = g->P;
  double *node = (double *)calloc(2 * (size_t)P, sizeof(double));
  if (!node) return ORC_ENOMEM;
  uint32_t key[2];
  run_key(cfg->seed, cfg->run_id, key);
  const int64_t cap = cfg->max_steps > 0 ? cfg->max_steps : ORC_DEFAULT_MAX_STEPS;
  double t = 0.0;
  uint32_t draw = 0;
  int64_t ev = 0;
  int32_t rec = 0;
  int status = ORC_OK;
#define DG_REBUILD()                                                             \
  do {                                                                          \
    for (int32_t j = 0; j < M; ++j) node[P + j] = propensity_of(n, j, x);        \
    for (int32_t k = P - 1; k >= 1; --k) node[k] = node[2 * k] + node[2 * k + 1]; \
  } while (0)
  DG_REBUILD();
  for (;;) {
    if (cfg->feedback == 2 && in_target(cfg, x)) break;
    double a0 = node[1];
    if (!(a0 > 0.0)) break;
    uint32_t ctr[4] = {draw, (uint32_t)iter, (uint32_t)slot, 0u}, r[4];
    ++draw;
    orc_philox4x32_10(ctr, key, r);
    double u1 = orc_u01(r[0], r[1]);
    double u2 = orc_u01(r[2], r[3]);
    double dt = -log(u1) / a0;
    double tn = t + dt;
    if (tn > cfg->tau) break;
    if (ev >= cap) { status = ORC_ESTEPCAP; break; }
    double target = u2 * a0;
    int32_t k = 1;
    while (k < P) {
      double L = node[2 * k], R = node[2 * k + 1];
      if (R == 0.0 || target < L) k = 2 * k;
      else { target = target - L; k = 2 * k + 1; }
    }
    const int32_t j = k - P;
    int over = 0;
    for (int32_t e = n->d_ptr[j]; e < n->d_ptr[j + 1]; ++e)
      if ((int64_t)x[n->d_sp[e]] + n->d_val[e] > ORC_MAX_COUNT) over = 1;
    if (over) { status = ORC_EOVERFLOW; break; }
    for (int32_t e = n->d_ptr[j]; e < n->d_ptr[j + 1]; ++e) x[n->d_sp[e]] += n->d_val[e];
    ++ev;
    t = tn;
    if ((cfg->feedback == 1 || cfg->feedback == 2) && in_target(cfg, x)) {
      ++rec;
      if (cfg->feedback == 2) break;
      memcpy(x, cfg->recycle_state, sizeof(int32_t) * S);
      DG_REBUILD();
      continue;
    }
    for (int32_t q = g->dep_ptr[j]; q < g->dep_ptr[j + 1]; ++q) {
      const int32_t i = g->dep[q];
      node[P + i] = propensity_of(n, i, x);
      for (int32_t a = (P + i) >> 1; a >= 1; a >>= 1) node[a] = node[2 * a] + node[2 * a + 1];
    }
  }
#undef DG_REBUILD
  free(node);
  if (cfg->feedback == 3 && in_target(cfg, x)) {             /* checked at the interval's end */
    ++rec;
    memcpy(x, cfg->recycle_state, sizeof(int32_t) * S);
  }
  *n_ev = ev;
  *n_rec = rec;
  if (t_last) *t_last = t;
  return status;
}

int orc_we_run_dg(const orc_dg *g, const orc_we_config *cfg, orc_we_out *out) {
  if (cfg->reweight_period > 0) return out->status = ORC_EINVAL;
  return we_run_impl(g->n, g, cfg, out);
}
