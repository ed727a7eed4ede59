// we_kernels.cu -- the resampling side of a WE iteration and the bookkeeping around it.
//
//   k_scan_bins   per run: bin occupancy -> task list, grouping cursors and output offsets
//   k_place       group each run's walkers by bin
//   k_resample    one warp per occupied bin: merge / split (Sec. II.B)
//   k_gather      copy species counts of the new ensemble from their parents
//   k_finalize    per-run counts and offsets, iteration counter
//   k_resample_run  runs whose walker lists fit in shared memory: the grouping and the
//                 split/merge of k_scan_bins + k_place + k_resample in one launch
//
// Every weight operation is a single IEEE double operation with an explicit round-to-nearest
// intrinsic; comparisons between non-negative doubles use their bit patterns.
#include "we_exact.cuh"
#include "we_ssa_common.cuh"

namespace we {

// ------------------------------------------------------------------------------------------
// Per run (one block): exclusive scans of bin counts and of bin occupancy give, for every
// occupied bin, where its walkers go when grouped by bin (in_offset) and where its M_targ
// resampled walkers go in the new ensemble (out_offset = M_targ * occupied bins before it).
// ------------------------------------------------------------------------------------------
// One block: exclusive scans over the bins, in bin order, of the counts c_b and of the
// occupancy [c_b > 0].  count_of(b) gives c_b; emit(b, c_b, walkers before b, occupied bins
// before b) is called once per bin by the thread that read it.  Returns (walkers, occupied bins).
template <typename CountOf, typename Emit>
__device__ __forceinline__ int2 scan_bins_block(int n_bins, CountOf count_of, Emit emit) {
  const int tid = threadIdx.x, B = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = B >> 5;
  __shared__ int s_cnt[32], s_occ[32];
  __shared__ int s_base_cnt, s_base_occ;
  if (tid == 0) { s_base_cnt = 0; s_base_occ = 0; }
  __syncthreads();
  for (int base = 0; base < n_bins; base += B) {
    const int b = base + tid;
    const int c = b < n_bins ? count_of(b) : 0;
    const int o = c > 0 ? 1 : 0;
    int ic = c, io = o;                                   // inclusive warp scans
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const int yc = __shfl_up_sync(0xffffffffu, ic, d);
      const int yo = __shfl_up_sync(0xffffffffu, io, d);
      if (lane >= d) { ic += yc; io += yo; }
    }
    if (lane == 31) { s_cnt[wid] = ic; s_occ[wid] = io; }
    __syncthreads();
    if (wid == 0) {
      int vc = lane < nw ? s_cnt[lane] : 0, vo = lane < nw ? s_occ[lane] : 0;
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const int yc = __shfl_up_sync(0xffffffffu, vc, d);
        const int yo = __shfl_up_sync(0xffffffffu, vo, d);
        if (lane >= d) { vc += yc; vo += yo; }
      }
      if (lane < nw) { s_cnt[lane] = vc; s_occ[lane] = vo; }
    }
    __syncthreads();
    const int wc = wid ? s_cnt[wid - 1] : 0, wo = wid ? s_occ[wid - 1] : 0;
    if (b < n_bins) emit(b, c, s_base_cnt + wc + ic - c, s_base_occ + wo + io - o);
    __syncthreads();
    if (tid == 0) { s_base_cnt += s_cnt[nw - 1]; s_base_occ += s_occ[nw - 1]; }
    __syncthreads();
  }
  return make_int2(s_base_cnt, s_base_occ);
}

__global__ void k_scan_bins(EnsView E, int n_bins) {
  const int r = blockIdx.x;
  int *bc = E.bin_count + (size_t)r * n_bins;
  int4 *tasks = E.tasks + (size_t)r * n_bins;
  int *cursor = E.cursor + (size_t)r * n_bins;
  const int M = E.m_targ;
  const int2 tot = scan_bins_block(n_bins, [&](int b) { return bc[b]; },
                                   [&](int b, int c, int ex_c, int ex_o) {
                                     if (c > 0) {
                                       tasks[ex_o] = make_int4(b, ex_c, c, ex_o * M);
                                       cursor[b] = ex_c;
                                     }
                                     bc[b] = 0;           // ready for the next interval
                                   });
  if (threadIdx.x == 0) {
    E.n_tasks[r] = tot.y;
    if ((long long)tot.y * M > E.cap) atomicCAS(&E.status[r], 0, kStatusOverflow);
  }
}

// Walkers of every run grouped by bin: each live walker takes the next free position of its
// bin (positions start at the bin's in_offset).  The order inside a bin is arbitrary; every
// later decision is keyed by the walker's slot, never by its position.
__global__ void k_place(EnsView E, int n_bins) {
  const int iter = *E.iter;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ld; g += gridDim.x * blockDim.x) {
    const int r = g / E.cap, w = g - r * E.cap;
    if (w >= E.count[r]) continue;
    const int b = E.bin[g];
    const int pos = atomicAdd(&E.cursor[(size_t)r * n_bins + b], 1);
    const size_t q = (size_t)r * E.cap + pos;
    E.sorted_slot[q] = w;
    E.sorted_w[q] = E.w[par][g];
    E.alive[q] = 1;
  }
}

// Warp argmin over the live entries of a bin list, keyed by (weight bits, slot).
__device__ __forceinline__ void warp_argmin(const double *sw, const int32_t *ss, const int32_t *al,
                                            int cnt, int exclude, int &best_i) {
  const int lane = threadIdx.x & 31;
  long long bw = 0x7FFFFFFFFFFFFFFFll;
  int bs = 0x7FFFFFFF, bi = -1;
  for (int i = lane; i < cnt; i += 32) {
    if (!al[i] || i == exclude) continue;
    const long long v = bits(sw[i]);
    const int sl = ss[i];
    if (v < bw || (v == bw && sl < bs)) { bw = v; bs = sl; bi = i; }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const long long ow = __shfl_xor_sync(0xffffffffu, bw, d);
    const int os = __shfl_xor_sync(0xffffffffu, bs, d);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, d);
    if (ow < bw || (ow == bw && os < bs)) { bw = ow; bs = os; bi = oi; }
  }
  best_i = bi;
}

// Four per-lane values as named registers (entries lane * 4 + q).  Selecting by a run-time q
// goes through selects; an array here would be turned into indexed local memory.
template <typename T>
struct Four {
  T v0, v1, v2, v3;
  __device__ __forceinline__ T get(int q) const { return q < 2 ? (q == 0 ? v0 : v1) : (q == 2 ? v2 : v3); }
  __device__ __forceinline__ void set(int q, T x) {
    v0 = q == 0 ? x : v0; v1 = q == 1 ? x : v1; v2 = q == 2 ? x : v2; v3 = q == 3 ? x : v3;
  }
};

// (w, s) lexicographic order on (weight bits, slot)
__device__ __forceinline__ bool key_lt(long long wa, int sa, long long wb, int sb) {
  return wa < wb || (wa == wb && sa < sb);
}

// ------------------------------------------------------------------------------------------
// Split/merge, one warp per occupied bin (Sec. II.B).  A bin's walkers are ordered by slot:
//   more than M_targ: merge the two lightest (ties: lower slot); of the pair, the lower-slot
//     walker p survives iff u < w_p/(w_p+w_q), u from Philox counter (k, iter, bin, 1) with k
//     the merge index, and takes the summed weight; repeat;
//   fewer than M_targ: give the next copy to the walker with the largest w_i/c_i (ties: lower
//     slot), until M_targ copies; each copy carries w_i/c_i.
// The resampled walkers are written in slot order, copies right after their parent, at the
// bin's output offset.
// ------------------------------------------------------------------------------------------
// Per-run constants of the split/merge.
struct ResampleCtx {
  int iter, par, M, slot_obs;
  size_t base;
  double *W2;
  int32_t *P2;
  uint32_t k0, k1;
  const unsigned long long *magic;
};

__device__ __forceinline__ ResampleCtx resample_ctx(const EnsView &E, int r) {
  ResampleCtx c;
  c.iter = *E.iter;
  c.par = c.iter & 1;
  c.M = E.m_targ;
  c.slot_obs = c.iter - E.first_iter;
  c.base = (size_t)r * E.cap;
  c.W2 = E.w[c.par ^ 1] + c.base;
  c.P2 = E.parent[c.par ^ 1] + c.base;
  c.k0 = (uint32_t)E.seed;
  c.k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  c.magic = E.div_magic;
  return c;
}

// Networks of up to kGatherInResample species have their species counts copied by the
// split/merge warps; larger ones by k_gather, whose loads are coalesced across walkers.
constexpr int kGatherInResample = 8;

// u < fl(w_p / s) for the merge's survivor, s = fl(w_p + w_q) (u, w_p, s as bits of positive
// doubles, u < 1): screened in FP32 first (settles all but the draws within about 2^-19 of the
// quotient), then the exact integer test, or the FP64 quotient where weights are too small for it.
__device__ __forceinline__ bool survivor_keeps(unsigned long long u, unsigned long long wp, unsigned long long s,
                                               bool exact) {
  const int f = ex_u_below_quotient_f32(u, wp, s);
  if (f >= 0) return f != 0;
  return exact ? ex_u_below_quotient(u, wp, s)
               : u < (unsigned long long)bits(__ddiv_rn(__longlong_as_double((long long)wp),
                                                        __longlong_as_double((long long)s)));
}

// Per-warp shared scratch of the queue form of the merges (bins of up to 128 walkers): the bin's
// walkers sorted by (weight, slot), and the merged walkers in the order of their keys.
constexpr int kQueueMax = 128;
struct MergeQueues {
  long long aw[kQueueMax];
  int32_t as[kQueueMax], ai[kQueueMax];
  long long qw[kQueueMax];
  int32_t qs[kQueueMax], qi[kQueueMax];
};

// The split/merge of one occupied bin by one warp: tk = (bin, -, cnt, output offset); lss, lsw,
// lal hold the bin's cnt walkers (slot, weight, copies) in any order, in global or shared
// memory, and are overwritten.  With kQueue (lists in shared memory, mq the warp's scratch) the
// merges of bins of up to 128 walkers take the queue form below.
template <bool kQueue>
__device__ __forceinline__ void resample_bin(const EnsView &E, int r, const ResampleCtx &cx, int4 tk,
                                             int32_t *lss, double *lsw, int32_t *lal, int gather,
                                             MergeQueues *mq) {
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const int iter = cx.iter, par = cx.par, M = cx.M, slot_obs = cx.slot_obs;
  const size_t base = cx.base;
  double *W2 = cx.W2;
  int32_t *P2 = cx.P2;
  const uint32_t k0 = cx.k0, k1 = cx.k1;
  const unsigned long long *magic = cx.magic;
  const int b = tk.x, cnt = tk.z, out0 = tk.w;
  if (out0 + M > E.cap) return;                          // capacity overflow, already flagged

  // Register form: up to 128 walkers (entries i = lane + 32 q as index lane * 4 + q), weights
  // as bits.  The integer split/merge decisions need normal weights (w >= 2^-999 keeps every
  // quotient normal) and copy counts up to 2048; other bins take the floating-point path.
  Four<long long> vv;
  Four<int> sl;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = lane + 32 * q;
    vv.set(q, i < cnt ? bits(lsw[i]) : -1ll);
    sl.set(q, i < cnt ? lss[i] : 0x7FFFFFFF);
  }
  bool exact = magic != nullptr && cnt <= 128 && M <= 2048;
  if (exact) {
    bool small = false;
#pragma unroll
    for (int q = 0; q < 4; ++q) small = small || (vv.get(q) >= 0 && (vv.get(q) >> 52) < 24);
    exact = !__any_sync(0xffffffffu, small);
  }

  if (kQueue && cnt > M && cnt <= kQueueMax) {
    // Merges, queue form.  The bin's walkers are sorted once by (weight, slot); merged walkers
    // join a second list that stays in key order, because each merged weight is at least the
    // previous one (the two lightest are merged, and every other walker weighs at least the
    // heavier of them, so the next pair sums to at least as much; rounding to nearest keeps the
    // order), so only a merged walker of equal weight and lower slot moves ahead of another.
    // The two lightest live walkers are then always among the heads of the two lists: the same
    // pairs, uniforms, survivor decisions (exact integer test, or the FP64 quotient where the
    // weights are not all normal) and weights as the forms below.  Every lane runs the loop on
    // the same values; lane 0 writes.
    Four<unsigned long long> ub;
    const int n_merge = cnt - M;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      unsigned long long u = 0;
      if (i < n_merge) {
        uint32_t c0 = (uint32_t)i, c1 = (uint32_t)iter, c2 = (uint32_t)b, c3 = 1u;
        philox4x32_10(c0, c1, c2, c3, k0, k1);
        u = (unsigned long long)bits(u01(c0, c1));
      }
      ub.set(q, u);
    }
    Four<int> rk;
#pragma unroll
    for (int q = 0; q < 4; ++q) rk.set(q, 0);
    for (int j = 0; j < cnt; ++j) {                       // ranks by (weight, slot): all distinct
      const long long vj = bits(lsw[j]);
      const int sj = lss[j];
#pragma unroll
      for (int q = 0; q < 4; ++q) rk.set(q, rk.get(q) + (key_lt(vj, sj, vv.get(q), sl.get(q)) ? 1 : 0));
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      if (i < cnt) { mq->aw[rk.get(q)] = vv.get(q); mq->as[rk.get(q)] = sl.get(q); mq->ai[rk.get(q)] = i; }
    }
    __syncwarp();
    int ia = 0, qh = 0, qt = 0;
    long long aw = mq->aw[0], qw = 0, tw = 0;               // tw, ts: key of the merged list's tail
    int as = mq->as[0], ai = mq->ai[0], qs = 0, qi = 0, ts = 0;
    auto pop = [&](long long &w, int &sl_, int &ix) {
      const bool from_a = ia < cnt && (qh >= qt || key_lt(aw, as, qw, qs));
      if (from_a) {
        w = aw; sl_ = as; ix = ai;
        if (++ia < cnt) { aw = mq->aw[ia]; as = mq->as[ia]; ai = mq->ai[ia]; }
      } else {
        w = qw; sl_ = qs; ix = qi;
        if (++qh < qt) { qw = mq->qw[qh]; qs = mq->qs[qh]; qi = mq->qi[qh]; }
      }
    };
    for (int km = 0; km < n_merge; ++km) {
      long long w1, w2;
      int s1, s2, i1, i2;
      pop(w1, s1, i1);
      pop(w2, s2, i2);
      const bool a_first = s1 < s2;                          // p: the lower slot of the pair
      const long long wp = a_first ? w1 : w2, wq = a_first ? w2 : w1;
      const int sp = a_first ? s1 : s2, sq = a_first ? s2 : s1;
      const int ip = a_first ? i1 : i2, iq = a_first ? i2 : i1;
      const unsigned long long u_k = __shfl_sync(0xffffffffu, ub.get(km >> 5), km & 31);
      const double wsum = __dadd_rn(__longlong_as_double(wp), __longlong_as_double(wq));
      const bool keep_p = survivor_keeps(u_k, (unsigned long long)wp, (unsigned long long)bits(wsum), exact);
      const long long nw = bits(wsum);
      const int ns = keep_p ? sp : sq, ni = keep_p ? ip : iq;
      int pos = qt;
      const bool behind = qt > qh && key_lt(nw, ns, tw, ts);  // equal weight, lower slot than the tail
      if (!behind) { tw = nw; ts = ns; }
      while (behind && pos > qh && key_lt(nw, ns, mq->qw[pos - 1], mq->qs[pos - 1])) {
        const long long mw = mq->qw[pos - 1];
        const int ms_ = mq->qs[pos - 1], mi = mq->qi[pos - 1];
        __syncwarp();
        if (lane == 0) { mq->qw[pos] = mw; mq->qs[pos] = ms_; mq->qi[pos] = mi; }
        __syncwarp();
        --pos;
      }
      if (lane == 0) { mq->qw[pos] = nw; mq->qs[pos] = ns; mq->qi[pos] = ni; }
      __syncwarp();
      ++qt;
      if (pos == qh) { qw = nw; qs = ns; qi = ni; }
    }
    // survivors: the rest of the sorted list (weights unchanged) and of the merged list
    for (int i = lane; i < cnt; i += 32) lal[i] = 0;
    __syncwarp();
    for (int t = ia + lane; t < cnt; t += 32) lal[mq->ai[t]] = 1;
    for (int t = qh + lane; t < qt; t += 32) {
      const int ix = mq->qi[t];
      lal[ix] = 1;
      lsw[ix] = __longlong_as_double(mq->qw[t]);
    }
    __syncwarp();
  } else if (!kQueue && cnt > M && exact) {               // (with kQueue the queue form takes these)
    // Merges.  Every merge's uniform is drawn up front (merge k's counter does not depend on
    // the others); each merge takes the two lightest live entries by (weight, slot) from one
    // branch-free shuffle reduction; the survivor decision is the integer form of
    // u < w_p / (w_p + w_q).
    Four<unsigned long long> ub;
    const int n_merge = cnt - M;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      unsigned long long u = 0;
      if (i < n_merge) {
        uint32_t c0 = (uint32_t)i, c1 = (uint32_t)iter, c2 = (uint32_t)b, c3 = 1u;
        philox4x32_10(c0, c1, c2, c3, k0, k1);
        u = (unsigned long long)bits(u01(c0, c1));
      }
      ub.set(q, u);
    }
    for (int km = 0; km < n_merge; ++km) {
      long long w1 = 0x7FFFFFFFFFFFFFFFll, w2 = 0x7FFFFFFFFFFFFFFFll;
      int s1 = 0x7FFFFFFF, s2 = 0x7FFFFFFF, o1 = -1, o2 = -1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long v = vv.get(q);
        const int sq = sl.get(q), oq = lane * 4 + q;
        const bool live = v >= 0;
        const bool lt1 = live && key_lt(v, sq, w1, s1);
        const bool lt2 = live && key_lt(v, sq, w2, s2);
        w2 = lt1 ? w1 : (lt2 ? v : w2);
        s2 = lt1 ? s1 : (lt2 ? sq : s2);
        o2 = lt1 ? o1 : (lt2 ? oq : o2);
        w1 = lt1 ? v : w1; s1 = lt1 ? sq : s1; o1 = lt1 ? oq : o1;
      }
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        const long long pw1 = __shfl_xor_sync(0xffffffffu, w1, d), pw2 = __shfl_xor_sync(0xffffffffu, w2, d);
        const int ps1 = __shfl_xor_sync(0xffffffffu, s1, d), ps2 = __shfl_xor_sync(0xffffffffu, s2, d);
        const int po1 = __shfl_xor_sync(0xffffffffu, o1, d), po2 = __shfl_xor_sync(0xffffffffu, o2, d);
        // the lighter of the two firsts leads; the second is the lighter of the other first
        // and the leader's own second
        const bool plead = key_lt(pw1, ps1, w1, s1);
        const long long cw = plead ? w1 : pw1, dw = plead ? pw2 : w2;
        const int cs = plead ? s1 : ps1, ds = plead ? ps2 : s2;
        const int co = plead ? o1 : po1, dob = plead ? po2 : o2;
        const bool clt = key_lt(cw, cs, dw, ds);
        w2 = clt ? cw : dw; s2 = clt ? cs : ds; o2 = clt ? co : dob;
        w1 = plead ? pw1 : w1; s1 = plead ? ps1 : s1; o1 = plead ? po1 : o1;
      }
      const bool a_first = s1 < s2;                        // p: the lower slot of the pair
      const long long wp = a_first ? w1 : w2, wq = a_first ? w2 : w1;
      const int op = a_first ? o1 : o2, oq = a_first ? o2 : o1;
      const unsigned long long u_k = __shfl_sync(0xffffffffu, ub.get(km >> 5), km & 31);
      const double wsum = __dadd_rn(__longlong_as_double(wp), __longlong_as_double(wq));
      const bool keep_p = survivor_keeps(u_k, (unsigned long long)wp, (unsigned long long)bits(wsum), true);
      const int osurv = keep_p ? op : oq, odead = keep_p ? oq : op;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        long long v = vv.get(q);
        v = lane * 4 + q == osurv ? bits(wsum) : v;
        v = lane * 4 + q == odead ? -1ll : v;
        vv.set(q, v);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      const long long v = vv.get(q);
      if (i < cnt) { lal[i] = v >= 0 ? 1 : 0; if (v >= 0) lsw[i] = __longlong_as_double(v); }
    }
    __syncwarp();
  } else if (cnt > M) {
    uint32_t kmerge = 0;
    for (int live = cnt; live > M; --live) {
      int ia, ib;
      warp_argmin(lsw, lss, lal, cnt, -1, ia);
      warp_argmin(lsw, lss, lal, cnt, ia, ib);
      if (lane == 0) {
        const bool a_first = lss[ia] < lss[ib];
        const int p = a_first ? ia : ib, q = a_first ? ib : ia;
        uint32_t c0 = kmerge, c1 = (uint32_t)iter, c2 = (uint32_t)b, c3 = 1u;
        philox4x32_10(c0, c1, c2, c3, k0, k1);
        const double u = u01(c0, c1);
        const double wsum = __dadd_rn(lsw[p], lsw[q]);
        const double prob = __ddiv_rn(lsw[p], wsum);
        if (bits(u) < bits(prob)) { lsw[p] = wsum; lal[q] = 0; }
        else { lsw[q] = wsum; lal[p] = 0; }
      }
      ++kmerge;
      __syncwarp();
    }
  } else if (cnt == 1 && M > 1) {
    if (lane == 0) lal[0] = M;                            // every copy goes to the one walker
    __syncwarp();
  } else if (kQueue && cnt < M && cnt <= 32) {
    // Splits, sorted form (bins of up to 32 walkers): lane k holds the walker of rank k by
    // (per-copy weight desc, slot asc); each round gives the next copy to lane 0's walker, whose
    // per-copy weight becomes fl(w / c) for its new copy count c (exact integer division, or
    // FP64 division where the weights are not all normal), and moves it down to its new rank
    // (one ballot, one shift).  The same receivers in the same order as the argmax rounds
    // below, so the same copy counts.
    const unsigned full = 0xffffffffu;
    const bool own = lane < cnt;
    long long v = vv.get(0);                                // entry i = lane (cnt <= 32)
    int s_ = sl.get(0), ix = lane, c = own ? 1 : 0;
    int rank = 0;
    for (int j = 0; j < cnt; ++j) {
      const long long vj = __shfl_sync(full, v, j);
      const int sj = __shfl_sync(full, s_, j);
      rank += (vj > v || (vj == v && sj < s_)) ? 1 : 0;
    }
    if (own) { mq->aw[rank] = v; mq->as[rank] = s_; mq->ai[rank] = ix; }
    __syncwarp();
    if (own) { v = mq->aw[lane]; s_ = mq->as[lane]; ix = mq->ai[lane]; }
    long long wo = v;                                       // every walker starts with one copy
    __syncwarp();
    for (int extra = cnt; extra < M; ++extra) {
      const long long w0 = __shfl_sync(full, wo, 0);
      const int c0 = __shfl_sync(full, c, 0) + 1;
      const int s0 = __shfl_sync(full, s_, 0), i0 = __shfl_sync(full, ix, 0);
      const long long v0 = exact ? (long long)ex_div_small((unsigned long long)w0, (unsigned)c0, magic[c0])
                                 : bits(__ddiv_rn(__longlong_as_double(w0), (double)c0));
      const bool above = lane >= 1 && own && (v > v0 || (v == v0 && s_ < s0));
      const int p = __popc(__ballot_sync(full, above));      // walkers that stay ahead of it
      const long long vn = __shfl_down_sync(full, v, 1), wn = __shfl_down_sync(full, wo, 1);
      const int sn = __shfl_down_sync(full, s_, 1), cn = __shfl_down_sync(full, c, 1);
      const int xn = __shfl_down_sync(full, ix, 1);
      if (lane < p) { v = vn; wo = wn; s_ = sn; c = cn; ix = xn; }
      else if (lane == p) { v = v0; wo = w0; s_ = s0; c = c0; ix = i0; }
    }
    if (own) lal[ix] = c;
    __syncwarp();
  } else if (cnt < M && exact) {
    // Splits: the next copy to the largest per-copy weight fl(w_i / c_i) (ties: lower slot);
    // each entry keeps the value it would have after one more copy (nv), so a round is one
    // branch-free argmax and one integer division by the lane that holds the receiver.
    Four<unsigned long long> wo, nv;
    Four<int> cc;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const long long v = vv.get(q);
      wo.set(q, (unsigned long long)v);
      cc.set(q, v >= 0 ? 1 : 0);
      nv.set(q, v >= 0 ? ex_div_small((unsigned long long)v, 2u, magic[2]) : 0ull);
    }
    for (int extra = cnt; extra < M; ++extra) {
      long long bv = -1;
      int bs = 0x7FFFFFFF, bo = -1;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const long long v = vv.get(q);
        const int sq = sl.get(q);
        const bool gt = v > bv || (v == bv && sq < bs);
        bv = gt ? v : bv; bs = gt ? sq : bs; bo = gt ? lane * 4 + q : bo;
      }
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, d);
        const int os = __shfl_xor_sync(0xffffffffu, bs, d);
        const int oo = __shfl_xor_sync(0xffffffffu, bo, d);
        const bool gt = ov > bv || (ov == bv && os < bs);
        bv = gt ? ov : bv; bs = gt ? os : bs; bo = gt ? oo : bo;
      }
      if ((bo >> 2) == lane) {
        const int q = bo & 3;
        const int c = cc.get(q) + 1;
        cc.set(q, c);
        vv.set(q, (long long)nv.get(q));
        nv.set(q, c + 1 <= M ? ex_div_small(wo.get(q), (unsigned)(c + 1), magic[c + 1]) : 0ull);
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = lane + 32 * q;
      if (i < cnt) lal[i] = cc.get(q);
    }
    __syncwarp();
  } else if (cnt < M) {
    for (int extra = cnt; extra < M; ++extra) {
      long long bv = -1;
      int bs = 0x7FFFFFFF, bi = -1;
      for (int i = lane; i < cnt; i += 32) {
        const long long v = bits(__ddiv_rn(lsw[i], (double)lal[i]));
        const int sli = lss[i];
        if (v > bv || (v == bv && sli < bs)) { bv = v; bs = sli; bi = i; }
      }
#pragma unroll
      for (int d = 16; d >= 1; d >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, d);
        const int os = __shfl_xor_sync(0xffffffffu, bs, d);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, d);
        if (ov > bv || (ov == bv && os < bs)) { bv = ov; bs = os; bi = oi; }
      }
      if (lane == 0) lal[bi] += 1;
      __syncwarp();
    }
  }
  // Compact the surviving entries (copies > 0) to the front of the list, order kept.
  int k = 0;
  for (int i0 = 0; i0 < cnt; i0 += 32) {
    const int i = i0 + lane;
    int sli = 0, c = 0;
    double wv = 0.0;
    if (i < cnt) { sli = lss[i]; c = lal[i]; wv = lsw[i]; }
    const unsigned m = __ballot_sync(0xffffffffu, c > 0);
    __syncwarp();
    if (c > 0) {
      const int d = k + __popc(m & lt_mask);
      lss[d] = sli; lal[d] = c; lsw[d] = wv;
    }
    k += __popc(m);
    __syncwarp();
  }
  // Output offset of each survivor: copies of all survivors with a lower slot.
  double wsum_local = 0.0;
  const int ld = E.R * E.cap;
  for (int i = lane; i < k; i += 32) {
    const int si = lss[i];
    int32_t xv[kGatherInResample];                        // the walker's species counts, loaded
#pragma unroll                                            // ahead of the offset sum
    for (int sp = 0; sp < kGatherInResample; ++sp)
      xv[sp] = (gather && sp < E.S) ? E.x[par][(size_t)sp * ld + base + si] : 0;
    int off = 0;
    for (int j = 0; j < k; ++j) off += (lss[j] < si) ? lal[j] : 0;
    const int c = lal[i];
    const double wi = lsw[i];
    double wc = wi;
    if (cnt < M && c > 1)
      wc = exact ? __longlong_as_double((long long)ex_div_small((unsigned long long)bits(wi), (unsigned)c, magic[c]))
                 : __ddiv_rn(wi, (double)c);
    for (int q = 0; q < c; ++q) {
      W2[out0 + off + q] = wc;
      P2[out0 + off + q] = si;
    }
    if (gather) {                                         // the copies' species counts
#pragma unroll
      for (int sp = 0; sp < kGatherInResample; ++sp)
        if (sp < E.S)
          for (int q = 0; q < c; ++q) E.x[par ^ 1][(size_t)sp * ld + base + out0 + off + q] = xv[sp];
    }
    // the c copies' weight, c * wc rounded once (the exact sum of the copies, rounded)
    wsum_local = __dadd_rn(wsum_local, c == 1 ? wc : __dmul_rn((double)c, wc));
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) wsum_local = __dadd_rn(wsum_local, __shfl_xor_sync(0xffffffffu, wsum_local, d));
  if (lane == 0 && slot_obs >= 0 && slot_obs < E.record_iters)
    atomicAdd(&E.obs_totw[slot_obs * E.R + r], wsum_local);
  __syncwarp();
}

__global__ void __launch_bounds__(128, 4) k_resample(EnsView E, int n_bins, int gather) {
  const int r = blockIdx.y;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  const int nt = E.n_tasks[r];
  const ResampleCtx cx = resample_ctx(E, r);
  for (int t = warp; t < nt; t += n_warps) {
    const int4 tk = E.tasks[(size_t)r * n_bins + t];
    const size_t q = cx.base + tk.y;
    resample_bin<false>(E, r, cx, tk, E.sorted_slot + q, E.sorted_w + q, E.alive + q, gather, nullptr);
  }
}

// ------------------------------------------------------------------------------------------
// Runs whose walker lists fit in shared memory: the grouping by bin and the split/merge in one
// launch.  G blocks serve a run.  Each block counts and scans the run's bins itself (no block
// waits for another), keeps the occupied bins whose task index is j mod G, groups only their
// walkers into its shared-memory lists, and splits/merges them, one warp per bin, the warps
// taking the block's bins in task order.  Decisions and output are those of k_scan_bins +
// k_place + k_resample: the order of a bin's list is arbitrary in both, and every decision is
// keyed by (weight, slot).  Block 0 of a run also publishes the run's task list (read by the
// reweighting), its task count and overflow status, and clears the run's bin counts (which the
// SSA epilogue accumulates for k_scan_bins).
// ------------------------------------------------------------------------------------------
constexpr int kRunThreads = 512;

__global__ void __launch_bounds__(kRunThreads, 1) k_resample_run(EnsView E, int n_bins) {
  extern __shared__ __align__(16) unsigned char smem_run[];
  const int r = blockIdx.y, j = blockIdx.x, G = gridDim.x;
  const int tid = threadIdx.x, B = blockDim.x, lane = tid & 31;
  const int cap = E.cap, M = E.m_targ;
  MergeQueues *mq = reinterpret_cast<MergeQueues *>(smem_run);         // one per warp
  unsigned long long *s_magic = reinterpret_cast<unsigned long long *>(mq + kRunThreads / 32);  // M + 1
  int4 *s_task = reinterpret_cast<int4 *>(s_magic + ((M + 2) & ~1));   // n_bins
  double *s_w = reinterpret_cast<double *>(s_task + n_bins);           // cap
  int32_t *s_slot = reinterpret_cast<int32_t *>(s_w + cap);            // cap
  int32_t *s_alive = s_slot + cap;                                     // cap
  int *s_cur = s_alive + cap;                                          // n_bins: counts, then cursors
  int *s_tob = s_cur + n_bins;                                         // n_bins: task index of each bin
  __shared__ int s_next;
  ResampleCtx cx = resample_ctx(E, r);
  // the exact division's reciprocals, read once per split round: from shared memory
  if (cx.magic) {
    for (int c = tid; c <= M; c += B) s_magic[c] = cx.magic[c];
    cx.magic = s_magic;
  }
  const int n = E.count[r];
  const int32_t *bin = E.bin + cx.base;
  for (int b = tid; b < n_bins; b += B) s_cur[b] = 0;
  __syncthreads();
  for (int w = tid; w < n; w += B) atomicAdd(&s_cur[bin[w]], 1);
  __syncthreads();
  const int2 tot = scan_bins_block(n_bins, [&](int b) { return s_cur[b]; },
                                   [&](int b, int c, int ex_c, int ex_o) {
                                     s_tob[b] = c > 0 ? ex_o : -1;
                                     if (c > 0) s_task[ex_o] = make_int4(b, ex_c, c, ex_o * M);
                                     s_cur[b] = ex_c;
                                   });
  const int nt = tot.y;
  if (j == 0) {
    int4 *tasks = E.tasks + (size_t)r * n_bins;
    int *bc = E.bin_count + (size_t)r * n_bins;
    for (int t = tid; t < nt; t += B) tasks[t] = s_task[t];
    for (int b = tid; b < n_bins; b += B) bc[b] = 0;
    if (tid == 0) {
      E.n_tasks[r] = nt;
      if ((long long)nt * M > cap) atomicCAS(&E.status[r], 0, kStatusOverflow);
    }
  }
  const double *w_in = E.w[cx.par] + cx.base;
  for (int w = tid; w < n; w += B) {
    const int b = bin[w];
    if (s_tob[b] % G != j) continue;
    const int pos = atomicAdd(&s_cur[b], 1);
    s_slot[pos] = w;
    s_w[pos] = w_in[w];
    s_alive[pos] = 1;
  }
  if (tid == 0) s_next = j;
  __syncthreads();
  for (;;) {
    int t = 0;
    if (lane == 0) t = atomicAdd(&s_next, G);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= nt) break;
    const int4 tk = s_task[t];
    resample_bin<true>(E, r, cx, tk, s_slot + tk.y, s_w + tk.y, s_alive + tk.y, 1, mq + (tid >> 5));
  }
}

// New counts of every run: M_targ per occupied bin (resampling) or unchanged (plain SSA).
__device__ __forceinline__ int new_count(const EnsView &E, int r, int resample) {
  if (!resample) return E.count[r];
  const long long c = (long long)E.n_tasks[r] * E.m_targ;
  return c > E.cap ? E.cap : (int)c;
}

// Species counts of the new ensemble, gathered from each walker's parent.  With plain SSA the
// parent is the walker itself and its weight is carried over.
__global__ void k_gather(EnsView E, int resample) {
  const int iter = *E.iter;
  const int par = iter & 1;
  const int ld = E.R * E.cap;
  for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < ld; g += gridDim.x * blockDim.x) {
    const int r = g / E.cap, w = g - r * E.cap;
    if (w >= new_count(E, r, resample)) continue;
    int src = w;
    if (resample) src = E.parent[par ^ 1][g];
    else { E.parent[par ^ 1][g] = w; E.w[par ^ 1][g] = E.w[par][g]; }
    const int gs = r * E.cap + src;
    for (int s = 0; s < E.S; ++s) E.x[par ^ 1][(size_t)s * ld + g] = E.x[par][(size_t)s * ld + gs];
  }
}

// One block: counts, run offsets and the walker-count observable; advance the iteration.
__global__ void k_finalize(EnsView E, int resample) {
  __shared__ int s_new[1024], s_old[1024];
  const int iter = *E.iter;
  const int slot = iter - E.first_iter;
  for (int r = threadIdx.x; r < E.R; r += blockDim.x) {
    const int c = new_count(E, r, resample);
    if (r < 1024) { s_new[r] = c; s_old[r] = E.count[r]; }   // both loads in one round trip
    if (slot >= 0 && slot < E.record_iters) E.obs_nw[slot * E.R + r] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int r = 0; r < E.R; ++r) {
      const int c = r < 1024 ? s_new[r] : new_count(E, r, resample);
      E.run_off[r] = acc;
      acc += c;
    }
    E.run_off[E.R] = acc;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < E.R; r += blockDim.x) {
    const int c = r < 1024 ? s_new[r] : new_count(E, r, resample);
    E.prev_count[r] = r < 1024 ? s_old[r] : E.count[r];
    E.count[r] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) *E.iter = iter + 1;
}

// Walker-major copy of one run's counts (for output).
// Walker-major copy of the live walkers' counts: of run r, or (r < 0) of all runs in run order.
__global__ void k_pack_states(EnsView E, int r, int32_t *out) {
  const int iter = *E.iter;
  const int par = iter & 1;
  const long long n = r < 0 ? E.run_off[E.R] : E.count[r];
  const int ld = E.R * E.cap;
  for (long long i = blockIdx.x * blockDim.x + threadIdx.x; i < n * E.S; i += (long long)gridDim.x * blockDim.x) {
    const int f = (int)(i / E.S), s = (int)(i - (long long)f * E.S);
    int rr = r, w = f;
    if (r < 0) {
      rr = E.R == 1 ? 0 : find_run(E.run_off, E.R, f);
      w = f - E.run_off[rr];
    }
    out[i] = E.x[par][(size_t)s * ld + (size_t)rr * E.cap + w];
  }
}

// ------------------------------------------------------------------------------------------
// Host-side launch helpers (called from we_host.cu).
// ------------------------------------------------------------------------------------------
bool gather_in_resample(const EnsView &E) { return E.S <= kGatherInResample && E.x[0] != nullptr; }

cudaError_t launch_resample_chain(const PropagateParams &prm, cudaStream_t st) {
  const EnsView &E = prm.ens;
  const int nb = prm.bins.n_bins;
  k_scan_bins<<<E.R, 256, 0, st>>>(E, nb);
  const int ld = E.R * E.cap;
  int pgrid = (ld + 255) / 256;
  if (pgrid > 152 * 8) pgrid = 152 * 8;
  k_place<<<pgrid, 256, 0, st>>>(E, nb);
  int per_run_tasks = nb < E.cap ? nb : E.cap;
  int bx = (per_run_tasks + 3) / 4;                 // 4 warps per block
  if (bx > 64) bx = 64;
  if (bx < 1) bx = 1;
  k_resample<<<dim3(bx, E.R), 128, 0, st>>>(E, nb, gather_in_resample(E) ? 1 : 0);
  return cudaGetLastError();
}

// Shared memory of k_resample_run for this ensemble (the warps' merge queues, the division
// reciprocals, task list, the three walker lists, bin cursors and task indices), or 0 when its runs do not fit or the split/merge does not gather.
size_t resample_run_smem(const EnsView &E, int n_bins) {
  if (!gather_in_resample(E) || n_bins < 1 || E.cap < 1) return 0;
  const size_t bytes = (kRunThreads / 32) * sizeof(MergeQueues) + 8 * (size_t)((E.m_targ + 2) & ~1) +
                       24 * (size_t)n_bins + 16 * (size_t)E.cap;
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    optin = 48 * 1024;
  }
  const size_t static_bytes = 1024;                      // the scan's and the task counter's
  return bytes + static_bytes <= (size_t)optin ? bytes : 0;
}

// Let k_resample_run take up to the device's opt-in shared memory per block.  The limit is a
// per-function setting of the process, so it is set once to the largest value (no ensemble
// lowers another's); it does not change the occupancy of a launch that asks for less.
cudaError_t resample_run_prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  e = e ? e : cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  e = e ? e : cudaFuncGetAttributes(&fa, k_resample_run);
  e = e ? e : cudaFuncSetAttribute(k_resample_run, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   optin - (int)fa.sharedSizeBytes);
  return e;
}

// Blocks per run of k_resample_run: about one bin per two warps (at most 16 blocks), and no more
// than two blocks per SM over all runs.  Measured on GB300: the Schloegl MFPT grid (80 bins,
// 10 runs) 111.2 / 110.3 / 110.1 ms per step with 5 / 10 / 16 blocks per run; the birth-death
// grid (61 bins, 10 runs) 5.08 / 5.03 / 5.84 ms with 4 / 8 / 16.
int resample_run_blocks(int n_bins, int runs) {
  int dev = 0, sms = 152;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    sms = 152;
  }
  int g = (n_bins + 7) / 8;
  g = g > 16 ? 16 : g;
  const int by_sms = (2 * sms) / (runs > 0 ? runs : 1);
  g = g > by_sms ? by_sms : g;
  return g < 1 ? 1 : g;
}

cudaError_t launch_resample_run(const PropagateParams &prm, int blocks_per_run, cudaStream_t st) {
  const EnsView &E = prm.ens;
  const int nb = prm.bins.n_bins;
  const size_t smem = resample_run_smem(E, nb);
  if (!smem) return cudaErrorInvalidValue;
  const int G = blocks_per_run > 0 ? blocks_per_run : resample_run_blocks(nb, E.R);
  k_resample_run<<<dim3(G, E.R), kRunThreads, smem, st>>>(E, nb);
  return cudaGetLastError();
}

cudaError_t launch_gather_finalize(const PropagateParams &prm, cudaStream_t st) {
  const EnsView &E = prm.ens;
  if (!(prm.resample && gather_in_resample(E))) {
    const int ld = E.R * E.cap;
    int grid = (ld + 255) / 256;
    if (grid > 152 * 8) grid = 152 * 8;
    k_gather<<<grid, 256, 0, st>>>(E, prm.resample);
  }
  k_finalize<<<1, 256, 0, st>>>(E, prm.resample);
  return cudaGetLastError();
}

// Brute-force transition time (Sec. II.C, Eq. "mld") of every run of an absorbing ensemble:
// one block per run.  Thread t sums the first-passage times t_i in [0, T] of slots t, t + 256,
// ... in slot order, then the 256 partial sums are added in a fixed pairwise order, so the
// result does not depend on timing.  out[5 r ..] = (N, n, sum t_i, mu, sigma) with
// mu = (sum t_i + (N - n) T) / n and sigma = mu / sqrt(n) (+inf for both when n = 0).
__global__ void __launch_bounds__(256) k_fpt_mle(EnsView E, double T, double *out) {
  __shared__ double s_sum[256];
  __shared__ int s_n[256];
  const int r = blockIdx.x, t = threadIdx.x;
  const int N = E.count[r];
  const double Tr = T > 0.0 ? T : __dmul_rn((double)*E.iter, E.tau);
  const double *f = E.fpt + (size_t)r * E.cap;
  double sum = 0.0;
  int n = 0;
  for (int w = t; w < N; w += 256) {
    const double v = f[w];
    if (v >= 0.0 && v <= Tr) { sum = __dadd_rn(sum, v); ++n; }
  }
  s_sum[t] = sum;
  s_n[t] = n;
  __syncthreads();
  for (int h = 128; h >= 1; h >>= 1) {
    if (t < h) { s_sum[t] = __dadd_rn(s_sum[t], s_sum[t + h]); s_n[t] += s_n[t + h]; }
    __syncthreads();
  }
  if (t == 0) {
    const int nn = s_n[0];
    const double st = s_sum[0];
    double mu = __longlong_as_double(0x7ff0000000000000ll), sg = mu;
    if (nn > 0) {
      mu = __ddiv_rn(__dadd_rn(st, __dmul_rn((double)(N - nn), Tr)), (double)nn);
      sg = __ddiv_rn(mu, __dsqrt_rn((double)nn));
    }
    double *o = out + 5 * (size_t)r;
    o[0] = (double)N; o[1] = (double)nn; o[2] = st; o[3] = mu; o[4] = sg;
  }
}

cudaError_t launch_fpt_mle(const EnsView &E, double T, double *out, cudaStream_t st) {
  k_fpt_mle<<<E.R, 256, 0, st>>>(E, T, out);
  return cudaGetLastError();
}

cudaError_t launch_pack_states(const EnsView &E, int r, int32_t *out, cudaStream_t st) {
  k_pack_states<<<152, 256, 0, st>>>(E, r, out);
  return cudaGetLastError();
}

}  // namespace we
