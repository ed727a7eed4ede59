// we_kernels.cu -- the resampling side of a WE iteration and the bookkeeping around it.
//
//   k_scan_bins   per run: bin occupancy -> task list, grouping cursors and output offsets
//   k_place       group each run's walkers by bin
//   k_resample    one warp per occupied bin: merge / split (Sec. II.B)
//   k_gather      copy species counts of the new ensemble from their parents
//   k_finalize    per-run counts and offsets, iteration counter
//
// Every weight operation is a single IEEE double operation with an explicit round-to-nearest
// intrinsic; comparisons between non-negative doubles use their bit patterns.
#include "we_ssa_common.cuh"

namespace we {

// ------------------------------------------------------------------------------------------
// Per run (one block): exclusive scans of bin counts and of bin occupancy give, for every
// occupied bin, where its walkers go when grouped by bin (in_offset) and where its M_targ
// resampled walkers go in the new ensemble (out_offset = M_targ * occupied bins before it).
// ------------------------------------------------------------------------------------------
__global__ void k_scan_bins(EnsView E, int n_bins) {
  const int r = blockIdx.x, tid = threadIdx.x, B = blockDim.x;
  const int lane = tid & 31, wid = tid >> 5, nw = B >> 5;
  __shared__ int s_cnt[32], s_occ[32];
  __shared__ int s_base_cnt, s_base_occ;
  if (tid == 0) { s_base_cnt = 0; s_base_occ = 0; }
  __syncthreads();
  int *bc = E.bin_count + (size_t)r * n_bins;
  int4 *tasks = E.tasks + (size_t)r * n_bins;
  for (int base = 0; base < n_bins; base += B) {
    const int b = base + tid;
    const int c = b < n_bins ? bc[b] : 0;
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
    const int ex_c = s_base_cnt + wc + ic - c;
    const int ex_o = s_base_occ + wo + io - o;
    if (o) {
      tasks[ex_o] = make_int4(b, ex_c, c, ex_o * E.m_targ);
      E.cursor[(size_t)r * n_bins + b] = ex_c;
    }
    if (b < n_bins) bc[b] = 0;                            // ready for the next interval
    __syncthreads();
    if (tid == 0) { s_base_cnt += s_cnt[nw - 1]; s_base_occ += s_occ[nw - 1]; }
    __syncthreads();
  }
  if (tid == 0) {
    E.n_tasks[r] = s_base_occ;
    if ((long long)s_base_occ * E.m_targ > E.cap) atomicCAS(&E.status[r], 0, kStatusOverflow);
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

// Lightest live entry (weight bits >= 0) of a register-resident bin list, entries lane * 4 + q,
// keyed by (weight bits, slot), skipping entry `skip`; the result on every lane.
__device__ __forceinline__ void reg_argmin(const long long (&vv)[4], const int (&sl)[4], int lane, int skip,
                                           long long &bw, int &bs, int &bo) {
  bw = 0x7FFFFFFFFFFFFFFFll; bs = 0x7FFFFFFF; bo = -1;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const bool ok = vv[q] >= 0 && lane * 4 + q != skip;
    if (ok && (vv[q] < bw || (vv[q] == bw && sl[q] < bs))) { bw = vv[q]; bs = sl[q]; bo = lane * 4 + q; }
  }
#pragma unroll
  for (int d = 16; d >= 1; d >>= 1) {
    const long long ow = __shfl_xor_sync(0xffffffffu, bw, d);
    const int os = __shfl_xor_sync(0xffffffffu, bs, d);
    const int oo = __shfl_xor_sync(0xffffffffu, bo, d);
    if (ow < bw || (ow == bw && os < bs)) { bw = ow; bs = os; bo = oo; }
  }
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
__global__ void __launch_bounds__(128) k_resample(EnsView E, int n_bins) {
  const int r = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int n_warps = (gridDim.x * blockDim.x) >> 5;
  const int nt = E.n_tasks[r];
  const int iter = *E.iter;
  const int par = iter & 1;
  const int M = E.m_targ;
  const size_t base = (size_t)r * E.cap;
  double *W2 = E.w[par ^ 1] + base;
  int32_t *P2 = E.parent[par ^ 1] + base;
  const uint32_t k0 = (uint32_t)E.seed;
  const uint32_t k1 = (uint32_t)(E.seed >> 32) + E.run_id[r];
  const int slot_obs = iter - E.first_iter;
  const unsigned lt_mask = (1u << lane) - 1u;

  for (int t = warp; t < nt; t += n_warps) {
    const int4 tk = E.tasks[(size_t)r * n_bins + t];
    const int b = tk.x, in0 = tk.y, cnt = tk.z, out0 = tk.w;
    if (out0 + M > E.cap) continue;                       // capacity overflow, already flagged
    int32_t *lss = E.sorted_slot + base + in0;
    double *lsw = E.sorted_w + base + in0;
    int32_t *lal = E.alive + base + in0;
    if (cnt > M && cnt <= 128) {
      // Up to 128 walkers: entries i = lane + 32 q in registers, the argmins by shuffles, and
      // every merge's uniform drawn up front (merge k's counter does not depend on the others).
      long long vv[4];                                     // weight bits; -1: merged away
      int sl[4];
      unsigned long long ub[4];                            // bits of u for merges lane + 32 q
      const int n_merge = cnt - M;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        if (i < cnt) { vv[q] = bits(lsw[i]); sl[q] = lss[i]; }
        else { vv[q] = -1; sl[q] = 0x7FFFFFFF; }
        ub[q] = 0;
        if (i < n_merge) {
          uint32_t c0 = (uint32_t)i, c1 = (uint32_t)iter, c2 = (uint32_t)b, c3 = 1u;
          philox4x32_10(c0, c1, c2, c3, k0, k1);
          ub[q] = (unsigned long long)bits(u01(c0, c1));
        }
      }
      for (int km = 0; km < n_merge; ++km) {
        long long wa, wb;
        int sa, sb, oa, ob;
        reg_argmin(vv, sl, lane, -1, wa, sa, oa);
        reg_argmin(vv, sl, lane, oa, wb, sb, ob);
        const bool a_first = sa < sb;                        // p: the lower slot of the pair
        const long long wp = a_first ? wa : wb, wq = a_first ? wb : wa;
        const int op = a_first ? oa : ob, oq = a_first ? ob : oa;
        unsigned long long u_k = 0;
#pragma unroll
        for (int q = 0; q < 4; ++q) if ((km >> 5) == q) u_k = ub[q];
        u_k = __shfl_sync(0xffffffffu, u_k, km & 31);
        int keep_p = 0;
        long long wsum_bits = 0;
        if (lane == 0) {
          const double wsum = __dadd_rn(__longlong_as_double(wp), __longlong_as_double(wq));
          const double prob = __ddiv_rn(__longlong_as_double(wp), wsum);
          keep_p = (long long)u_k < bits(prob) ? 1 : 0;
          wsum_bits = bits(wsum);
        }
        keep_p = __shfl_sync(0xffffffffu, keep_p, 0);
        wsum_bits = __shfl_sync(0xffffffffu, wsum_bits, 0);
        const int osurv = keep_p ? op : oq, odead = keep_p ? oq : op;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (lane * 4 + q == osurv) vv[q] = wsum_bits;
          if (lane * 4 + q == odead) vv[q] = -1;
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        if (i < cnt) { lal[i] = vv[q] >= 0 ? 1 : 0; if (vv[q] >= 0) lsw[i] = __longlong_as_double(vv[q]); }
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
    } else if (cnt < M && cnt <= 128) {
      // Up to 128 walkers: each lane keeps its entries' per-copy weights w_i/c_i in registers,
      // so a round divides once (for the walker that received the copy), not once per walker.
      double wv[4];
      long long vv[4];
      int cc[4], sl[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        if (i < cnt) { wv[q] = lsw[i]; vv[q] = bits(wv[q]); cc[q] = 1; sl[q] = lss[i]; }
        else { wv[q] = 0.0; vv[q] = -1; cc[q] = 0; sl[q] = 0x7FFFFFFF; }
      }
      for (int extra = cnt; extra < M; ++extra) {
        long long bv = -1;
        int bs = 0x7FFFFFFF, bo = -1;
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (vv[q] > bv || (vv[q] == bv && sl[q] < bs)) { bv = vv[q]; bs = sl[q]; bo = lane * 4 + q; }
#pragma unroll
        for (int d = 16; d >= 1; d >>= 1) {
          const long long ov = __shfl_xor_sync(0xffffffffu, bv, d);
          const int os = __shfl_xor_sync(0xffffffffu, bs, d);
          const int oo = __shfl_xor_sync(0xffffffffu, bo, d);
          if (ov > bv || (ov == bv && os < bs)) { bv = ov; bs = os; bo = oo; }
        }
        double wsel = wv[0];
        int csel = cc[0];
#pragma unroll
        for (int q = 1; q < 4; ++q)
          if ((bo & 3) == q) { wsel = wv[q]; csel = cc[q]; }
        csel += 1;
        if ((bo >> 2) == lane) {                          // one division per round, by the owner
          const long long vnew = bits(__ddiv_rn(wsel, (double)csel));
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if ((bo & 3) == q) { cc[q] = csel; vv[q] = vnew; }
        }
      }
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = lane + 32 * q;
        if (i < cnt) lal[i] = cc[q];
      }
      __syncwarp();
    } else if (cnt < M) {
      for (int extra = cnt; extra < M; ++extra) {
        long long bv = -1;
        int bs = 0x7FFFFFFF, bi = -1;
        for (int i = lane; i < cnt; i += 32) {
          const long long v = bits(__ddiv_rn(lsw[i], (double)lal[i]));
          const int sl = lss[i];
          if (v > bv || (v == bv && sl < bs)) { bv = v; bs = sl; bi = i; }
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
      int sl = 0, c = 0;
      double wv = 0.0;
      if (i < cnt) { sl = lss[i]; c = lal[i]; wv = lsw[i]; }
      const unsigned m = __ballot_sync(0xffffffffu, c > 0);
      __syncwarp();
      if (c > 0) {
        const int d = k + __popc(m & lt_mask);
        lss[d] = sl; lal[d] = c; lsw[d] = wv;
      }
      k += __popc(m);
      __syncwarp();
    }
    // Output offset of each survivor: copies of all survivors with a lower slot.
    double wsum_local = 0.0;
    for (int i = lane; i < k; i += 32) {
      const int si = lss[i];
      int off = 0;
      for (int j = 0; j < k; ++j) off += (lss[j] < si) ? lal[j] : 0;
      const int c = lal[i];
      const double wi = lsw[i];
      const double wc = (cnt < M) ? __ddiv_rn(wi, (double)c) : wi;
      for (int q = 0; q < c; ++q) {
        W2[out0 + off + q] = wc;
        P2[out0 + off + q] = si;
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
  __shared__ int s_new[1024];
  const int iter = *E.iter;
  const int slot = iter - E.first_iter;
  for (int r = threadIdx.x; r < E.R; r += blockDim.x) {
    const int c = new_count(E, r, resample);
    if (r < 1024) s_new[r] = c;
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
    E.prev_count[r] = E.count[r];
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
  k_resample<<<dim3(bx, E.R), 128, 0, st>>>(E, nb);
  return cudaGetLastError();
}

cudaError_t launch_gather_finalize(const PropagateParams &prm, cudaStream_t st) {
  const EnsView &E = prm.ens;
  const int ld = E.R * E.cap;
  int grid = (ld + 255) / 256;
  if (grid > 152 * 8) grid = 152 * 8;
  k_gather<<<grid, 256, 0, st>>>(E, prm.resample);
  k_finalize<<<1, 256, 0, st>>>(E, prm.resample);
  return cudaGetLastError();
}

cudaError_t launch_pack_states(const EnsView &E, int r, int32_t *out, cudaStream_t st) {
  k_pack_states<<<152, 256, 0, st>>>(E, r, out);
  return cudaGetLastError();
}

}  // namespace we
