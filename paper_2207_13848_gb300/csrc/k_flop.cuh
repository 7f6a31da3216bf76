// FLOP per output row (Algorithm 1, Sec. V-A) fused with the per-row prediction
// (Eq. 4, or Eq. 2 for the reference design) and the exclusive scan into the
// allocation offsets, as one persistent launch.
//
// Work split: the rows' end markers and A's nonzeros form one merged sequence
// of M + nnz(A) items (the merge-path decomposition of Merrill and Garland,
// "Merge-based parallel sparse matrix-vector multiplication", SC 2016).  Block
// c takes the items [c*D/G, (c+1)*D/G), so every block reads the same number of
// nonzeros plus row ends, whatever the row-length skew.  A row owned by block c
// is one whose end marker lies in c's range; the part of a row that started in
// an earlier block arrives as a carry published by that block.
//
// Inside a block the rows are taken in windows of kWin rows (their end offsets
// staged in shared memory); the window's nonzeros are processed kChunk at a
// time, kItems consecutive nonzeros per thread.  A thread finds the row of its
// first nonzero by binary search in the staged ends, gathers the B row lengths
// of its nonzeros (the gathers are issued before they are consumed), and adds
// per-row partial sums into shared memory.
//
// All blocks are co-resident (cooperative launch).  Blocks exchange three
// things through flags in the workspace, each wait bounded: the carry of a row
// that spans blocks, the block's total of predicted nnz (for the scan), and, in
// the reference design, the block's FLOP total (F is needed before any
// prediction).
#pragma once

#include "common.cuh"

namespace spg {

constexpr int kFlopThreads = 512;
constexpr int kItems = 8;                       // nonzeros per thread per chunk
constexpr int kChunk = kFlopThreads * kItems;   // nonzeros per chunk
constexpr int kWin = 2048;                      // rows per window
constexpr int kRowsPerThread = 4;               // rows per thread in the write-out

enum FlopMode { kModeFlop = 0, kModePredict = 1, kModeReference = 2 };

struct FlopArgs {
  int64_t M, K, nnzA, nnzB;
  const int* a_rpt;
  const int* a_col;
  const int* b_rpt;
  int* flop;             // [M] per-row FLOP (caller's flop_row or workspace)
  int* pred;             // [M] per-row prediction (predict / reference)
  long long* offsets;    // [M + 1]
  Workspace ws;
  spgemm_result_t* res;
};

// Number of row ends among the first d items of the merged sequence: the
// largest i in [0, M] with i == 0 or rpt[i] + i <= d.  One warp, 32-way search.
__device__ long long merge_path_rows(const int* rpt, long long M, long long d) {
  const int lane = threadIdx.x & 31;
  long long lo = 0, hi = M + 1;  // predicate true at lo, false at hi
  while (hi - lo > 1) {
    const long long step = (hi - lo + 31) / 32;
    const long long x = lo + (long long)(lane + 1) * step;
    bool pr = false;
    if (x < hi) pr = (long long)__ldg(rpt + x) + x <= d;
    const unsigned b = __ballot_sync(kFull, pr);
    // predicate is monotone, so the true lanes form a prefix
    const int cnt = __popc(b);
    const long long nlo = lo + (long long)cnt * step;
    hi = min(hi, nlo + step);
    lo = nlo;
  }
  return lo;
}

struct FlopShared {
  int ends[kWin];
  int fsum[kWin];
  long long red[kFlopThreads / 32 + 1];
  long long bc[8];
};

__device__ __forceinline__ int upper_bound_smem(const int* v, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (v[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

template <int MODE>
__global__ void __launch_bounds__(kFlopThreads) k_flop_pred(FlopArgs a) {
  __shared__ FlopShared sm;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, c = blockIdx.x;
  WsHeader* hdr = a.ws.hdr;
  const unsigned ep = *reinterpret_cast<volatile unsigned*>(&hdr->epoch) + 1u;
  Slot* slots = a.ws.slots;

  // ---- this block's share of the merged sequence
  const long long D = a.M + a.nnzA;
  if (warp == 0) {
    const long long d0 = (long long)c * D / G, d1 = (long long)(c + 1) * D / G;
    const long long i0 = merge_path_rows(a.a_rpt, a.M, d0);
    const long long i1 = merge_path_rows(a.a_rpt, a.M, d1);
    if (lane == 0) {
      sm.bc[0] = i0;
      sm.bc[1] = min(max(d0 - i0, 0ll), (long long)a.nnzA);
      sm.bc[2] = i1;
      sm.bc[3] = min(max(d1 - i1, 0ll), (long long)a.nnzA);
    }
  }
  __syncthreads();
  const long long i0 = sm.bc[0], j0 = sm.bc[1], i1 = sm.bc[2];
  const long long j1 = max(sm.bc[3], j0);
  const bool tail_row = i1 < a.M;              // row i1 continues into the next block
  const long long r_end = tail_row ? i1 + 1 : i1;
  const bool head_split = (i0 < a.M) && (c > 0) && ((long long)__ldg(a.a_rpt + i0) < j0);

  bool bad = false;
  const double ratio = (MODE == kModePredict && hdr->f_acc) ? (double)hdr->z_acc / (double)hdr->f_acc : 0.0;
  long long ftot = 0, ptot = 0;  // per-thread sums over complete rows
  long long head_part = 0, tail_part = 0;

  // ---- phase 1: FLOP of every row touching this block's items
  for (long long wa = i0; wa < r_end; wa += kWin) {
    const int nw = (int)min((long long)kWin, r_end - wa);
    for (int k = t; k < nw; k += kFlopThreads) {
      const long long r = wa + k;
      long long e = (r == i1) ? j1 : (long long)__ldg(a.a_rpt + r + 1);
      e = min(max(e, j0), j1);
      sm.ends[k] = (int)e;
      sm.fsum[k] = 0;
    }
    long long js = max((long long)__ldg(a.a_rpt + wa), j0);
    js = min(js, j1);
    __syncthreads();
    const long long je = max((long long)sm.ends[nw - 1], js);
    for (long long s = js; s < je; s += kChunk) {
      const long long jt = s + (long long)t * kItems;
      if (jt < je) {
        const int n_u = (int)min((long long)kItems, je - jt);
        int col[kItems];
#pragma unroll
        for (int u = 0; u < kItems; ++u) col[u] = u < n_u ? __ldg(a.a_col + jt + u) : 0;
        int lo_[kItems], hi_[kItems];
#pragma unroll
        for (int u = 0; u < kItems; ++u) {
          lo_[u] = 0;
          hi_[u] = 0;
          if (u < n_u) {
            if ((unsigned)col[u] < (unsigned long long)a.K) {
              lo_[u] = __ldg(a.b_rpt + col[u]);
              hi_[u] = __ldg(a.b_rpt + col[u] + 1);
            } else {
              bad = true;
            }
          }
        }
        int k = upper_bound_smem(sm.ends, nw, (int)jt);
        int acc = 0;
#pragma unroll
        for (int u = 0; u < kItems; ++u) {
          if (u < n_u) {
            const int j = (int)(jt + u);
            while (k < nw - 1 && j >= sm.ends[k]) {
              if (acc) atomicAdd(&sm.fsum[k], acc);
              acc = 0;
              ++k;
            }
            int len = hi_[u] - lo_[u];
            if (len < 0 || lo_[u] < 0 || (long long)hi_[u] > a.nnzB) {
              bad = true;
              len = 0;
            }
            acc += len;
          }
        }
        if (acc) atomicAdd(&sm.fsum[min(k, nw - 1)], acc);
      }
    }
    __syncthreads();
    for (int k = t; k < nw; k += kFlopThreads) {
      const long long r = wa + k;
      const int v = sm.fsum[k];
      if (tail_row && r == i1) {
        tail_part = v;  // only one thread sees it
      } else if (head_split && r == i0) {
        head_part = v;
      } else {
        a.flop[r] = v;
        ftot += v;
        if (MODE == kModePredict) {
          ptot += (hdr->f_acc == 0) ? v : pred_proposed((uint32_t)v, hdr->z_acc, hdr->f_acc, ratio);
        }
      }
    }
    __syncthreads();
  }

  // gather the per-thread head/tail parts (each was set by at most one thread)
  const long long head_sum = block_sum<kFlopThreads>(head_part, sm.red);
  const long long tail_sum = block_sum<kFlopThreads>(tail_part, sm.red);
  if (__syncthreads_or(bad) && t == 0) set_status(hdr, SPGEMM_STATUS_ERR_BAD_INPUT);

  // ---- carry of rows spanning blocks (thread 0; waits only on block c-1)
  if (t == 0) {
    long long extra_f = 0, extra_p = 0;
    if (head_split && i0 == i1) {
      // the whole block lies inside one row: pass the carry on
      long long cin = 0;
      if (flag_wait(&slots[c - 1].carry_flag, ep, &hdr->status)) cin = slots[c - 1].carry;
      slots[c].carry = cin + tail_sum;
      flag_store(&slots[c].carry_flag, ep);
    } else {
      slots[c].carry = tail_row ? tail_sum : 0;
      flag_store(&slots[c].carry_flag, ep);
      if (head_split) {
        long long cin = 0;
        if (flag_wait(&slots[c - 1].carry_flag, ep, &hdr->status)) cin = slots[c - 1].carry;
        const long long v0 = cin + head_sum;
        a.flop[i0] = (int)v0;
        extra_f = v0;
        if (MODE == kModePredict)
          extra_p = (hdr->f_acc == 0) ? v0 : pred_proposed((uint32_t)v0, hdr->z_acc, hdr->f_acc, ratio);
      }
    }
    sm.bc[4] = extra_f;
    sm.bc[5] = extra_p;
  }
  __syncthreads();
  const long long blk_f = block_sum<kFlopThreads>(ftot, sm.red) + sm.bc[4];
  long long blk_p = block_sum<kFlopThreads>(ptot, sm.red) + sm.bc[5];

  if (MODE != kModeFlop) {
    // ---- the reference design needs F before any prediction
    double ratio_ref = 0.0;
    u128 zm = 0, den = 0;
    bool sat = false;
    const bool ref_empty = hdr->s_acc == 0;
    if (MODE == kModeReference) {
      if (t == 0) {
        slots[c].ftot = blk_f;
        flag_store(&slots[c].ftot_flag, ep);
      }
      long long fpart = 0;
      for (int q = t; q < G; q += kFlopThreads) {
        if (q == c) {
          fpart += blk_f;
        } else if (flag_wait(&slots[q].ftot_flag, ep, &hdr->status)) {
          fpart += *reinterpret_cast<volatile long long*>(&slots[q].ftot);
        }
      }
      const long long F = block_sum<kFlopThreads>(fpart, sm.red);
      zm = (u128)hdr->z_acc * (u128)(unsigned long long)a.M;
      den = (u128)(unsigned long long)F * (u128)hdr->s_acc;
      ratio_ref = (F > 0 && !ref_empty) ? ((double)hdr->z_acc * (double)a.M) / ((double)F * (double)hdr->s_acc) : 0.0;
      long long pp = 0;
      for (long long r = i0 + t; r < i1; r += kFlopThreads) {
        const int v = a.flop[r];
        pp += ref_empty ? v : pred_reference((uint32_t)v, zm, den, ratio_ref, &sat);
      }
      blk_p = block_sum<kFlopThreads>(pp, sm.red);
    }

    // ---- exclusive scan across blocks: sum of the totals of blocks 0..c-1
    if (t == 0) {
      slots[c].total = blk_p;
      flag_store(&slots[c].total_flag, ep);
    }
    long long ppart = 0;
    for (int q = t; q < c; q += kFlopThreads) {
      if (flag_wait(&slots[q].total_flag, ep, &hdr->status))
        ppart += *reinterpret_cast<volatile long long*>(&slots[q].total);
    }
    long long run = block_sum<kFlopThreads>(ppart, sm.red);

    // ---- phase 2: predictions and offsets of the owned rows [i0, i1)
    for (long long rb = i0; rb < i1; rb += (long long)kFlopThreads * kRowsPerThread) {
      const long long r0 = rb + (long long)t * kRowsPerThread;
      int pv[kRowsPerThread];
      long long loc = 0;
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        const long long r = r0 + u;
        pv[u] = 0;
        if (r < i1) {
          const int v = a.flop[r];
          if (MODE == kModePredict)
            pv[u] = (hdr->f_acc == 0) ? v : pred_proposed((uint32_t)v, hdr->z_acc, hdr->f_acc, ratio);
          else
            pv[u] = ref_empty ? v : pred_reference((uint32_t)v, zm, den, ratio_ref, &sat);
          loc += pv[u];
        }
      }
      long long tot;
      long long ex = block_excl_scan<kFlopThreads>(loc, sm.red, &tot) + run;
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        const long long r = r0 + u;
        if (r < i1) {
          a.pred[r] = pv[u];
          a.offsets[r] = ex;
          ex += pv[u];
        }
      }
      run += tot;
    }
    if (c == G - 1 && t == 0) {
      a.offsets[a.M] = run;
      a.res->pred_total = run;
    }
    if (__syncthreads_or(sat) && t == 0) set_status(hdr, SPGEMM_STATUS_WARN_SATURATED);
  }

  // ---- totals and reset by the last block to finish
  if (t == 0) {
    atomicAdd(&hdr->F_acc, (unsigned long long)blk_f);
    __threadfence();
    const unsigned prev = atomicAdd(&hdr->done, 1u);
    if (prev == (unsigned)G - 1) {
      __threadfence();
      volatile WsHeader* vh = hdr;
      unsigned st = vh->status;
      const bool empty = (MODE == kModePredict) ? vh->f_acc == 0 : (MODE == kModeReference ? vh->s_acc == 0 : false);
      if (empty) st |= SPGEMM_STATUS_WARN_EMPTY_SAMPLE;
      a.res->flop_total = (long long)vh->F_acc;
      a.res->flop_s = (long long)vh->f_acc;
      a.res->nnz_s = (long long)vh->z_acc;
      a.res->n_sampled = (long long)vh->s_acc;
      if (MODE == kModeFlop) a.res->pred_total = 0;
      a.res->status = (int)st;
      vh->f_acc = 0;
      vh->z_acc = 0;
      vh->s_acc = 0;
      vh->F_acc = 0;
      vh->heavy_count = 0;
      vh->status = 0;
      vh->done = 0;
      __threadfence();
      vh->epoch = ep;
    }
  }
}

}  // namespace spg
