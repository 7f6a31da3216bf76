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
// Inside a block, A's nonzeros are taken kChunk at a time (the chunk grid is
// aligned to 16 bytes, so every thread reads its kItems consecutive column ids
// with two 128-bit loads, issued one chunk ahead).  Each nonzero's B row length
// comes from one 128-bit load around B.rpt[c] (a second load only when the pair
// straddles it); the lengths go to shared memory.  Then one thread per row sums
// its row's segment of the chunk (segments longer than kLong are summed by
// whole warps), into per-row sums of the current window of kWin rows, whose end
// offsets sit in shared memory.  When a window's rows are complete it is
// emitted: the prediction of each row is computed once and written.
//
// All blocks are co-resident (the grid never exceeds what the device holds at
// once).  Blocks exchange three things through flags in the workspace, each
// wait bounded: the carry of a row that spans blocks, the block's total of
// predicted nnz (for the scan), and, in the reference design, the block's FLOP
// total (F is needed before any prediction).
#pragma once

#include "common.cuh"

namespace spg {

constexpr int kFlopThreads = 512;
constexpr int kItems = 8;                       // nonzeros per thread per chunk
constexpr int kChunk = kFlopThreads * kItems;   // nonzeros per chunk
constexpr int kWin = 2048;                      // rows per window
constexpr int kLong = 64;                       // longer row segments are summed by warps
constexpr int kMaxLong = kChunk / kLong + 1;
constexpr int kRowsPerThread = 4;               // rows per thread in the offsets pass

enum FlopMode { kModeFlop = 0, kModePredict = 1, kModeReference = 2 };

struct FlopArgs {
  int64_t M, K, nnzA, nnzB;
  const int* a_rpt;
  const int* a_col;
  const int* b_rpt;
  int* flop;             // [M] per-row FLOP: caller's flop_row, or null (predict) / workspace (others)
  int* pred;             // [M] per-row prediction (predict / reference)
  long long* offsets;    // [M + 1]
  int vec_ok;            // A.col and B.rpt are 16-byte aligned: 128-bit loads allowed
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
  alignas(16) int lbuf[kChunk];  // B row lengths of the chunk's nonzeros
  int ends[kWin];    // end offset of each window row (clamped to the block's range)
  int fsum[kWin];    // per-row FLOP of the window rows
  int long_k[kMaxLong], long_a[kMaxLong], long_b[kMaxLong];
  int long_n;
  int win_js;        // first nonzero of the window's first row (clamped)
  long long red[kFlopThreads / 32 + 1];
  long long bc[8];
};

// First index k in [lo, n) with v[k] >= key, or n.
__device__ __forceinline__ int lower_bound_smem(const int* v, int lo, int n, int key) {
  int hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// B row length of column id c, with bounds checks; one 128-bit load when possible.
struct LenLoad {
  int4 v;
  int extra;
};

template <int MODE>
__global__ void __launch_bounds__(kFlopThreads, 2) k_flop_pred(FlopArgs a) {
  __shared__ FlopShared sm;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, c = blockIdx.x;
  WsHeader* hdr = a.ws.hdr;
  const unsigned ep = *reinterpret_cast<volatile unsigned*>(&hdr->epoch) + 1u;
  Slot* slots = a.ws.slots;
  const int K = (int)a.K;

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
  if (t == 0) sm.long_n = 0;
  __syncthreads();
  const int i0 = (int)sm.bc[0], j0 = (int)sm.bc[1], i1 = (int)sm.bc[2];
  const int j1 = (int)max(sm.bc[3], sm.bc[1]);
  const bool tail_row = i1 < a.M;  // row i1 continues into the next block
  const int r_end = tail_row ? i1 + 1 : i1;
  const bool head_split = (i0 < a.M) && (c > 0) && (__ldg(a.a_rpt + i0) < j0);

  bool bad = false;
  const unsigned long long fz = hdr->f_acc, zz = hdr->z_acc;
  const double ratio = (MODE == kModePredict && fz) ? (double)zz / (double)fz : 0.0;
  long long ftot = 0, ptot = 0;  // per-thread sums over complete rows
  long long head_part = 0, tail_part = 0;

  // ---- window of rows [wa, wa + nw)
  int wa = i0, nw = 0;
  auto load_window = [&](int start) {
    wa = start;
    nw = min(kWin, r_end - wa);
    for (int k = t; k < nw; k += kFlopThreads) {
      const int r = wa + k;
      int e = (tail_row && r == i1) ? j1 : __ldg(a.a_rpt + r + 1);
      e = min(max(e, j0), j1);
      sm.ends[k] = e;
      sm.fsum[k] = 0;
    }
    if (t == 0) sm.win_js = min(max(__ldg(a.a_rpt + wa), j0), j1);
  };
  auto emit_window = [&]() {
    for (int k = t; k < nw; k += kFlopThreads) {
      const int r = wa + k;
      const int v = sm.fsum[k];
      if (tail_row && r == i1) {
        tail_part = v;  // seen by one thread only
      } else if (head_split && r == i0) {
        head_part = v;
      } else {
        ftot += v;
        if (MODE == kModePredict) {
          const int p = fz == 0 ? v : pred_proposed((uint32_t)v, zz, fz, ratio);
          a.pred[r] = p;
          ptot += p;
          if (a.flop) a.flop[r] = v;
        } else {
          a.flop[r] = v;
        }
      }
    }
  };

  // ---- column ids of this thread's items of a chunk, as two 128-bit loads
  auto load_cols = [&](int cs, int* col) {
    const int q0 = cs + t * kItems;
    if (a.vec_ok && (long long)q0 + kItems <= a.nnzA && q0 >= 0) {
      const int4 x = __ldg(reinterpret_cast<const int4*>(a.a_col + q0));
      const int4 y = __ldg(reinterpret_cast<const int4*>(a.a_col + q0 + 4));
      col[0] = x.x; col[1] = x.y; col[2] = x.z; col[3] = x.w;
      col[4] = y.x; col[5] = y.y; col[6] = y.z; col[7] = y.w;
    } else {
#pragma unroll
      for (int u = 0; u < kItems; ++u) {
        const int q = q0 + u;
        col[u] = (q >= 0 && q < a.nnzA) ? __ldg(a.a_col + q) : 0;
      }
    }
  };

  load_window(i0);
  const int cs0 = j0 & ~3;
  int col[kItems];
  if (cs0 < j1) load_cols(cs0, col);
  int ka = 0;
  __syncthreads();

  // ---- phase 1: FLOP of every row touching this block's items
  for (int cs = cs0; cs < j1; cs += kChunk) {
    const int lo = max(cs, j0), hi = min(cs + kChunk, j1);
    // B row lengths of this thread's items, gathers issued four at a time
    int len[kItems];
#pragma unroll
    for (int h = 0; h < kItems; h += 4) {
      LenLoad ld[4];
      bool use[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = cs + t * kItems + h + u;
        const int cc = col[h + u];
        use[u] = q >= lo && q < hi;
        ld[u].v = make_int4(0, 0, 0, 0);
        ld[u].extra = 0;
        if (use[u]) {
          if ((unsigned)cc >= (unsigned)K) {
            bad = true;
            use[u] = false;
          } else if (a.vec_ok && (cc | 3) <= K) {
            ld[u].v = __ldg(reinterpret_cast<const int4*>(a.b_rpt) + (cc >> 2));
            if ((cc & 3) == 3) ld[u].extra = __ldg(a.b_rpt + cc + 1);
          } else {
            ld[u].v.x = __ldg(a.b_rpt + cc);
            ld[u].v.y = __ldg(a.b_rpt + cc + 1);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int cc = col[h + u];
        int b0, b1;
        if (a.vec_ok && (cc | 3) <= K) {
          const int r = cc & 3;
          b0 = r == 0 ? ld[u].v.x : r == 1 ? ld[u].v.y : r == 2 ? ld[u].v.z : ld[u].v.w;
          b1 = r == 0 ? ld[u].v.y : r == 1 ? ld[u].v.z : r == 2 ? ld[u].v.w : ld[u].extra;
        } else {
          b0 = ld[u].v.x;
          b1 = ld[u].v.y;
        }
        int l = b1 - b0;
        if (use[u] && (l < 0 || b0 < 0 || (long long)b1 > a.nnzB)) {
          bad = true;
          l = 0;
        }
        len[h + u] = use[u] ? l : 0;
      }
    }
    {
      // prefetch the next chunk's column ids
      if (cs + kChunk < j1) load_cols(cs + kChunk, col);
      int4* lb = reinterpret_cast<int4*>(sm.lbuf + t * kItems);
      lb[0] = make_int4(len[0], len[1], len[2], len[3]);
      lb[1] = make_int4(len[4], len[5], len[6], len[7]);
    }
    __syncthreads();
    // one thread per row of the window overlapping [pos, hi)
    int pos = lo;
    for (;;) {
      const int kb = lower_bound_smem(sm.ends, ka, nw, hi);  // first row ending at or after hi
      const int kend = min(kb, nw - 1);
      for (int k = ka + t; k <= kend; k += kFlopThreads) {
        const int rs = k == 0 ? sm.win_js : sm.ends[k - 1];
        const int sa = max(rs, pos), sb = min(sm.ends[k], hi);
        if (sb - sa > kLong) {
          const int e = atomicAdd(&sm.long_n, 1);
          sm.long_k[e] = k;
          sm.long_a[e] = sa;
          sm.long_b[e] = sb;
        } else {
          int acc = 0;
          for (int q = sa; q < sb; ++q) acc += sm.lbuf[q - cs];
          sm.fsum[k] += acc;
        }
      }
      __syncthreads();
      const int nl = sm.long_n;
      if (nl) {
        for (int e = 0; e < nl; ++e) {
          const int sa = sm.long_a[e], sb = sm.long_b[e];
          int acc = 0;
          for (int q = sa + t; q < sb; q += kFlopThreads) acc += sm.lbuf[q - cs];
          acc = warp_sum(acc);
          if (lane == 0 && acc) atomicAdd(&sm.fsum[sm.long_k[e]], acc);
        }
        __syncthreads();
        if (t == 0) sm.long_n = 0;
      }
      if (kb < nw) {
        ka = kend;
        break;
      }
      // every row of the window ends before hi: emit it, move to the next rows
      emit_window();
      __syncthreads();
      load_window(wa + nw);
      __syncthreads();
      pos = sm.win_js;
      ka = 0;
      if (nw <= 0) break;
    }
  }
  // rows left after the last nonzero (the last window and trailing empty rows)
  if (nw > 0) emit_window();
  __syncthreads();
  while (wa + nw < r_end) {
    load_window(wa + nw);
    __syncthreads();
    emit_window();
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
        extra_f = v0;
        if (MODE == kModePredict) {
          const int p = fz == 0 ? (int)v0 : pred_proposed((uint32_t)v0, zz, fz, ratio);
          a.pred[i0] = p;
          if (a.flop) a.flop[i0] = (int)v0;
          extra_p = p;
        } else {
          a.flop[i0] = (int)v0;
        }
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
    bool sat = false;
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
      const unsigned long long S = hdr->s_acc;
      const u128 zm = (u128)zz * (u128)(unsigned long long)a.M;
      const u128 den = (u128)(unsigned long long)F * (u128)S;
      const double ratio_ref = (F > 0 && S) ? ((double)zz * (double)a.M) / ((double)F * (double)S) : 0.0;
      long long pp = 0;
      for (int r = i0 + t; r < i1; r += kFlopThreads) {
        const int v = a.flop[r];
        const int p = S == 0 ? v : pred_reference((uint32_t)v, zm, den, ratio_ref, &sat);
        a.pred[r] = p;
        pp += p;
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

    // ---- phase 2: offsets of the owned rows [i0, i1)
    for (int rb = i0; rb < i1; rb += kFlopThreads * kRowsPerThread) {
      const int r0 = rb + t * kRowsPerThread;
      int pv[kRowsPerThread];
      long long loc = 0;
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        pv[u] = (r0 + u < i1) ? a.pred[r0 + u] : 0;
        loc += pv[u];
      }
      long long tot;
      long long ex = block_excl_scan<kFlopThreads>(loc, sm.red, &tot) + run;
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        if (r0 + u < i1) {
          a.offsets[r0 + u] = ex;
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
