// FLOP per output row (Algorithm 1, Sec. V-A) fused with the per-row prediction
// (Eq. 4, or Eq. 2 for the reference design) and the exclusive scan into the
// allocation offsets, as one persistent launch.
//
// Work split: the rows' end markers and A's nonzeros form one merged sequence
// of M + nnz(A) items (the merge-path decomposition of Merrill and Garland,
// "Merge-based parallel sparse matrix-vector multiplication", SC 2016).  Block
// c takes the items [c*D/G, (c+1)*D/G) and splits them again, evenly, among
// its warps, so every warp reads the same number of nonzeros plus row ends,
// whatever the row-length skew.  A row belongs to the warp (and block) holding
// its end marker; the part of a row that started in an earlier warp or block
// is carried over.
//
// Each warp streams its range on its own, with no block-wide barrier: per step
// it reads kSub column ids with fully coalesced 128-bit loads (issued one step
// ahead), looks up each nonzero's B row length in a byte table built per call
// (k_degree_table; B.rpt only for lengths of 255 or more), and stores the
// inclusive prefix sums of the step's lengths in a warp-private shared buffer.
// Lane l owns row rbase + l of a 32-row window whose end offsets it holds in a
// register; the row's share of the step is the difference of two prefix sums,
// whatever its length.  When the window's rows are complete the warp writes
// their predictions (computed once per row) and moves on.  After the stream,
// one thread joins the rows split between warps, then blocks exchange, through flags in the workspace with bounded
// waits: the carry of a row that spans blocks, the block's total of predicted
// nnz (for the scan), and, in the reference design, the block's FLOP total (F
// is needed before any prediction).  All blocks are co-resident (the grid
// never exceeds what the device holds at once).
#pragma once

#include "common.cuh"

namespace spg {

// Build-time tuning knobs (defaults are the tuned values on GB300).
#ifndef SPG_FLOP_THREADS
#define SPG_FLOP_THREADS 256
#endif
#ifndef SPG_FLOP_MIN_BLOCKS
#define SPG_FLOP_MIN_BLOCKS 4
#endif
#ifndef SPG_LANE_ITEMS
#define SPG_LANE_ITEMS 8
#endif

constexpr int kFlopThreads = SPG_FLOP_THREADS;
constexpr int kFlopWarps = kFlopThreads / 32;
constexpr int kLaneItems = SPG_LANE_ITEMS;      // nonzeros per lane per step (multiple of 4)
constexpr int kSub = 32 * kLaneItems;           // nonzeros per warp step
constexpr int kRowsPerThread = 4;               // rows per thread in the offsets pass
constexpr int kNoEnd = 0x7fffffff;

enum FlopMode { kModeFlop = 0, kModePredict = 1, kModeReference = 2 };

struct FlopArgs {
  int64_t M, K, nnzA, nnzB;
  const int* a_rpt;
  const int* a_col;
  const int* b_rpt;
  const unsigned char* deg8;  // [K] B row lengths capped at kDegEscape (k_degree_table)
  int* flop;             // [M] per-row FLOP: caller's flop_row, or null (predict) / workspace (others)
  int* pred;             // [M] per-row prediction (predict / reference)
  long long* offsets;    // [M + 1]
  int vec_ok;            // A.col and B.rpt are 16-byte aligned: 128-bit loads allowed
  Workspace ws;
  spgemm_result_t* res;
};

// Number of row ends among the first d items of the merged sequence: the
// largest i in [0, M] with i == 0 or rpt[i] + i <= d (the predicate is
// monotone in i).  Two independent searches run at once, one per half-warp
// (16-way each): iA for dA and iB for dB, both over the whole matrix.  Cuts the dependent loads of a block's set-up from two
// nested searches to one.
__device__ void merge_path_rows2(const int* rpt, long long M, long long dA, long long dB,
                                 long long* iA, long long* iB) {
  const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
  const long long d = half ? dB : dA;
  long long lo = 0, hi = M + 1;  // predicate true at lo, false at hi
  for (;;) {
    const bool active = hi - lo > 1;
    if (!__any_sync(kFull, active)) break;
    const long long step = (hi - lo + 15) / 16;
    const long long x = lo + (long long)(hl + 1) * step;
    const bool pr = active && x < hi && (long long)__ldg(rpt + x) + x <= d;
    const unsigned b = __ballot_sync(kFull, pr);
    const unsigned mine = half ? (b >> 16) : (b & 0xffffu);
    if (active) {
      const long long nlo = lo + (long long)__popc(mine) * step;
      hi = min(hi, nlo + step);
      lo = nlo;
    }
  }
  *iA = __shfl_sync(kFull, lo, 0);
  *iB = __shfl_sync(kFull, lo, 16);
}

// What a warp leaves for the block after its stream.
struct WarpInfo {
  int first_row;    // the warp's first row
  int has_end;      // the warp holds at least one row end
  int head_split;   // its first row started before the warp's range
  int head_part;    // that row's partial FLOP within the warp (when it also ends here)
  int tail_part;    // partial FLOP of the row open at the warp's end
  int pad[3];
};

// What a block's pass over one range of the merged sequence leaves behind.
struct RangeOut {
  int i0, i1, j0;              // rows [i0, i1) end in the range; j0 = its first nonzero
  long long run;               // partial FLOP of the row open at the range's end
  long long head_known;        // the first row's FLOP minus the carry (if head_pending)
  long long extra_f, extra_p;  // FLOP / predictions of rows split between warps
  bool dep;                    // the whole range lies inside one row
  bool head_pending;           // the first row waits for the previous range's carry
};

template <int NW>
struct FlopSharedT {
  alignas(16) int lens[NW][kSub];  // prefix sums of B row lengths over a warp's step
  WarpInfo info[NW];
  long long red[NW + 1];
  long long bc[8];
  RangeOut out;
};
using FlopShared = FlopSharedT<kFlopWarps>;

// B row-length table lookup.  A plain (coherent) load: the fused predictor
// builds the table earlier in the same launch, so the read-only path is not
// used for it.
__device__ __forceinline__ unsigned table_load(const unsigned char* p) { return *p; }

// One block (or the group of NW warps starting at warp WOFF, synchronised by
// hardware barrier BAR) streams the items [d0, d1) of the merged sequence: every row that
// ends in the range and starts in it gets its prediction (predict mode) or its
// FLOP written; rows split between warps are joined here; the row split with
// the previous range (has_prev) and the row left open at the end are reported
// in *out (written by the group's first thread; all its threads may read it on
// return).  ftot/ptot receive this thread's share of the FLOP / prediction
// sums of finished rows.  pre_wl0/pre_wl1, when not negative, are the warp's
// row bounds for its share of [d0, d1) (found earlier by merge_path_rows2).
template <int MODE, int NW, int WOFF = 0, int BAR = 0>
__device__ __forceinline__ void flop_range(const FlopArgs& a, long long d0, long long d1, bool has_prev,
                                           unsigned long long fz, unsigned long long zz, double ratio,
                                           FlopSharedT<NW>& sm, RangeOut* out, long long& ftot,
                                           long long& ptot, bool& bad, int* sflop = nullptr,
                                           int sflop_n = 0, bool flop_global = true,
                                           long long pre_wl0 = -1, long long pre_wl1 = -1) {
  // ---- the range is split evenly among the block's warps; each warp finds
  // both of its bounds in one pass, and the range's bounds are the first
  // warp's start and the last warp's end
  const int t = threadIdx.x, lane = t & 31, warp = (t >> 5) - WOFF;
  const bool leader = t == WOFF * 32;
  const int K = (int)a.K;
  const int M = (int)a.M;
  const long long wd0 = d0 + (d1 - d0) * warp / NW;
  const long long wd1 = d0 + (d1 - d0) * (warp + 1) / NW;
  long long wl0 = pre_wl0, wl1 = pre_wl1;  // the warp's row bounds, when the caller found them
  if (pre_wl0 < 0) merge_path_rows2(a.a_rpt, a.M, wd0, wd1, &wl0, &wl1);
  if (lane == 0 && warp == 0) sm.bc[0] = wl0;
  if (lane == 0 && warp == NW - 1) sm.bc[1] = wl1;
  group_sync<BAR, NW * 32>();
  const long long bi0 = sm.bc[0], bi1 = sm.bc[1];
  const int i0 = (int)bi0, i1 = (int)bi1;
  // FLOP mode: the block's row r goes to sflop[r - (i0 & ~3)] when it fits
  // there (so that groups of 4 rows starting at a multiple of 4 are 16-byte
  // aligned in shared memory), and to a.flop[r] when flop_global or when it
  // does not fit
  auto store_flop = [&](int r, int v) {
    const int o = r - (i0 & ~3);
    const bool in_s = sflop != nullptr && (unsigned)o < (unsigned)sflop_n;
    if (in_s) sflop[o] = v;
    if (flop_global || !in_s) a.flop[r] = v;
  };
  const int j0 = (int)min(max(d0 - bi0, 0ll), (long long)a.nnzA);
  const int j1 = (int)max(min(max(d1 - bi1, 0ll), (long long)a.nnzA), (long long)j0);
  const int wi0 = (int)wl0, wi1 = (int)wl1;
  const int wj0 = (int)min(max(wd0 - wl0, (long long)j0), (long long)j1);
  const int wj1 = (int)min(max(wd1 - wl1, (long long)wj0), (long long)j1);
  const bool wtail = wi1 < M;                 // row wi1 continues past this warp
  const int rows_hi = wtail ? wi1 + 1 : wi1;  // rows touched: [wi0, rows_hi)
  const bool whead = wi0 < M && __ldg(a.a_rpt + wi0) < wj0;  // first row started earlier

  int head_part = 0, tail_part = 0;
  int* lw = sm.lens[warp];

  // ---- the 32-row window [rbase, rbase + 32): lane l holds row rbase + l's end
  int rbase = wi0;
  int e_l = kNoEnd, st_l = 0;
  // raw end offset of this lane's row in the next window, loaded one window ahead
  int e_next = 0;
  auto fetch_next = [&](int rb) {
    const int r = rb + lane;
    e_next = (r < rows_hi && !(wtail && r == wi1)) ? __ldg(a.a_rpt + r + 1) : 0;
  };
  auto load_rows = [&](int rb, int start_of_rb) {  // rb's ends were fetched by fetch_next(rb)
    rbase = rb;
    const int r = rb + lane;
    if (r < rows_hi) {
      const int e = (wtail && r == wi1) ? wj1 : e_next;
      e_l = min(max(e, wj0), wj1);
    } else {
      e_l = kNoEnd;
    }
    const int prev = __shfl_up_sync(kFull, e_l, 1);
    st_l = lane == 0 ? start_of_rb : prev;
    fetch_next(rb + 32);
  };
  int acc = 0;
  auto emit_rows = [&]() {
    const int r = rbase + lane;
    if (r < rows_hi) {
      const int v = acc;
      if (wtail && r == wi1) {
        tail_part = v;
      } else if (whead && r == wi0) {
        head_part = v;
      } else {
        ftot += v;
        if (MODE == kModePredict) {
          const int p = fz == 0 ? v : pred_proposed((uint32_t)v, zz, fz, ratio);
          a.pred[r] = p;
          ptot += p;
          if (a.flop) a.flop[r] = v;
        } else {
          store_flop(r, v);
        }
      }
    }
    acc = 0;
  };

  fetch_next(wi0);
  load_rows(wi0, min(max(wi0 < M ? __ldg(a.a_rpt + wi0) : wj0, wj0), wj1));

  // ---- column ids of a step: lane l takes [s + 4l, s + 4l + 4) and the same +128
  auto load_cols = [&](int s, int* col) {
#pragma unroll
    for (int h = 0; h < kLaneItems / 4; ++h) {
      const int q0 = s + 4 * lane + 128 * h;
      if (a.vec_ok && q0 >= 0 && (long long)q0 + 4 <= a.nnzA) {
        const int4 x = __ldg(reinterpret_cast<const int4*>(a.a_col + q0));
        col[4 * h] = x.x;
        col[4 * h + 1] = x.y;
        col[4 * h + 2] = x.z;
        col[4 * h + 3] = x.w;
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = q0 + u;
          col[4 * h + u] = (q >= 0 && q < a.nnzA) ? __ldg(a.a_col + q) : 0;
        }
      }
    }
  };

  const int s0 = wj0 & ~3;
  int col[kLaneItems];
  if (s0 < wj1) load_cols(s0, col);

  for (int s = s0; s < wj1; s += kSub) {
    const int lo = max(s, wj0), hi = min(s + kSub, wj1);
    // B row lengths from the byte table (B.rpt only for lengths >= kDegEscape),
    // then their inclusive prefix sums over the step's kSub items (mod 2^32).
    unsigned len[kLaneItems];
#pragma unroll
    for (int u = 0; u < kLaneItems; ++u) {  // all of the lane's gathers in flight at once
      const int q = s + 4 * lane + 128 * (u >> 2) + (u & 3);
      const int cc = col[u];
      len[u] = 0;
      if (q >= lo && q < hi) {
        if ((unsigned)cc < (unsigned)K) {
          len[u] = table_load(a.deg8 + cc);
        } else {
          bad = true;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kLaneItems; ++u) {
      if (len[u] == kDegEscape) {
        const int cc = col[u];
        const int b0 = __ldg(a.b_rpt + cc), b1 = __ldg(a.b_rpt + cc + 1);
        len[u] = (unsigned)(b1 - b0);  // validated by the table kernel
      }
    }
    unsigned run_half = 0;
#pragma unroll
    for (int h = 0; h < kLaneItems / 4; ++h) {
      const unsigned p0 = len[4 * h], p1 = p0 + len[4 * h + 1], p2 = p1 + len[4 * h + 2],
                     p3 = p2 + len[4 * h + 3];
      const unsigned incl = warp_incl_scan(p3);
      const unsigned base = run_half + incl - p3;
      *reinterpret_cast<uint4*>(lw + 4 * lane + 128 * h) = make_uint4(base + p0, base + p1, base + p2, base + p3);
      run_half += __shfl_sync(kFull, incl, 31);
    }
    if (s + kSub < wj1) load_cols(s + kSub, col);  // next step's ids, in flight during the sums
    __syncwarp();

    // per-row sums over [lo, hi) from the prefix sums; the window moves on
    // while its rows complete
    for (;;) {
      const bool mine = rbase + lane < rows_hi;
      const int sa = max(st_l, lo), sb = min(e_l, hi);
      if (mine && sb > sa) {
        const unsigned pb = lw[sb - 1 - s];
        const unsigned pa = sa > s ? (unsigned)lw[sa - 1 - s] : 0u;
        acc += (int)(pb - pa);
      }
      const int ll = min(31, rows_hi - 1 - rbase);
      const int last_end = __shfl_sync(kFull, e_l, ll);
      if (last_end > hi || rbase + 32 >= rows_hi) break;  // rows continue into the next step
      // all 32 rows of the window end within this step
      emit_rows();
      load_rows(rbase + 32, last_end);
    }
    __syncwarp();
  }
  // rows left after the last nonzero: the current window, then empty rows
  emit_rows();
  while (rbase + 32 < rows_hi) {
    const int last_end = __shfl_sync(kFull, e_l, 31);
    load_rows(rbase + 32, last_end);
    emit_rows();
  }

  // ---- per-warp summary for the block
  tail_part = __reduce_add_sync(kFull, tail_part);
  head_part = __reduce_add_sync(kFull, head_part);
  if (lane == 0) {
    WarpInfo& w = sm.info[warp];
    w.first_row = wi0;
    w.has_end = wi1 > wi0;
    w.head_split = whead;
    w.head_part = head_part;
    w.tail_part = tail_part;
  }
  const bool blk_head_split = (i0 < M) && has_prev && (__ldg(a.a_rpt + i0) < j0);
  group_sync<BAR, NW * 32>();

  // ---- rows split between warps (thread 0).  Only the range's first row can
  // depend on the carry from the previous range.
  if (leader) {
    long long run = 0;          // partial of the open row entering warp w
    bool dep = blk_head_split;  // ... plus the previous block's carry
    long long head_known = 0;   // block's first row: everything but the carry
    bool head_pending = false;
    long long extra_f = 0, extra_p = 0;
    for (int w = 0; w < NW; ++w) {
      const WarpInfo& in = sm.info[w];
      if (!in.has_end) {
        run += in.tail_part;
        continue;
      }
      if (in.head_split) {
        const long long v = run + in.head_part;
        if (dep) {
          head_known = v;
          head_pending = true;
        } else {
          extra_f += v;
          if (MODE == kModePredict) {
            const int p = fz == 0 ? (int)v : pred_proposed((uint32_t)v, zz, fz, ratio);
            a.pred[in.first_row] = p;
            if (a.flop) a.flop[in.first_row] = (int)v;
            extra_p += p;
          } else {
            store_flop(in.first_row, (int)v);
          }
        }
      }
      dep = false;
      run = in.tail_part;
    }
    out->i0 = i0;
    out->i1 = i1;
    out->j0 = j0;
    out->run = run;
    out->head_known = head_known;
    out->extra_f = extra_f;
    out->extra_p = extra_p;
    out->dep = dep;
    out->head_pending = head_pending;
  }
  group_sync<BAR, NW * 32>();
}

template <int MODE>
__global__ void __launch_bounds__(kFlopThreads, SPG_FLOP_MIN_BLOCKS) k_flop_pred(FlopArgs a) {
  __shared__ FlopShared sm;
  const int t = threadIdx.x;
  const int G = gridDim.x, c = blockIdx.x;
  WsHeader* hdr = a.ws.hdr;
  const unsigned ep = *reinterpret_cast<volatile unsigned*>(&hdr->epoch) + 1u;
  Slot* slots = a.ws.slots;
  const int M = (int)a.M;
  const unsigned long long fz = hdr->f_acc, zz = hdr->z_acc;
  const double ratio = (MODE == kModePredict && fz) ? (double)zz / (double)fz : 0.0;

  // ---- this block's share of the merged sequence
  const long long D = a.M + a.nnzA;
  const long long d0 = (long long)c * D / G, d1 = (long long)(c + 1) * D / G;
  bool bad = false;
  long long ftot = 0, ptot = 0;
  flop_range<MODE>(a, d0, d1, c > 0, fz, zz, ratio, sm, &sm.out, ftot, ptot, bad);
  if (__syncthreads_or(bad) && t == 0) set_status(hdr, SPGEMM_STATUS_ERR_BAD_INPUT);
  const int i0 = sm.out.i0, i1 = sm.out.i1;

  if (t == 0) {
    const long long run = sm.out.run, head_known = sm.out.head_known;
    const bool dep = sm.out.dep, head_pending = sm.out.head_pending;
    long long extra_f = sm.out.extra_f, extra_p = sm.out.extra_p;
    // carries between blocks (waits only on block c-1)
    if (dep) {
      // the whole block lies inside one row: pass the carry on
      long long cin = 0;
      if (flag_wait(&slots[c - 1].carry_flag, ep, &hdr->status)) cin = slots[c - 1].carry;
      slots[c].carry = cin + run;
      flag_store(&slots[c].carry_flag, ep);
    } else {
      slots[c].carry = i1 < M ? run : 0;
      flag_store(&slots[c].carry_flag, ep);
      if (head_pending) {
        long long cin = 0;
        if (flag_wait(&slots[c - 1].carry_flag, ep, &hdr->status)) cin = slots[c - 1].carry;
        const long long v = cin + head_known;
        extra_f += v;
        if (MODE == kModePredict) {
          const int p = fz == 0 ? (int)v : pred_proposed((uint32_t)v, zz, fz, ratio);
          a.pred[i0] = p;
          if (a.flop) a.flop[i0] = (int)v;
          extra_p += p;
        } else {
          a.flop[i0] = (int)v;
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
