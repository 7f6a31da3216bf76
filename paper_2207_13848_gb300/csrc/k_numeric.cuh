// Numeric product C = A*B written into an allocation sized by the prediction:
// the consumer of the predicted structure.  The prediction sizes the memory of
// C before any product is formed, which is what the sampled compression ratio
// is for (Sec. I: it replaces the symbolic phase of a two-phase SpGEMM).  Two
// ways to use it:
//   - per-row shares: row i goes to alloc[i] when its exact size fits
//     alloc[i+1] - alloc[i] (the offsets of Eq. 4 per row);
//   - one pool of the predicted total (Z2* = F z*/f*, Eq. 4): each row takes
//     exactly its size from one of kPoolStripes bump pointers over equal slices
//     of the pool (the stripe chosen by a hash of the row, the next ones when it
//     is full), so the rows' positions follow their completion, not their order.
// Either way the start of every row is recorded (-1 when it did not fit, an
// overflow).  The compaction pass then builds the exact CSR: every row that was
// written moves (a flat, balanced copy over the exact layout), the rows that
// overflowed are computed again.
//
// Rows are computed row-wise (Gustavson): every product a_ik * b_kc of row i is
// added into an accumulator keyed by its column c.  Accumulators:
//   - one warp per row with at most kNumWarpCap products: an open-addressing
//     table of (column, value) pairs in the warp's slice of shared memory;
//   - heavier rows are queued and taken by whole blocks: a shared table of
//     kNumBlockSlots pairs (rows of at most kNumBlockCap products), else a dense
//     shared accumulator over kNumDenseCols columns at a time, pass after pass
//     over B's column range (entries then come out in ascending column order).
// Column ids within a row come out in no particular order (table order), except
// from the dense passes.  Values are single precision, summed in whatever order
// the shared-memory atomics take; the structure does not depend on that order.
#pragma once

#include "common.cuh"
#include "k_dedup.cuh"  // ceil_log2

namespace spg {

constexpr int kNumThreads = 64;                    // warp-per-row pass: 2 warps per block (fastest of 64, 128, 256)
constexpr int kNumWarps = kNumThreads / 32;
constexpr int kNumWarpSlots = 1024;                // (column, value) slots per warp: 8 KB
constexpr int kNumWarpCap = kNumWarpSlots / 2;     // products per row for the warp path
constexpr int kNumHeavyThreads = 1024;             // block-per-row pass
constexpr int kNumBlockSlots = 16384;              // block table: 64 KB of columns + 64 KB of values
constexpr int kNumBlockCap = kNumBlockSlots / 2;   // products per row for the block table
constexpr int kNumDenseCols = 49152;               // columns per dense pass (192 KB of values)
constexpr int kNumDenseWords = kNumDenseCols / 32;  // its occupancy bitmap (6 KB)
constexpr int kPoolStripes = 64;                   // pool mode: bump pointers (one per workspace slot)
constexpr int kNumUnroll = 4;                      // block pass: products per lane loaded at once

constexpr size_t kNumRowsSmem = (size_t)kNumWarps * kNumWarpSlots * (sizeof(int) + sizeof(float));
constexpr size_t kNumBlockTableSmem = (size_t)kNumBlockSlots * (sizeof(int) + sizeof(float));
constexpr size_t kNumDenseSmem = (size_t)kNumDenseCols * sizeof(float) + kNumDenseWords * sizeof(unsigned);
// the block-per-row pass runs on its own, so it takes shared memory over L1
constexpr size_t kNumHeavySmem = kNumDenseSmem > kNumBlockTableSmem ? kNumDenseSmem : kNumBlockTableSmem;

enum NumMode { kNumInto = 0, kNumCompact = 1 };

struct NumArgs {
  long long M, K, N, nnzA, nnzB;
  const int* a_rpt;
  const int* a_col;
  const float* a_val;
  const int* b_rpt;
  const int* b_col;
  const float* b_val;
  const long long* alloc;  // [M + 1] per-row shares of the allocation, or null: one pool
  int* c_col;              // the allocation (alloc_cap entries)
  float* c_val;
  long long alloc_cap;
  int pool_stripes;        // pool mode: stripes of the pool in use (1 .. kPoolStripes)
  Slot* slots;             // pool mode: slots[s].pool is stripe s's bump pointer
  long long* row_start;    // [M] where each row was written in the allocation (-1: not written);
                           // written by kNumInto, read by kNumCompact
  int* nnz_row;            // [M] exact nnz per row: written by kNumInto, read by kNumCompact
  const long long* out_rpt;  // kNumCompact: [M + 1] exact offsets
  int* out_col;              // kNumCompact: the exact CSR's entries (out_cap of them)
  float* out_val;
  long long out_cap;
  int mode;
  unsigned* heavy_count;     // block-per-row queue: heavy[h] = row + 1, 0 = empty
  int* heavy;
  long long heavy_cap;
  unsigned* status;          // SPGEMM_STATUS_* bits
  spgemm_numeric_result_t* res;
};

// B's row k as [s, s + len), bounds checked (bad ids count as empty).
__device__ __forceinline__ void num_b_row(const NumArgs& a, int k, long long& s, long long& len, bool& bad) {
  s = 0;
  len = 0;
  if ((unsigned)k >= (unsigned long long)a.K) {
    bad = true;
    return;
  }
  long long b = __ldg(a.b_rpt + k), e = __ldg(a.b_rpt + k + 1);
  if (!clamp_range(b, e, a.nnzB)) bad = true;
  s = b;
  len = e - b;
}

// Slot of `key` in an open-addressing table of 2^lg slots (keys -1 = empty),
// inserting it if absent; -1 only if the table is full (it holds at most half
// as many keys as slots, so the probe ends).
__device__ __forceinline__ int num_slot(int* keys, int lg, int key) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = (uint32_t)key * 0x9E3779B1u >> (32 - lg);
  for (uint32_t it = 0; it <= mask; ++it) {
    const int old = atomicCAS(&keys[h], -1, key);
    if (old == -1 || old == key) return (int)h;
    h = (h + 1) & mask;
  }
  return -1;
}

// Room for a row whose share of the allocation is [d, d1), cut to what the
// arrays hold (alloc_cap entries).
__device__ __forceinline__ long long num_alloc_room(const NumArgs& a, long long d, long long d1) {
  const long long cap = d1 - d;
  if (d < 0 || cap <= 0 || d >= a.alloc_cap) return 0;
  return min(cap, a.alloc_cap - d);
}

// A row's own bounds in its target when it has them before its size is known
// (its share of the allocation, or its exact offsets); none in pool mode.
// Read when the row starts, so that the round trip overlaps the row's work.
struct NumBounds {
  long long lo, hi;
  bool have;
};
__device__ __forceinline__ NumBounds num_bounds(const NumArgs& a, int row) {
  NumBounds b{0, 0, false};
  if (a.mode != kNumInto) {
    b = NumBounds{a.out_rpt[row], a.out_rpt[row + 1], true};
  } else if (a.alloc) {
    b = NumBounds{a.alloc[row], a.alloc[row + 1], true};
  }
  return b;
}

// Pool mode: n entries from a stripe of the pool (the row's stripe first);
// returns their first position, or -1 when no stripe has room.
__device__ long long num_pool_take(const NumArgs& a, int row, long long n) {
  if (n == 0) return 0;
  const int S = a.pool_stripes;
  const long long size = (a.alloc_cap + S - 1) / S;
  const int s0 = (int)((((unsigned)row * 2654435761u) >> 16) % (unsigned)S);
  for (int k = 0; k < S; ++k) {
    const int st = (s0 + k) % S;
    const long long base = (long long)st * size, len = min(a.alloc_cap - base, size);
    if (len < n) continue;
    unsigned long long* ctr = &a.slots[st].pool;
    if ((long long)*reinterpret_cast<volatile unsigned long long*>(ctr) + n > len) continue;  // full
    const long long pos = (long long)atomicAdd(ctr, (unsigned long long)n);
    if (pos + n <= len) return base + pos;
  }
  return -1;
}

// Where a row of n entries goes: its first entry's index and its capacity in
// the target (0 when it does not fit).  Called by one thread per row; in the
// numeric pass it also records the row's start (or -1).
struct NumTarget {
  long long dst, cap;
  int* col;
  float* val;
  long long limit;  // the target arrays' length: nothing is written at or past it
};

__device__ NumTarget num_target(const NumArgs& a, int row, long long n, const NumBounds* pre = nullptr) {
  NumTarget t;
  const NumBounds b = pre && pre->have ? *pre : num_bounds(a, row);
  if (a.mode == kNumInto) {
    t.col = a.c_col;
    t.val = a.c_val;
    t.limit = a.alloc_cap;
    if (a.alloc) {
      t.dst = b.lo;
      t.cap = num_alloc_room(a, b.lo, b.hi);
    } else {
      t.dst = num_pool_take(a, row, n);
      t.cap = t.dst >= 0 ? n : 0;
    }
    const bool fits = t.dst >= 0 && n <= t.cap;
    a.row_start[row] = fits ? t.dst : -1;
    if (!fits) t.cap = 0;
  } else {
    t.dst = b.lo;
    t.cap = b.hi - b.lo;
    t.col = a.out_col;
    t.val = a.out_val;
    t.limit = a.out_cap;
  }
  if (t.cap < 0 || t.dst < 0) {
    t.cap = 0;
    t.dst = 0;
  }
  return t;
}

__device__ __forceinline__ void num_put(const NumTarget& t, long long pos, int col, float val) {
  const long long q = t.dst + pos;
  if (pos < t.cap && q < t.limit) {
    t.col[q] = col;
    t.val[q] = val;
  }
}

// Queues a row for the block-per-row pass (lane 0 of the calling warp).
__device__ __forceinline__ void num_queue(const NumArgs& a, int row) {
  const unsigned h = atomicAdd(a.heavy_count, 1u);
  if (h < (unsigned long long)a.heavy_cap) flag_store(reinterpret_cast<unsigned*>(a.heavy + h), (unsigned)(row + 1));
  else atomicOr(a.status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);  // the queue holds every row: cannot happen
}

// One warp computes row `row` into its target (when it fits), with a table of
// kNumWarpSlots (column, value) pairs.  Returns the row's nnz, or -1 when the
// row has more than kNumWarpCap products and was queued for a block.
__device__ long long num_row_warp(const NumArgs& a, int row, int* keys, float* vals, bool& bad) {
  const int lane = threadIdx.x & 31;
  NumBounds pre{0, 0, false};
  if (lane == 0) pre = num_bounds(a, row);
  long long rb = __ldg(a.a_rpt + row), re = __ldg(a.a_rpt + row + 1);
  if (!clamp_range(rb, re, a.nnzA)) bad = true;
  // the FLOP of the row; the first 32 entries' B rows and values stay in
  // registers for the products loop
  long long flop = 0, s0 = 0, len0 = 0;
  float av0 = 0.0f;
  for (long long j = rb + lane; j < re; j += 32) {
    long long s, len;
    num_b_row(a, __ldg(a.a_col + j), s, len, bad);
    if (j - rb < 32) {
      s0 = s;
      len0 = len;
      av0 = __ldg(a.a_val + j);
    }
    flop += len;
  }
  flop = warp_sum(flop);
  if (flop > kNumWarpCap) {
    if (lane == 0) num_queue(a, row);
    return -1;
  }
  const int lg = max(5, ceil_log2((uint32_t)(2 * flop)));
  const int P = 1 << lg;
  for (int i = lane; i < P; i += 32) {
    keys[i] = -1;
    vals[i] = 0.0f;
  }
  __syncwarp();
  // products, 32 entries of A at a time: lane p of a step takes product p
  for (long long g = rb; g < re; g += 32) {
    long long s = s0, len = len0;
    float av = av0;
    if (g != rb) {
      s = 0;
      len = 0;
      av = 0.0f;
      if (g + lane < re) {
        num_b_row(a, __ldg(a.a_col + g + lane), s, len, bad);
        av = __ldg(a.a_val + g + lane);
      }
    }
    const int ilen = (int)len;
    const int inc = warp_incl_scan(ilen);
    const int excl = inc - ilen;
    const long long base = s - excl;  // B position of product p of this entry = base + p
    const int T = __shfl_sync(kFull, inc, 31);
    for (int pb = 0; pb < T; pb += 128) {
      int col[4];
      float pv[4];
      bool act[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int p = pb + 32 * u + lane;
        int o = 0;  // owner: the last lane whose exclusive prefix is <= p
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const int ex = __shfl_sync(kFull, excl, o + step);
          if (ex <= p) o += step;
        }
        const long long ob = __shfl_sync(kFull, base, o);
        const float oa = __shfl_sync(kFull, av, o);
        act[u] = p < T;
        col[u] = 0;
        pv[u] = 0.0f;
        if (act[u]) {
          col[u] = __ldg(a.b_col + ob + p);
          pv[u] = oa * __ldg(a.b_val + ob + p);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!act[u]) continue;
        if ((unsigned)col[u] >= (unsigned long long)a.N) {
          bad = true;
          continue;
        }
        const int h = num_slot(keys, lg, col[u]);
        if (h >= 0) atomicAdd(&vals[h], pv[u]);
      }
    }
  }
  __syncwarp();
  // count, then write when the row fits its target
  int nnz = 0;
  for (int i0 = 0; i0 < P; i0 += 32) nnz += __popc(__ballot_sync(kFull, keys[i0 + lane] != -1));
  NumTarget t{};
  if (lane == 0) t = num_target(a, row, nnz, &pre);
  t.dst = __shfl_sync(kFull, t.dst, 0);
  t.cap = __shfl_sync(kFull, t.cap, 0);
  t.limit = __shfl_sync(kFull, t.limit, 0);
  t.col = a.mode == kNumInto ? a.c_col : a.out_col;
  t.val = a.mode == kNumInto ? a.c_val : a.out_val;
  if (nnz <= t.cap) {
    int pos = 0;
    for (int i0 = 0; i0 < P; i0 += 32) {
      const int k = keys[i0 + lane];
      const unsigned bal = __ballot_sync(kFull, k != -1);
      if (k != -1) num_put(t, pos + __popc(bal & ((1u << lane) - 1u)), k, vals[i0 + lane]);
      pos += __popc(bal);
    }
  }
  __syncwarp();
  return nnz;
}

// Per-entry staging of the block-per-row pass: A's entries are taken
// kNumHeavyThreads at a time; ex = exclusive product offsets, bs = B position
// of product 0 of the entry minus its offset, av = the entry's value.
struct NumHeavySmem {
  long long ex[kNumHeavyThreads + 1];
  long long bs[kNumHeavyThreads];
  float av[kNumHeavyThreads];
  long long red[kNumHeavyThreads / 32 + 1];
  long long tgt[3];  // the row's target, from thread 0: dst, cap, limit
};

// Calls f(col, value) for every product of A's row [rb, re) once, by the whole
// block (warp w takes a contiguous run of each group's products, lanes
// interleaved for coalesced reads of B).  Without VAL, B's values are not read
// (f gets 0).
template <bool VAL = true, class F>
__device__ void num_block_products(const NumArgs& a, long long rb, long long re, NumHeavySmem& sm, bool& bad,
                                   F&& f) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  for (long long g = rb; g < re; g += kNumHeavyThreads) {
    long long s = 0, len = 0;
    float av = 0.0f;
    if (g + t < re) {
      num_b_row(a, __ldg(a.a_col + g + t), s, len, bad);
      av = __ldg(a.a_val + g + t);
    }
    long long T;
    const long long excl = block_excl_scan<kNumHeavyThreads>(len, sm.red, &T);
    sm.ex[t] = excl;
    sm.bs[t] = s - excl;
    sm.av[t] = av;
    const int nent = (int)min((long long)kNumHeavyThreads, re - g);
    if (t == 0) sm.ex[nent] = T;
    __syncthreads();
    const long long Q = ((T + 32 * 32 - 1) / (32 * 32)) * 32;
    const long long p_beg = (long long)warp * Q, p_end = min(T, p_beg + Q);
    long long p = p_beg + lane;
    if (p_beg < p_end) {
      int lo_i = 0, hi_i = nent;  // owner of p: the last entry with ex <= p
      while (hi_i - lo_i > 1) {
        const int mid = (lo_i + hi_i) >> 1;
        if (sm.ex[mid] <= p) lo_i = mid; else hi_i = mid;
      }
      int o = lo_i;
      // kNumUnroll products per lane are loaded before any is used
      for (; p < p_end; p += 32 * kNumUnroll) {
        int col[kNumUnroll];
        float pv[kNumUnroll];
#pragma unroll
        for (int u = 0; u < kNumUnroll; ++u) {
          const long long pu = p + 32 * u;
          col[u] = -1;
          pv[u] = 0.0f;
          if (pu < p_end) {
            while (o + 1 < nent && sm.ex[o + 1] <= pu) ++o;
            const long long q = sm.bs[o] + pu;
            col[u] = __ldg(a.b_col + q);
            if (VAL) pv[u] = sm.av[o] * __ldg(a.b_val + q);
          }
        }
#pragma unroll
        for (int u = 0; u < kNumUnroll; ++u) {
          if (p + 32 * u >= p_end) continue;
          if ((unsigned)col[u] >= (unsigned long long)a.N) {
            bad = true;
            continue;
          }
          f(col[u], pv[u]);
        }
      }
    }
    __syncthreads();
  }
}

// One block computes a queued row into its target; returns its nnz.
__device__ long long num_row_block(const NumArgs& a, int row, NumHeavySmem& sm, unsigned char* dyn, bool& bad) {
  const int t = threadIdx.x;
  long long rb = __ldg(a.a_rpt + row), re = __ldg(a.a_rpt + row + 1);
  if (!clamp_range(rb, re, a.nnzA)) bad = true;
  long long fl = 0;
  for (long long j = rb + t; j < re; j += kNumHeavyThreads) {
    long long s, len;
    num_b_row(a, __ldg(a.a_col + j), s, len, bad);
    fl += len;
  }
  const long long flop = block_sum<kNumHeavyThreads>(fl, sm.red);
  // the row's target, from thread 0, once its size n is known
  auto target = [&](long long n) {
    if (t == 0) {
      const NumTarget x = num_target(a, row, n);
      sm.tgt[0] = x.dst;
      sm.tgt[1] = x.cap;
      sm.tgt[2] = x.limit;
    }
    __syncthreads();
    NumTarget x;
    x.dst = sm.tgt[0];
    x.cap = sm.tgt[1];
    x.limit = sm.tgt[2];
    x.col = a.mode == kNumInto ? a.c_col : a.out_col;
    x.val = a.mode == kNumInto ? a.c_val : a.out_val;
    return x;
  };
  if (flop <= kNumBlockCap) {
    int* keys = reinterpret_cast<int*>(dyn);
    float* vals = reinterpret_cast<float*>(dyn + (size_t)kNumBlockSlots * sizeof(int));
    const int lg = max(5, ceil_log2((uint32_t)(2 * flop)));
    const int P = 1 << lg;
    for (int i = t; i < P; i += kNumHeavyThreads) {
      keys[i] = -1;
      vals[i] = 0.0f;
    }
    __syncthreads();
    num_block_products(a, rb, re, sm, bad, [&](int col, float v) {
      const int h = num_slot(keys, lg, col);
      if (h >= 0) atomicAdd(&vals[h], v);
    });
    // thread t owns slots [t * per, (t + 1) * per)
    const int per = (P + kNumHeavyThreads - 1) / kNumHeavyThreads;
    const int s0 = min(P, t * per), s1 = min(P, s0 + per);
    long long c = 0;
    for (int i = s0; i < s1; ++i) c += keys[i] != -1;
    long long nnz;
    long long pos = block_excl_scan<kNumHeavyThreads>(c, sm.red, &nnz);
    const NumTarget tg = target(nnz);
    if (nnz <= tg.cap)
      for (int i = s0; i < s1; ++i)
        if (keys[i] != -1) num_put(tg, pos++, keys[i], vals[i]);
    __syncthreads();
    return nnz;
  }
  // dense passes over B's columns, kNumDenseCols at a time (entries in
  // ascending column order).  A share or an exact slot is known up front: one
  // sweep writes and counts.  A place in the pool needs the row's size first:
  // one sweep counts, the next writes.
  float* acc = reinterpret_cast<float*>(dyn);
  unsigned* bits = reinterpret_cast<unsigned*>(dyn + (size_t)kNumDenseCols * sizeof(float));
  auto sweep = [&](bool write, const NumTarget& tg) -> long long {
    long long nnz = 0;
    for (long long lo = 0; lo < a.N; lo += kNumDenseCols) {
      const long long hi = min(a.N, lo + (long long)kNumDenseCols);
      for (int i = t; i < kNumDenseCols; i += kNumHeavyThreads) acc[i] = 0.0f;
      for (int i = t; i < kNumDenseWords; i += kNumHeavyThreads) bits[i] = 0u;
      __syncthreads();
      auto mark = [&](int col, float v) {
        if (col >= lo && col < hi) {
          const int o = (int)(col - lo);
          if (write) atomicAdd(&acc[o], v);
          atomicOr(&bits[o >> 5], 1u << (o & 31));
        }
      };
      if (write) num_block_products<true>(a, rb, re, sm, bad, mark);
      else num_block_products<false>(a, rb, re, sm, bad, mark);
      // thread t owns bitmap words [t * per, (t + 1) * per): ascending columns
      constexpr int per = (kNumDenseWords + kNumHeavyThreads - 1) / kNumHeavyThreads;
      const int w0 = min(kNumDenseWords, t * per), w1 = min(kNumDenseWords, w0 + per);
      long long c = 0;
      for (int w = w0; w < w1; ++w) c += __popc(bits[w]);
      long long cnt;
      long long pos = nnz + block_excl_scan<kNumHeavyThreads>(c, sm.red, &cnt);
      if (write) {
        for (int w = w0; w < w1; ++w) {
          unsigned m = bits[w];
          while (m) {
            const int b = __ffs(m) - 1;
            m &= m - 1;
            const int o = w * 32 + b;
            num_put(tg, pos++, (int)(lo + o), acc[o]);
          }
        }
      }
      nnz += cnt;
      __syncthreads();
    }
    return nnz;
  };
  long long nnz;
  if (a.mode == kNumCompact) {  // the exact slot is known
    nnz = sweep(true, target(a.nnz_row[row]));
  } else if (a.alloc) {  // a share: written while it fits, dropped if the row turns out larger
    const NumTarget tg = target(0);
    nnz = sweep(true, tg);
    if (t == 0 && nnz > tg.cap) a.row_start[row] = -1;
  } else {  // the pool: the size first, then the entries
    nnz = sweep(false, NumTarget{});
    const NumTarget tg = target(nnz);
    if (tg.cap >= nnz && nnz > 0) sweep(true, tg);
  }
  return nnz;
}

// Records one computed row: its nnz (kNumInto) and, when it was not written
// (row_start = -1), the overflow (per-thread sums, added at the end).
struct NumTally {
  long long nnz = 0, over_rows = 0, over_nnz = 0;
  __device__ void add(const NumArgs& a, int row, long long nnz_row) {
    nnz += nnz_row;
    if (a.mode == kNumInto) {
      a.nnz_row[row] = (int)nnz_row;
      if (a.row_start[row] < 0) {
        over_rows += 1;
        over_nnz += nnz_row;
      }
    }
  }
};

// One thread per warp (rows pass) or per block (heavy pass) adds its tally to
// the result record.
__device__ void num_publish(const NumArgs& a, const NumTally& tl, bool bad) {
  if (bad) atomicOr(a.status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
  if (a.mode != kNumInto) return;
  if (tl.nnz) atomicAdd(reinterpret_cast<unsigned long long*>(&a.res->nnz_total), (unsigned long long)tl.nnz);
  if (tl.over_rows) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.res->overflow_rows), (unsigned long long)tl.over_rows);
    atomicAdd(reinterpret_cast<unsigned long long*>(&a.res->overflow_nnz), (unsigned long long)tl.over_nnz);
  }
}

// Warp-per-row pass over all rows (grid-stride over warps).
__global__ void __launch_bounds__(kNumThreads) k_numeric_rows(NumArgs a) {
  extern __shared__ __align__(16) unsigned char num_dyn[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* keys = reinterpret_cast<int*>(num_dyn) + warp * kNumWarpSlots;
  float* vals = reinterpret_cast<float*>(num_dyn + (size_t)kNumWarps * kNumWarpSlots * sizeof(int)) + warp * kNumWarpSlots;
  const long long gw = (long long)blockIdx.x * kNumWarps + warp, nw = (long long)gridDim.x * kNumWarps;
  NumTally tl;
  bool bad = false;
  if (a.mode == kNumCompact) {
    // only the rows that overflowed their allocation are computed again (the
    // others are moved by k_numeric_move): 32 rows checked at a time
    for (long long r0 = gw * 32; r0 < a.M; r0 += nw * 32) {
      const long long r = r0 + lane;
      bool over = false;
      if (r < a.M) {
        const int n = a.nnz_row[r];
        if (a.out_rpt[r] + n > a.out_cap) bad = true;  // exact arrays too short
        over = a.row_start[r] < 0;
      }
      unsigned m = __ballot_sync(kFull, over);
      while (m) {
        const int l = __ffs(m) - 1;
        m &= m - 1;
        num_row_warp(a, (int)(r0 + l), keys, vals, bad);
      }
    }
  } else {
    for (long long r = gw; r < a.M; r += nw) {
      const long long nnz = num_row_warp(a, (int)r, keys, vals, bad);
      if (nnz >= 0 && lane == 0) tl.add(a, (int)r, nnz);
    }
  }
  bad = __any_sync(kFull, bad);
  if (lane == 0) num_publish(a, tl, bad);
}

// Compaction, the rows that were written: the exact layout's positions
// [0, out_rpt[M]) are split evenly among the warps; warp w finds the row of
// its first position (a 32-way search over out_rpt), then lane l takes
// positions q0 + l, q0 + l + 32, ..., following the row boundaries with a
// cursor, and copies entry q - out_rpt[row] of the row from row_start[row].
// Positions of rows that overflowed are left to the recomputation.
constexpr int kMoveThreads = 256;
constexpr int kMoveUnroll = 8;
__global__ void __launch_bounds__(kMoveThreads) k_numeric_move(NumArgs a) {
  const int lane = threadIdx.x & 31;
  const long long nw = ((long long)gridDim.x * kMoveThreads) >> 5;
  const long long w = ((long long)blockIdx.x * kMoveThreads + threadIdx.x) >> 5;
  const long long Z = a.out_rpt[a.M];
  const long long q0 = Z * w / nw, q1 = Z * (w + 1) / nw;
  if (q0 >= q1) return;
  // the last row r with out_rpt[r] <= q0 (rows with no entries are skipped by the cursor)
  long long lo = 0, hi = a.M;  // out_rpt[lo] <= q0 < out_rpt[hi] (q0 < Z)
  while (hi - lo > 1) {
    const long long step = (hi - lo + 31) / 32;
    const long long x = lo + (long long)(lane + 1) * step;
    const bool le = x < hi && a.out_rpt[x] <= q0;
    const unsigned b = __ballot_sync(kFull, le);
    const long long nlo = lo + (long long)__popc(b) * step;
    hi = min(hi, nlo + step);
    lo = nlo;
  }
  // the cursor row: its exact range [rs, re), whether it fitted its
  // allocation, and the shift from an exact position to its allocation
  long long row = lo;
  long long rs = a.out_rpt[row], re = a.out_rpt[row + 1];
  bool fits = false;
  long long shift = 0;
  auto locate = [&]() {
    const long long st = a.row_start[row];
    fits = st >= 0 && st + (re - rs) <= a.alloc_cap;
    shift = st - rs;
  };
  locate();
  for (long long qb = q0; qb < q1; qb += 32 * kMoveUnroll) {
    int cv[kMoveUnroll];
    float vv[kMoveUnroll];
    long long dq[kMoveUnroll];
#pragma unroll
    for (int u = 0; u < kMoveUnroll; ++u) {
      const long long q = qb + lane + 32 * u;
      dq[u] = -1;
      if (q < q1) {
        if (q >= re) {  // advance to the row holding q
          do {
            ++row;
            rs = re;
            re = a.out_rpt[row + 1];
          } while (q >= re);
          locate();
        }
        if (fits) {
          cv[u] = a.c_col[q + shift];
          vv[u] = a.c_val[q + shift];
          dq[u] = q;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kMoveUnroll; ++u) {
      if (dq[u] >= 0 && dq[u] < a.out_cap) {
        a.out_col[dq[u]] = cv[u];
        a.out_val[dq[u]] = vv[u];
      }
    }
  }
}

// Block-per-row pass over the queued rows.
__global__ void __launch_bounds__(kNumHeavyThreads) k_numeric_heavy(NumArgs a) {
  extern __shared__ __align__(16) unsigned char num_dyn[];
  __shared__ NumHeavySmem sm;
  const unsigned n_heavy = (unsigned)min((long long)*a.heavy_count, a.heavy_cap);
  NumTally tl;
  bool bad = false;
  for (unsigned h = blockIdx.x; h < n_heavy; h += gridDim.x) {
    const int row = a.heavy[h] - 1;
    __syncthreads();
    if (threadIdx.x == 0) a.heavy[h] = 0;
    if (row < 0 || row >= a.M) {
      bad = true;
      continue;
    }
    const long long nnz = num_row_block(a, row, sm, num_dyn, bad);
    if (threadIdx.x == 0) tl.add(a, row, nnz);
  }
  bad = __syncthreads_or(bad);
  if (threadIdx.x == 0) num_publish(a, tl, bad);
}

// Last step of a numeric call: the result record gets the status, the
// allocation total and (compaction) the exact total; the queue count is reset.
__global__ void k_numeric_finish(NumArgs a, unsigned* hdr_status) {
  volatile unsigned* hc = a.heavy_count;
  const unsigned n = *hc;
  if ((long long)n > a.heavy_cap) atomicOr(a.status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
  *hc = 0;
  if (a.mode == kNumInto) a.res->alloc_total = a.alloc ? (a.M > 0 ? a.alloc[a.M] : 0) : a.alloc_cap;
  for (int st = 0; st < kPoolStripes; ++st) a.slots[st].pool = 0;
  a.res->status |= (int)*reinterpret_cast<volatile unsigned*>(hdr_status);
  *reinterpret_cast<volatile unsigned*>(hdr_status) = 0u;
}

}  // namespace spg
