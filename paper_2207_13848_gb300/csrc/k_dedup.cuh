// Exact nnz of output rows by deduplicating their products (Sec. IV-B; the hash
// loop of Algorithm 2, Sec. V-B), re-designed for the GPU:
//   - rows with at most 32 products: one warp holds every product in a lane and
//     counts distinct column ids with __match_any_sync (no memory table);
//   - rows with at most heavy_thr products (kWarpCap by default): one warp,
//     open-addressing table in the warp's slice of shared memory;
//   - heavier rows are queued and handled by a whole thread block, with a
//     shared-memory hash table (up to kBlockHashCap products) or a bitmap over
//     the columns of B (split into column ranges when N exceeds its capacity).
// The count does not depend on the method used, so every path gives the same
// integers as the dense-marker count of the definition.
#pragma once

#include "common.cuh"

namespace spg {

// ---------------------------------------------------------------- parameters
constexpr int kDedupThreads = 256;            // threads per block of the warp-per-row pass
constexpr int kDedupWarps = kDedupThreads / 32;
constexpr int kWarpTable = 1024;              // hash slots per warp
constexpr int kListCap = 2048;                // sampled rows staged per block before processing
constexpr int kWarpCap = kWarpTable / 2;      // products per row for the warp path
constexpr int kHeavyThreads = 1024;           // threads per block of the heavy pass
constexpr int kBlockHashCap = 16384;          // products per row for the block hash path
constexpr int kBlockHashSlots = 2 * kBlockHashCap;
constexpr int kHeavyUnroll = 8;               // products per lane loaded at once in the heavy pass

enum RowSource { kSrcBernoulli = 0, kSrcDraws = 1, kSrcAllRows = 2 };

struct DedupArgs {
  int64_t M, K, N, nnzA, nnzB;
  const int* a_rpt;
  const int* a_col;
  const int* b_rpt;
  const int* b_col;
  int src;             // RowSource
  uint64_t seed;
  uint64_t threshold;  // Bernoulli threshold in [0, 2^32]
  int64_t n_cand;      // candidates: M (Bernoulli, all rows) or the number of draws
  int* nnz_out;        // all-rows mode: nnz per row (int32[M]); otherwise null
  Workspace ws;
  unsigned int* status;  // where SPGEMM_STATUS_* bits go (the header's, or a batch case's)
  // Rows with more than heavy_thr products (at most half the warp table) are
  // queued for the block-per-row pass: heavy[atomicAdd(heavy_count, 1)] =
  // heavy_base + row + 1, while fewer than heavy_cap entries are queued.  A
  // queue entry of 0 is empty; whoever takes an entry sets it back to 0, so the
  // queue is empty again after every call.
  unsigned int* heavy_count;
  int* heavy;
  long long heavy_cap;
  int heavy_base;
  int heavy_thr;
  // Optional second queue for the largest rows (more than big_thr products),
  // filled from the top of the same array: heavy[heavy_cap - 1 -
  // atomicAdd(big_count, 1)].  A consumer that takes these first keeps the
  // longest rows from being counted last.  big_count == null: one queue.
  unsigned int* big_count;
  long long big_thr;
};

__device__ __forceinline__ uint32_t mix_key(int key) { return (uint32_t)key * 0x9E3779B1u; }

// Inserts `key` into an open-addressing table of 2^lg slots initialised to -1.
// Returns 1 if the key was not present.  The table always has a free slot (it
// holds at most half as many keys as slots), so the probe ends; the loop bound
// only guards against a corrupted table.
__device__ __forceinline__ int table_insert(int* tbl, int lg, int key) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = mix_key(key) >> (32 - lg);
  for (uint32_t it = 0; it <= mask; ++it) {
    int old = atomicCAS(&tbl[h], -1, key);
    if (old == -1) return 1;
    if (old == key) return 0;
    h = (h + 1) & mask;
  }
  return 0;
}

__device__ __forceinline__ int ceil_log2(uint32_t x) { return x <= 1 ? 0 : 32 - __clz(x - 1); }

// Reads B's row k as [s, s+len), with every bound checked; bad ids count as empty.
__device__ __forceinline__ void b_row(const DedupArgs& a, int k, long long& s, long long& len,
                                      bool& bad) {
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

// One warp computes flop and (unless the row is heavy) nnz of `row`, with a
// table `tbl` of at least 2 * a.heavy_thr slots.  Returns nnz, or -1 when the
// row was queued for the heavy pass.  flop is returned through *flop_out (same
// value on every lane).
__device__ long long dedup_row_warp(const DedupArgs& a, int row, int* tbl, long long* flop_out) {
  const int lane = threadIdx.x & 31;
  bool bad = false;
  long long rb = __ldg(a.a_rpt + row), re = __ldg(a.a_rpt + row + 1);
  if (!clamp_range(rb, re, a.nnzA)) bad = true;
  const long long nent = re - rb;

  // FLOP of the row (Algorithm 1 restricted to one row).  The first group of 32
  // entries is kept in registers for the small path.
  long long s0 = 0, len0 = 0, flop = 0;
  for (long long j = rb + lane; j < re; j += 32) {
    long long s, len;
    b_row(a, __ldg(a.a_col + j), s, len, bad);
    if (j - rb < 32) {
      s0 = s;
      len0 = len;
    }
    flop += len;
  }
  flop = warp_sum(flop);
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(a.status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
  *flop_out = flop;
  if (flop == 0) return 0;

  if (nent <= 32 && flop <= 32) {
    // Every product in one lane: lane p takes product p.
    const int len = (int)len0;
    const int inc = warp_incl_scan(len);
    const int excl = inc - len;
    const int base = (int)s0 - excl;  // column position = base of the owner + p
    const int p = lane;
    int o = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1) {
      int ex = __shfl_sync(kFull, excl, o + step);
      if (ex <= p) o += step;
    }
    const int ob = __shfl_sync(kFull, base, o);
    const bool act = p < flop;
    const unsigned mask = __ballot_sync(kFull, act);
    bool leader = false;
    if (act) {
      int col = __ldg(a.b_col + ob + p);
      unsigned m = __match_any_sync(mask, col);
      leader = (__ffs(m) - 1) == lane;
    }
    return __popc(__ballot_sync(kFull, leader));
  }

  if (flop <= a.heavy_thr) {
    const int lg = max(6, ceil_log2((uint32_t)(2 * flop)));
    const int P = 1 << lg;
    for (int i = lane; i < P; i += 32) tbl[i] = -1;
    __syncwarp();
    int cnt = 0;
    for (long long g = rb; g < re; g += 32) {
      long long s = s0, len = len0;  // the first group was read by the FLOP loop
      if (g != rb) {
        s = 0;
        len = 0;
        if (g + lane < re) b_row(a, __ldg(a.a_col + g + lane), s, len, bad);
      }
      const int ilen = (int)len;
      const int inc = warp_incl_scan(ilen);
      const int excl = inc - ilen;
      const int base = (int)s - excl;
      const int T = __shfl_sync(kFull, inc, 31);
      for (int pb = 0; pb < T; pb += 128) {
        int col[4];
        bool act[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int p = pb + 32 * u + lane;
          int o = 0;
#pragma unroll
          for (int step = 16; step > 0; step >>= 1) {
            int ex = __shfl_sync(kFull, excl, o + step);
            if (ex <= p) o += step;
          }
          const int ob = __shfl_sync(kFull, base, o);
          act[u] = p < T;
          col[u] = act[u] ? __ldg(a.b_col + ob + p) : 0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (act[u]) cnt += table_insert(tbl, lg, col[u]);
      }
    }
    __syncwarp();
    return warp_sum(cnt);
  }

  if (lane == 0) {
    const unsigned entry = (unsigned)(a.heavy_base + row + 1);
    if (a.big_count && flop > a.big_thr) {
      const unsigned h = atomicAdd(a.big_count, 1u);
      if (h < (unsigned long long)a.heavy_cap)
        flag_store(reinterpret_cast<unsigned*>(a.heavy + (a.heavy_cap - 1 - h)), entry);
    } else {
      const unsigned h = atomicAdd(a.heavy_count, 1u);
      if (h < (unsigned long long)a.heavy_cap) flag_store(reinterpret_cast<unsigned*>(a.heavy + h), entry);
    }
  }
  return -1;
}

// Pass 1: candidates -> rows (sample or all rows), warp-per-row deduplication.
// Each block takes a contiguous slice of the candidates, hashes them and stages
// the selected rows in shared memory (up to kListCap at a time), then hands the
// staged rows to its warps, so the warps' per-row memory latencies overlap.
__global__ void __launch_bounds__(kDedupThreads) k_dedup_rows(DedupArgs a) {
  extern __shared__ int dyn[];
  int* tbl = dyn + (threadIdx.x >> 5) * kWarpTable;
  __shared__ int list[kListCap];
  __shared__ int list_n;
  __shared__ long long red[kDedupWarps + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const long long c_beg = (long long)blockIdx.x * a.n_cand / gridDim.x;
  const long long c_end = (long long)(blockIdx.x + 1) * a.n_cand / gridDim.x;
  long long f_loc = 0, z_loc = 0, s_loc = 0;
  long long base = c_beg;
  while (base < c_end) {
    if (threadIdx.x == 0) list_n = 0;
    __syncthreads();
    // stage selected rows until the list could overflow or the slice ends; n
    // (the same in every thread, from the barrier's count) is the number staged
    int n = 0;
    for (;;) {
      const long long cand = base + threadIdx.x;
      bool take = false;
      int row = 0;
      if (cand < c_end) {
        if (a.src == kSrcAllRows) {
          take = true;
          row = (int)cand;
        } else if (a.src == kSrcBernoulli) {
          take = (uint64_t)sample_hash32(a.seed, (uint64_t)cand) < a.threshold;
          row = (int)cand;
        } else {
          take = true;
          row = (int)(((uint64_t)sample_hash32(a.seed, (uint64_t)cand) * (uint64_t)a.M) >> 32);
        }
      }
      const unsigned bal = __ballot_sync(kFull, take);
      int wbase = 0;
      if (lane == 0 && bal) wbase = atomicAdd(&list_n, __popc(bal));
      wbase = __shfl_sync(kFull, wbase, 0);
      if (take) list[wbase + __popc(bal & ((1u << lane) - 1u))] = row;
      base += kDedupThreads;
      n += __syncthreads_count(take);
      if (base >= c_end || n > kListCap - kDedupThreads) break;
    }
    for (int e = warp; e < n; e += kDedupWarps) {
      const int r = list[e];
      long long flop;
      long long nnz = dedup_row_warp(a, r, tbl, &flop);
      if (lane == 0) {
        f_loc += flop;
        s_loc += 1;
        if (nnz >= 0) {
          z_loc += nnz;
          if (a.nnz_out) a.nnz_out[r] = (int)nnz;
        }
      }
    }
    __syncthreads();
  }
  const long long f = block_sum<kDedupThreads>(f_loc, red);
  const long long z = block_sum<kDedupThreads>(z_loc, red);
  const long long s = block_sum<kDedupThreads>(s_loc, red);
  if (threadIdx.x == 0) {
    if (f) atomicAdd(&a.ws.hdr->f_acc, (unsigned long long)f);
    if (z) atomicAdd(&a.ws.hdr->z_acc, (unsigned long long)z);
    if (s) atomicAdd(&a.ws.hdr->s_acc, (unsigned long long)s);
  }
}

// Pass 2: one block per queued heavy row.  The products of the row are walked
// in groups of kHeavyThreads entries of A; inside a group each warp takes a
// contiguous run of products with its lanes interleaved (coalesced reads of B's
// column ids), and each lane tracks the entry its product belongs to.
struct HeavySmem {
  long long ex[kHeavyThreads + 1];  // exclusive product offsets of the group's entries
  long long bs[kHeavyThreads];      // B row start minus the entry's offset
  long long red[kHeavyThreads / 32 + 1];
};

// The products [p_beg, p_end) of one warp in a group of entries (sm.ex: the
// entries' exclusive product offsets, with ex[nent] = T; sm.bs: B row start
// minus the offset), lanes interleaved: each lane keeps its current entry's
// bounds in registers and reads shared memory only when it crosses into the
// next entry.  I is the index type: int when the group has fewer than 2^31
// products (every offset then fits), else long long.  kHeavyUnroll column ids
// per lane are loaded before any is used, so that many loads of each lane are
// in flight at once.
template <bool BITMAP, typename I>
__device__ __forceinline__ long long heavy_products(const DedupArgs& a, const HeavySmem& sm, int nent, I p_beg,
                                                    I p_end, unsigned* tab, int lg_or_words, long long lo,
                                                    long long hi, bool& bad) {
  const int lane = threadIdx.x & 31;
  long long cnt = 0;
  I p = p_beg + lane;
  if (p_beg >= p_end) return 0;
  // owner of p: last entry with ex <= p (binary search over nent entries)
  int lo_i = 0, hi_i = nent;  // ex[lo_i] <= p < ex[hi_i] (for p < T)
  while (hi_i - lo_i > 1) {
    const int mid = (lo_i + hi_i) >> 1;
    if (sm.ex[mid] <= (long long)p) lo_i = mid; else hi_i = mid;
  }
  int o = lo_i;
  I ex_next = (I)sm.ex[o + 1];  // o + 1 <= nent, and ex[nent] = T > every product
  // q[pu] is the column id of product pu while pu lies in entry o
  const int* q = a.b_col + sm.bs[o];
  const unsigned lo32 = (unsigned)lo, range = (unsigned)(hi - lo);
  // one bitmap pass over all of B's columns: an id outside it is out of range
  const bool whole = lo == 0 && hi == a.N;
  auto advance = [&](I pu) {  // into the entry holding pu (skipping empty ones)
    while (pu >= ex_next) {
      ++o;
      ex_next = (I)sm.ex[o + 1];
      q = a.b_col + sm.bs[o];
    }
  };
  auto put = [&](int c) {
    if (BITMAP) {
      const unsigned off = (unsigned)c - lo32;
      if (off < range) {
        atomicOr(&tab[off >> 5], __funnelshift_l(0u, 1u, off));  // bit off & 31
      } else if (whole || (unsigned)c >= (unsigned long long)a.N) {
        bad = true;
      }
    } else {
      cnt += table_insert(reinterpret_cast<int*>(tab), lg_or_words, c);
    }
  };
  for (; p < p_end; p += 32 * kHeavyUnroll) {
    int col[kHeavyUnroll];
    if (p + 32 * (kHeavyUnroll - 1) < p_end) {  // the lane's whole step lies in the range
#pragma unroll
      for (int u = 0; u < kHeavyUnroll; ++u) {
        advance(p + 32 * u);
        col[u] = __ldg(q + (p + 32 * u));
      }
#pragma unroll
      for (int u = 0; u < kHeavyUnroll; ++u) put(col[u]);
    } else {
#pragma unroll
      for (int u = 0; u < kHeavyUnroll; ++u) {
        const I pu = p + 32 * u;
        col[u] = -1;
        if (pu < p_end) {
          advance(pu);
          col[u] = __ldg(q + pu);
        }
      }
#pragma unroll
      for (int u = 0; u < kHeavyUnroll; ++u)
        if (p + 32 * u < p_end) put(col[u]);
    }
  }
  return cnt;
}

// preloaded: the row is one group whose offsets heavy_row_flop left in sm.
template <bool BITMAP, bool COUNT = true>
__device__ long long heavy_count_pass(const DedupArgs& a, long long rb, long long re, HeavySmem& sm,
                                      unsigned* tab, int lg_or_words, long long lo, long long hi,
                                      bool& bad, bool preloaded = false) {
  const int t = threadIdx.x, warp = t >> 5;
  long long cnt = 0;
  for (long long g = rb; g < re; g += kHeavyThreads) {
    const int nent = (int)min((long long)kHeavyThreads, re - g);
    if (!preloaded) {
      long long s = 0, len = 0;
      if (g + t < re) b_row(a, __ldg(a.a_col + g + t), s, len, bad);
      long long Tg;
      const long long excl = block_excl_scan<kHeavyThreads>(len, sm.red, &Tg);
      sm.ex[t] = excl;
      sm.bs[t] = s - excl;
      if (t == 0) sm.ex[nent] = Tg;
      __syncthreads();
    }
    const long long T = sm.ex[nent];
    // warp w takes products [w*Q, (w+1)*Q), Q a multiple of 32
    const long long Q = ((T + 32 * 32 - 1) / (32 * 32)) * 32;
    const long long p_beg = (long long)warp * Q, p_end = min(T, p_beg + Q);
    if (T < (1ll << 31) - 4096) {  // every offset (and the lanes' lookahead) and B position fits 32 bits
      cnt += heavy_products<BITMAP, int>(a, sm, nent, (int)min(p_beg, T), (int)p_end, tab, lg_or_words, lo, hi,
                                         bad);
    } else {
      cnt += heavy_products<BITMAP, long long>(a, sm, nent, p_beg, p_end, tab, lg_or_words, lo, hi, bad);
    }
    __syncthreads();
  }
  if (!COUNT) return 0;  // bitmap left in tab for the caller
  if (BITMAP) {
    for (int i = t; i < lg_or_words; i += kHeavyThreads) cnt += __popc(tab[i]);
  }
  return block_sum<kHeavyThreads>(cnt, sm.red);
}

// Exact nnz of one heavy row by the whole block (kHeavyThreads threads): a
// shared hash table when the row has at most kBlockHashCap products, else a
// bitmap over B's columns, one column range of bitmap_words * 32 at a time.
// The row's A entry range [*rb, *re) and its FLOP, by the whole block.  With
// `preloaded` given, a row of at most kHeavyThreads entries leaves its
// entries' product offsets and B row starts in sm (*preloaded = true) for the
// counting pass, which then reads no row bounds again; they are visible to
// every thread after the caller's next __syncthreads.
__device__ long long heavy_row_flop(const DedupArgs& a, int row, HeavySmem& sm, long long* rb_out,
                                    long long* re_out, bool& bad, bool* preloaded = nullptr) {
  long long rb = __ldg(a.a_rpt + row), re = __ldg(a.a_rpt + row + 1);
  if (!clamp_range(rb, re, a.nnzA)) bad = true;
  *rb_out = rb;
  *re_out = re;
  if (preloaded) *preloaded = false;
  if (preloaded && re - rb <= kHeavyThreads) {
    const int t = threadIdx.x;
    long long s = 0, len = 0;
    if (rb + t < re) b_row(a, __ldg(a.a_col + rb + t), s, len, bad);
    long long T;
    const long long excl = block_excl_scan<kHeavyThreads>(len, sm.red, &T);
    sm.ex[t] = excl;
    sm.bs[t] = s - excl;
    if (t == 0) sm.ex[re - rb] = T;
    *preloaded = true;
    return T;
  }
  long long fl = 0;
  for (long long j = rb + threadIdx.x; j < re; j += kHeavyThreads) {
    long long s, len;
    b_row(a, __ldg(a.a_col + j), s, len, bad);
    fl += len;
  }
  return block_sum<kHeavyThreads>(fl, sm.red);
}

// Exact nnz of the row whose entries are [rb, re) and FLOP is flop, by the
// whole block (see heavy_row_nnz); preloaded as heavy_row_flop set it.
__device__ long long heavy_row_count(const DedupArgs& a, long long rb, long long re, long long flop,
                                     HeavySmem& sm, unsigned* tab, int bitmap_words, bool& bad,
                                     bool preloaded = false) {
  long long nnz = 0;
  if (flop <= kBlockHashCap) {
    const int lg = ceil_log2((uint32_t)(2 * flop));
    for (int i = threadIdx.x; i < (1 << lg); i += kHeavyThreads) tab[i] = 0xffffffffu;
    __syncthreads();
    nnz = heavy_count_pass<false>(a, rb, re, sm, tab, lg, 0, 0, bad, preloaded);
  } else {
    const long long range = (long long)bitmap_words * 32;
    for (long long lo = 0; lo < a.N; lo += range) {
      const long long hi = min((long long)a.N, lo + range);
      const int words = (int)((hi - lo + 31) / 32);
      for (int i = threadIdx.x; i < words; i += kHeavyThreads) tab[i] = 0u;
      __syncthreads();
      nnz += heavy_count_pass<true>(a, rb, re, sm, tab, words, lo, hi, bad, preloaded);
    }
  }
  return nnz;
}

__device__ long long heavy_row_nnz(const DedupArgs& a, int row, HeavySmem& sm, unsigned* tab,
                                   int bitmap_words, bool& bad, long long* flop_out = nullptr) {
  long long rb, re;
  bool pre;
  const long long flop = heavy_row_flop(a, row, sm, &rb, &re, bad, &pre);
  if (flop_out) *flop_out = flop;
  return heavy_row_count(a, rb, re, flop, sm, tab, bitmap_words, bad, pre);
}

__global__ void __launch_bounds__(kHeavyThreads) k_dedup_heavy(DedupArgs a, int bitmap_words) {
  extern __shared__ unsigned tab[];
  __shared__ HeavySmem sm;
  const unsigned n_heavy = (unsigned)min((long long)*a.heavy_count, a.heavy_cap);
  for (unsigned h = blockIdx.x; h < n_heavy; h += gridDim.x) {
    const int row = a.heavy[h] - 1;
    __syncthreads();
    if (threadIdx.x == 0) a.heavy[h] = 0;
    bool bad = false;
    const long long nnz = heavy_row_nnz(a, row, sm, tab, bitmap_words, bad);
    if (threadIdx.x == 0) {
      atomicAdd(&a.ws.hdr->z_acc, (unsigned long long)nnz);
      if (a.nnz_out) a.nnz_out[row] = (int)nnz;
    }
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(a.status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
  }
}

}  // namespace spg
