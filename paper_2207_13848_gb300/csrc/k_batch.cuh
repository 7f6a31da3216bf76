// Batched structure prediction: many independent predictions ("cases") of
// uneven sizes run as four persistent launches, each spanning every case of
// the batch (the method of each case is the single-case one: sample, exact nnz
// of the sampled rows, compression ratio, FLOP per row, prediction and scan):
//   kb_tables - the B row-length byte tables of all cases, with validation of
//               B's offsets;
//   kb_sample - the sample of every case and the exact nnz of its rows (warp
//               per row), from chunks of the concatenated candidate sequence
//               claimed one at a time; heavy rows of all cases share one queue;
//   kb_heavy  - the queued rows of all cases, one block per row, claimed one at
//               a time;
//   kb_flop   - FLOP per row, prediction and allocation offsets for every case,
//               from tiles of each case's merged sequence claimed one at a time;
//               the scan across a case's tiles is a decoupled look-back (Merrill
//               and Garland, "Single-pass parallel prefix scan with decoupled
//               look-back", NVIDIA tech. report NVR-2016-002).
// Work is claimed in increasing order and a tile only ever waits for tiles of
// lower index (its predecessors in the same case), which were claimed earlier
// by running blocks; so no wait can deadlock, whatever the number of blocks
// resident at once.  The kernel boundaries order the phases: every case's
// sample totals are final before the first FLOP tile starts.
#pragma once

#include "common.cuh"
#include "k_dedup.cuh"
#include "k_flop.cuh"

namespace spg {

// One case as planned on the host (written into the workspace by the prepare
// call).  Candidates, tiles and table blocks of all cases are numbered in case
// order.
struct BatchCase {
  const int* a_rpt;
  const int* a_col;
  const int* b_rpt;
  const int* b_col;
  long long M, K, N, nnzA, nnzB;
  unsigned long long seed, threshold;  // sample: hash seed and Bernoulli threshold
  long long n_cand;                    // candidates of the sample (rows or draws)
  long long cand_off;                  // index of the first one in the batch
  long long row_base;                  // batch-wide id of row 0 (heavy queue)
  long long tab_blk0;                  // first kb_tables block of the case
  int* pred;                           // [M]
  long long* offsets;                  // [M + 1]
  int* flop;                           // [M] or null
  spgemm_result_t* res;
  unsigned char* deg8;                 // [K] byte table, 16-byte aligned
  int src;                             // kSrcBernoulli or kSrcDraws
  int vec_ok;                          // A.col 16-byte aligned
  int tile0, ntiles;                   // FLOP tiles [tile0, tile0 + ntiles), ntiles >= 1
};

// Per-case accumulators; zero between runs (the case's last tile resets them).
struct alignas(64) CaseAcc {
  unsigned long long f;  // f*: FLOP of the sampled rows
  unsigned long long z;  // z*: nnz of the sampled rows
  unsigned long long s;  // |S|
  unsigned long long F;  // total FLOP
  unsigned int status;   // SPGEMM_STATUS_* bits
  unsigned int tiles_done;
  unsigned int pad[6];
};

struct alignas(128) BatchHeader {
  // work counters, zeroed before every run
  unsigned long long sample_ctr;  // candidate chunks claimed
  unsigned int heavy_count;       // rows queued for kb_heavy
  unsigned int heavy_ctr;         // queued rows claimed (the big rows' queue first, then the other)
  unsigned int tile_ctr;          // FLOP tiles claimed
  unsigned int tiles_done;        // FLOP tiles finished
  unsigned int big_count;         // rows of more than kBatchBigProducts products queued (from the top)
  unsigned int bar[2];            // grid barriers of the single-launch form (kb_all)
  unsigned int status;            // SPGEMM_STATUS_* bits of the whole run (a barrier that gave up)
  unsigned int pad0[6];
  // flag epoch of the last completed run (only grows)
  unsigned int epoch;
  unsigned int pad1[15];
};
constexpr size_t kBatchCounterBytes = 64;  // the leading counters of BatchHeader

// Sampled rows with more products than this go to a second queue that
// kb_heavy drains first, so the longest rows do not start last.
constexpr long long kBatchBigProducts = 1ll << 18;

constexpr int kTabRowsPerBlock = 4096;  // B rows per kb_tables block (4 per thread-word, 4 words per thread)
constexpr int kTabThreads = 256;

struct BatchArgs {
  BatchHeader* hdr;
  const BatchCase* cases;
  CaseAcc* acc;
  Slot* slots;               // [total_tiles]
  const int* tile_case;      // [total_tiles] case of each tile
  const int* chunk_case;     // [total_chunks] case of each chunk's first candidate
  const int* tab_case;       // [total_tab_blocks] case of each table block
  int* heavy;                // [heavy_cap] batch-wide row ids queued for kb_heavy
  int n_cases;
  int total_tiles;
  long long total_cand;
  long long total_chunks;
  long long sample_chunk;    // candidates per chunk
  long long heavy_cap;
  long long total_tab_blocks;  // units of kTabRowsPerBlock B rows (kb_tables blocks)
  int heavy_thr;             // products per row above which a row is queued
};

// Index of the last case i with key(i) <= x, for keys that never decrease with
// i and key(0) <= x: one warp, 32 probes per step.
template <class Key>
__device__ __forceinline__ int warp_last_le(int n, long long x, Key key) {
  const int lane = threadIdx.x & 31;
  int lo = 0, hi = n;  // key(lo) <= x, and key(hi) > x or hi == n
  while (hi - lo > 1) {
    const int step = (hi - lo + 31) / 32;
    const int p = lo + (lane + 1) * step;
    const bool le = p < hi && key(p) <= x;
    const int k = __popc(__ballot_sync(kFull, le));
    const int nlo = lo + k * step;
    hi = min(hi, nlo + step);
    lo = nlo;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// B row-length tables of every case (see k_degree_table), kTabRowsPerBlock
// rows of one case per block.
// ---------------------------------------------------------------------------
// Table unit tb (kTabRowsPerBlock rows of one case) by the nthreads threads of a
// block or group (thread `t` of them).
__device__ __forceinline__ void batch_table_unit(const BatchArgs& b, long long tb, int t, int nthreads) {
  const int c = __ldg(b.tab_case + tb);
  const BatchCase& k = b.cases[c];
  const long long K = k.K, nnzB = k.nnzB;
  const long long r0 = (tb - k.tab_blk0) * (long long)kTabRowsPerBlock;
  bool bad = false;
  for (long long k0 = r0 + t * 4; k0 < min(K, r0 + kTabRowsPerBlock); k0 += (long long)nthreads * 4) {
    unsigned word = 0;
    long long prev = __ldg(k.b_rpt + k0);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (k0 + u < K) {
        const long long next = __ldg(k.b_rpt + k0 + u + 1);
        long long d = next - prev;
        if (d < 0 || prev < 0 || next > nnzB) {
          bad = true;
          d = 0;
        }
        word |= (unsigned)(d < kDegEscape ? d : kDegEscape) << (8 * u);
        prev = next;
      }
    }
    *reinterpret_cast<unsigned*>(k.deg8 + k0) = word;
  }
  if (bad) atomicOr(&b.acc[c].status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
}

__global__ void __launch_bounds__(kTabThreads) kb_tables(BatchArgs b) {
  batch_table_unit(b, blockIdx.x, threadIdx.x, kTabThreads);
}

// Fills the per-warp (or per-block) deduplication arguments of case c.
__device__ __forceinline__ void batch_dedup_args(const BatchArgs& b, int c, DedupArgs& d) {
  const BatchCase& k = b.cases[c];
  d.M = k.M;
  d.K = k.K;
  d.N = k.N;
  d.nnzA = k.nnzA;
  d.nnzB = k.nnzB;
  d.a_rpt = k.a_rpt;
  d.a_col = k.a_col;
  d.b_rpt = k.b_rpt;
  d.b_col = k.b_col;
  d.src = k.src;
  d.seed = k.seed;
  d.threshold = k.threshold;
  d.n_cand = k.n_cand;
  d.nnz_out = nullptr;
  d.status = &b.acc[c].status;
  d.heavy_count = &b.hdr->heavy_count;
  d.heavy = b.heavy;
  d.heavy_cap = b.heavy_cap;
  d.heavy_base = (int)k.row_base;
  d.heavy_thr = b.heavy_thr;
  d.big_count = &b.hdr->big_count;
  d.big_thr = kBatchBigProducts;
}

// ---------------------------------------------------------------------------
// Samples of all cases and the exact nnz of their rows.  A block claims a
// chunk of the concatenated candidates, hashes them (each thread walking
// forward through the cases its candidates fall in), stages the selected
// (case, row) pairs in shared memory and hands them to its warps; a warp adds
// its rows' FLOP / nnz / count to the case's accumulators when it moves on to
// another case.  TABLE = hash slots per warp (>= 2 * heavy_thr).
// ---------------------------------------------------------------------------
// Shared state of the sampled-row pass for a block of NT threads.
template <int NT>
struct SampleShared {
  int list_row[kListCap];
  int list_case[kListCap];
  DedupArgs wa[NT / 32];
  int list_n;
  long long s_chunk;
  int s_case;
};

// The sampled-row pass by a block of NT threads: all of them stage candidates,
// the first AW warps count the staged rows; dyn holds AW warp tables of TABLE
// slots.
template <int TABLE, int NT, int AW = NT / 32>
__device__ __forceinline__ void batch_sample_phase(const BatchArgs& b, int* dyn, SampleShared<NT>& sh) {
  static_assert(kListCap > NT, "a staging round fits the list");
  int* list_row = sh.list_row;
  int* list_case = sh.list_case;
  DedupArgs* wa = sh.wa;
  int& list_n = sh.list_n;
  long long& s_chunk = sh.s_chunk;
  int& s_case = sh.s_case;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int* tbl = dyn + warp * TABLE;
  int cur = -1;  // the warp's current case
  long long f_loc = 0, z_loc = 0, s_loc = 0;
  auto flush = [&]() {
    if (lane == 0 && cur >= 0) {
      CaseAcc& A = b.acc[cur];
      if (f_loc) atomicAdd(&A.f, (unsigned long long)f_loc);
      if (z_loc) atomicAdd(&A.z, (unsigned long long)z_loc);
      if (s_loc) atomicAdd(&A.s, (unsigned long long)s_loc);
    }
    f_loc = z_loc = s_loc = 0;
  };
  for (;;) {
    if (t == 0) {
      const long long ch = (long long)atomicAdd(&b.hdr->sample_ctr, 1ull);
      s_chunk = ch;
      if (ch < b.total_chunks) s_case = __ldg(b.chunk_case + ch);
    }
    __syncthreads();
    const long long chunk = s_chunk;
    if (chunk >= b.total_chunks) break;
    long long base = chunk * b.sample_chunk;
    const long long c_end = min(b.total_cand, base + b.sample_chunk);
    // this thread's case, and its candidate range [lo_x, hi_x)
    int cx = s_case;
    long long lo_x = b.cases[cx].cand_off, hi_x = lo_x + b.cases[cx].n_cand;
    while (base < c_end) {
      if (t == 0) list_n = 0;
      __syncthreads();
      int n = 0;  // rows staged: the same in every thread (the barrier's count)
      for (;;) {
        const long long x = base + t;
        bool take = false;
        int row = 0;
        // (every candidate below total_cand lies in some case, so the walk
        // stops inside the array; the bound only guards a corrupted plan)
        while (x < c_end && x >= hi_x && cx + 1 < b.n_cases) {
          ++cx;
          lo_x = b.cases[cx].cand_off;
          hi_x = lo_x + b.cases[cx].n_cand;
        }
        if (x < c_end && x >= lo_x && x < hi_x) {
          const BatchCase& k = b.cases[cx];
          const unsigned long long loc = (unsigned long long)(x - lo_x);
          const uint32_t h = sample_hash32(k.seed, loc);
          if (k.src == kSrcBernoulli) {
            take = (uint64_t)h < k.threshold;
            row = (int)loc;
          } else {
            take = true;
            row = (int)(((uint64_t)h * (uint64_t)k.M) >> 32);
          }
        }
        const unsigned bal = __ballot_sync(kFull, take);
        int wbase = 0;
        if (lane == 0 && bal) wbase = atomicAdd(&list_n, __popc(bal));
        wbase = __shfl_sync(kFull, wbase, 0);
        if (take) {
          const int e = wbase + __popc(bal & ((1u << lane) - 1u));
          list_row[e] = row;
          list_case[e] = cx;
        }
        base += NT;
        n += __syncthreads_count(take);
        if (base >= c_end || n > kListCap - NT) break;
      }
      for (int e = warp; warp < AW && e < n; e += AW) {
        const int c = list_case[e], r = list_row[e];
        if (c != cur) {
          flush();
          cur = c;
          if (lane == 0) batch_dedup_args(b, c, wa[warp]);
          __syncwarp();
        }
        long long flop;
        const long long nnz = dedup_row_warp(wa[warp], r, tbl, &flop);
        if (lane == 0) {
          f_loc += flop;
          s_loc += 1;
          if (nnz >= 0) z_loc += nnz;
        }
      }
      __syncthreads();
    }
  }
  flush();
}

template <int TABLE>
__global__ void __launch_bounds__(kDedupThreads) kb_sample(BatchArgs b) {
  extern __shared__ int dyn[];
  __shared__ SampleShared<kDedupThreads> sh;
  batch_sample_phase<TABLE, kDedupThreads>(b, dyn, sh);
}

// ---------------------------------------------------------------------------
// Heavy rows of all cases, one block per row (see heavy_row_nnz): first the
// rows of more than kBatchBigProducts products (queued from the top of the
// array), then the others, each claimed one at a time.  A block claims its
// next row when it starts one (the claim's round trip is hidden behind the
// row), and finds a row's case among the cases' first rows, held in shared
// memory for batches of at most kCaseCache cases.
// ---------------------------------------------------------------------------
constexpr int kCaseCache = 1024;
struct HeavyShared {
  HeavySmem sm;
  DedupArgs ha;
  long long s_h;
  int s_case;
  int row_base[kCaseCache];  // cases' first batch-wide rows (total rows < 2^31)
};

// The heavy-row pass by a block of kHeavyThreads threads; tab holds
// bitmap_words words of shared memory.
__device__ __forceinline__ void batch_heavy_phase(const BatchArgs& b, unsigned* tab, int bitmap_words,
                                                  HeavyShared& hs) {
  HeavySmem& sm = hs.sm;
  DedupArgs& ha = hs.ha;
  long long& s_h = hs.s_h;
  int& s_case = hs.s_case;
  const int t = threadIdx.x;
  const unsigned n_big = (unsigned)min((long long)b.hdr->big_count, b.heavy_cap);
  const unsigned n_heavy = (unsigned)min((long long)b.hdr->heavy_count, b.heavy_cap - n_big);
  const bool cached = b.n_cases <= kCaseCache;
  if (cached)
    for (int i = t; i < b.n_cases; i += kHeavyThreads) hs.row_base[i] = (int)b.cases[i].row_base;
  unsigned q_next = 0;  // thread 0: the claim in flight
  if (t == 0) q_next = atomicAdd(&b.hdr->heavy_ctr, 1u);
  for (;;) {
    if (t == 0) {
      const unsigned q = q_next;
      long long h = -1;
      if (q < n_big) {
        h = b.heavy_cap - 1 - q;
      } else if (q - n_big < n_heavy) {
        h = q - n_big;
      }
      s_h = h;
      if (h >= 0) q_next = atomicAdd(&b.hdr->heavy_ctr, 1u);  // the next row, claimed during this one
    }
    __syncthreads();  // (also orders the case cache)
    const long long h = s_h;
    if (h < 0) break;
    const int g = b.heavy[h] - 1;
    if (t < 32) {
      const int c = cached ? warp_last_le(b.n_cases, (long long)g, [&](int i) { return (long long)hs.row_base[i]; })
                           : warp_last_le(b.n_cases, (long long)g, [&](int i) { return b.cases[i].row_base; });
      if (t == 0) {
        s_case = c;
        batch_dedup_args(b, c, ha);
      }
    }
    __syncthreads();
    if (t == 0) b.heavy[h] = 0;  // taken: every thread has read the entry
    const int c = s_case;
    bool bad = false;
    const long long nnz = heavy_row_nnz(ha, g - ha.heavy_base, sm, tab, bitmap_words, bad);
    if (t == 0) atomicAdd(&b.acc[c].z, (unsigned long long)nnz);
    if (__syncthreads_or(bad) && t == 0) atomicOr(&b.acc[c].status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
  }
}

__global__ void __launch_bounds__(kHeavyThreads) kb_heavy(BatchArgs b, int bitmap_words) {
  extern __shared__ unsigned tab[];
  __shared__ HeavyShared hs;
  batch_heavy_phase(b, tab, bitmap_words, hs);
}

// ---------------------------------------------------------------------------
// Exclusive prefix of `tile` over the tiles [first, tile) of its case, by one
// warp: each lane watches one predecessor, 32 at a time going backwards, until
// one of them has published its inclusive prefix (ftot_flag; the case's first
// tile publishes it at once) - the aggregates (total_flag) of the tiles after
// it are added on.  Waits give up after about a second each and set TIMEOUT.
// ---------------------------------------------------------------------------
__device__ long long lookback_excl(Slot* slots, int first, int tile, unsigned ep, unsigned* status) {
  const int lane = threadIdx.x & 31;
  long long excl = 0;
  for (int hi = tile - 1; hi >= first; hi -= 32) {
    const int q = hi - lane;
    int st = 0;
    long long v = 0;
    if (q >= first) {
      const uint64_t t0 = global_ns();
      unsigned ns = 32;
      for (int it = 0; it < (1 << 26); ++it) {
        if (flag_load(&slots[q].ftot_flag) == ep) {
          st = 2;
          v = *reinterpret_cast<volatile long long*>(&slots[q].ftot);
          break;
        }
        if (flag_load(&slots[q].total_flag) == ep) {
          st = 1;
          v = *reinterpret_cast<volatile long long*>(&slots[q].total);
          break;
        }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
        if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) {
          atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
          st = 2;  // stop here
          break;
        }
      }
    }
    const unsigned incl = __ballot_sync(kFull, st == 2);
    const int stop = incl ? __ffs(incl) - 1 : 31;
    excl += warp_sum((lane <= stop && q >= first) ? v : 0ll);
    if (incl) break;
  }
  return excl;
}

// ---------------------------------------------------------------------------
// FLOP per row, prediction and offsets of all cases, tile by tile.
// ---------------------------------------------------------------------------
template <int NW>
struct FlopPhaseShared {
  FlopSharedT<NW> sm;
  FlopArgs fa;
  int s_tile, s_case, s_tile0, s_ntiles;
};

// The FLOP / prediction / offsets pass by a block of NT threads.
template <int NT>
__device__ __forceinline__ void batch_flop_phase(const BatchArgs& b, FlopPhaseShared<NT / 32>& fp) {
  constexpr int NW = NT / 32;
  FlopSharedT<NW>& sm = fp.sm;
  FlopArgs& fa = fp.fa;
  int& s_tile = fp.s_tile;
  int& s_case = fp.s_case;
  int& s_tile0 = fp.s_tile0;
  int& s_ntiles = fp.s_ntiles;
  const int t = threadIdx.x;
  BatchHeader* hdr = b.hdr;
  const unsigned ep = *reinterpret_cast<volatile unsigned*>(&hdr->epoch) + 1u;
  Slot* slots = b.slots;
  for (;;) {
    if (t == 0) {
      const int tile = (int)atomicAdd(&hdr->tile_ctr, 1u);
      s_tile = tile;
      if (tile < b.total_tiles) {
        const int c = __ldg(b.tile_case + tile);
        const BatchCase& k = b.cases[c];
        s_case = c;
        s_tile0 = k.tile0;
        s_ntiles = k.ntiles;
        fa.M = k.M;
        fa.K = k.K;
        fa.nnzA = k.nnzA;
        fa.nnzB = k.nnzB;
        fa.a_rpt = k.a_rpt;
        fa.a_col = k.a_col;
        fa.b_rpt = k.b_rpt;
        fa.deg8 = k.deg8;
        fa.flop = k.flop;
        fa.pred = k.pred;
        fa.offsets = k.offsets;
        fa.vec_ok = k.vec_ok;
        fa.res = k.res;
      }
    }
    __syncthreads();
    const int tile = s_tile;
    if (tile >= b.total_tiles) break;
    const int c = s_case, tile0 = s_tile0, nt = s_ntiles, lt = tile - tile0;
    CaseAcc& acc = b.acc[c];
    unsigned* status = &acc.status;
    const long long M = fa.M;
    const long long D = M + fa.nnzA;
    const long long d0 = D * lt / nt, d1 = D * (lt + 1) / nt;
    const unsigned long long fz = acc.f, zz = acc.z;
    const double ratio = fz ? (double)zz / (double)fz : 0.0;

    bool bad = false;
    long long ftot = 0, ptot = 0;
    flop_range<kModePredict, NW>(fa, d0, d1, lt > 0, fz, zz, ratio, sm, &sm.out, ftot, ptot, bad);
    if (__syncthreads_or(bad) && t == 0) atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
    const int i0 = sm.out.i0, i1 = sm.out.i1;

    // ---- carries between the tiles of the case (waits only on tile - 1)
    if (t == 0) {
      const long long run = sm.out.run, head_known = sm.out.head_known;
      long long extra_f = sm.out.extra_f, extra_p = sm.out.extra_p;
      if (sm.out.dep) {
        long long cin = 0;
        if (flag_wait(&slots[tile - 1].carry_flag, ep, status)) cin = slots[tile - 1].carry;
        slots[tile].carry = cin + run;
        flag_store(&slots[tile].carry_flag, ep);
      } else {
        slots[tile].carry = i1 < M ? run : 0;
        flag_store(&slots[tile].carry_flag, ep);
        if (sm.out.head_pending) {
          long long cin = 0;
          if (flag_wait(&slots[tile - 1].carry_flag, ep, status)) cin = slots[tile - 1].carry;
          const long long v = cin + head_known;
          const int p = fz == 0 ? (int)v : pred_proposed((uint32_t)v, zz, fz, ratio);
          fa.pred[i0] = p;
          if (fa.flop) fa.flop[i0] = (int)v;
          extra_f += v;
          extra_p += p;
        }
      }
      sm.bc[4] = extra_f;
      sm.bc[5] = extra_p;
    }
    __syncthreads();
    const long long blk_f = block_sum<NT>(ftot, sm.red) + sm.bc[4];
    const long long blk_p = block_sum<NT>(ptot, sm.red) + sm.bc[5];

    // ---- exclusive prefix of the tile within its case
    if (t < 32) {
      if (t == 0) {
        if (lt == 0) {
          slots[tile].ftot = blk_p;
          flag_store(&slots[tile].ftot_flag, ep);
        } else {
          slots[tile].total = blk_p;
          flag_store(&slots[tile].total_flag, ep);
        }
      }
      const long long excl = lt > 0 ? lookback_excl(slots, tile0, tile, ep, status) : 0;
      if (t == 0) {
        if (lt > 0) {
          slots[tile].ftot = excl + blk_p;
          flag_store(&slots[tile].ftot_flag, ep);
        }
        sm.bc[6] = excl;
      }
    }
    __syncthreads();
    long long run = sm.bc[6];

    // ---- offsets of the rows [i0, i1)
    for (int rb = i0; rb < i1; rb += NT * kRowsPerThread) {
      const int r0 = rb + t * kRowsPerThread;
      int pv[kRowsPerThread];
      long long loc = 0;
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        pv[u] = (r0 + u < i1) ? fa.pred[r0 + u] : 0;
        loc += pv[u];
      }
      long long tot;
      long long ex = block_excl_scan<NT>(loc, sm.red, &tot) + run;
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u) {
        if (r0 + u < i1) {
          fa.offsets[r0 + u] = ex;
          ex += pv[u];
        }
      }
      run += tot;
    }

    // ---- the case's last tile writes offsets[M]; its last finisher the result
    if (t == 0) {
      if (lt == nt - 1) fa.offsets[M] = run;
      atomicAdd(&acc.F, (unsigned long long)blk_f);
      __threadfence();
      const unsigned prev = atomicAdd(&acc.tiles_done, 1u);
      if (prev == (unsigned)nt - 1) {
        __threadfence();
        volatile CaseAcc* va = &acc;
        unsigned st = va->status;
        if (va->f == 0) st |= SPGEMM_STATUS_WARN_EMPTY_SAMPLE;
        st |= *reinterpret_cast<volatile unsigned*>(&hdr->status);  // a grid barrier that gave up
        spgemm_result_t* res = fa.res;
        res->flop_total = (long long)va->F;
        res->flop_s = (long long)va->f;
        res->nnz_s = (long long)va->z;
        res->n_sampled = (long long)va->s;
        res->pred_total = *reinterpret_cast<volatile long long*>(&slots[tile0 + nt - 1].ftot);
        res->status = (int)st;
        va->f = 0;
        va->z = 0;
        va->s = 0;
        va->F = 0;
        va->status = 0;
        va->tiles_done = 0;
      }
      __threadfence();
      if (atomicAdd(&hdr->tiles_done, 1u) == (unsigned)b.total_tiles - 1) {
        __threadfence();
        *reinterpret_cast<volatile unsigned*>(&hdr->epoch) = ep;
      }
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kFlopThreads, SPG_FLOP_MIN_BLOCKS) kb_flop(BatchArgs b) {
  __shared__ FlopPhaseShared<kFlopWarps> fp;
  batch_flop_phase<kFlopThreads>(b, fp);
}

// ---------------------------------------------------------------------------
// The whole batch as ONE persistent launch: one block of kAllThreads threads
// per SM (cooperative: every block resident), running the four phases in turn
// with a grid barrier where a phase needs the previous one complete in every
// block: the tables and the samples before the heavy rows (the queue is
// final), the heavy rows before the FLOP pass (every case's f* and z* are
// final).  Each phase claims its work units as the separate kernels do.  The
// dynamic shared memory (kAllDynSmem) holds the warp tables of the sampled-row
// pass (32 warps x TABLE slots), then the heavy rows' bitmap, then the FLOP
// pass's buffers; it is held to 128 KB so the FLOP pass keeps a large L1.
// ---------------------------------------------------------------------------
constexpr int kAllThreads = 1024;
constexpr size_t kAllDynSmem = 128 * 1024;
static_assert(kAllThreads == kHeavyThreads, "the heavy rows are counted by the whole block");
static_assert(sizeof(FlopPhaseShared<kAllThreads / 32>) <= kAllDynSmem, "the FLOP pass's buffers fit");

union AllShared {
  SampleShared<kAllThreads> sample;
  HeavyShared heavy;
};

// Every block arrives at barrier *ctr, then waits (bounded; a wait that gives
// up sets the run's status) until all G have.
__device__ __forceinline__ void batch_grid_barrier(unsigned* ctr, unsigned G, unsigned* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(ctr, 1u);
    count_wait(ctr, G, status);
    __threadfence();
  }
  __syncthreads();
}

template <int TABLE>
__global__ void __launch_bounds__(kAllThreads, 1) kb_all(BatchArgs b, int bitmap_words) {
  // warps that count sampled rows: as many as the warp tables fit
  constexpr int kAW = (int)(kAllDynSmem / ((size_t)TABLE * sizeof(int))) < kAllThreads / 32
                          ? (int)(kAllDynSmem / ((size_t)TABLE * sizeof(int)))
                          : kAllThreads / 32;
  static_assert(kAW >= 1, "warp tables fit");
  extern __shared__ __align__(16) int all_dyn[];
  __shared__ AllShared ash;
  const unsigned G = gridDim.x;
  BatchHeader* hdr = b.hdr;
  // 1. the B row-length tables (used by the FLOP pass only)
  for (long long tb = blockIdx.x; tb < b.total_tab_blocks; tb += G) batch_table_unit(b, tb, threadIdx.x, kAllThreads);
  // 2. the samples and their rows' nnz; heavy rows queued
  if (b.total_chunks > 0) batch_sample_phase<TABLE, kAllThreads, kAW>(b, all_dyn, ash.sample);
  batch_grid_barrier(&hdr->bar[0], G, &hdr->status);
  // 3. the heavy rows
  batch_heavy_phase(b, reinterpret_cast<unsigned*>(all_dyn), bitmap_words, ash.heavy);
  batch_grid_barrier(&hdr->bar[1], G, &hdr->status);
  // 4. FLOP per row, prediction and offsets
  batch_flop_phase<kAllThreads>(b, *reinterpret_cast<FlopPhaseShared<kAllThreads / 32>*>(all_dyn));
}

}  // namespace spg
