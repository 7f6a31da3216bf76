// The structure prediction of one product C = A * B as ONE persistent launch:
// the proposed method (Eq. 4, Algorithm 2) or the reference design of the
// prior sampling method (Eq. 2), from the sample to the allocation offsets.
//
// One 1024-thread block per SM; blocks meet only through counters and flags in
// the workspace (all blocks are co-resident: the launch is cooperative and the
// grid never exceeds what the device holds at once; every wait gives up after
// about a second and reports SPGEMM_STATUS_ERR_TIMEOUT instead of hanging).
// Each block runs two warp groups side by side, each on its own hardware
// barrier, then the whole block finishes:
//   sampling group (the first kSampWarps warps): the block's slice of the sample candidates
//     (Sec. IV-A); FLOP and exact nnz of the sampled rows (Sec. IV-B; the hash
//     loop of Algorithm 2).  The rows are counted together, stage by stage, so
//     a batch of rows waits for each memory round trip once: their A offsets,
//     the B ranges of all their entries, then all their products,
//     deduplicated as (row, column) keys in one shared-memory table.  Rows too
//     long for a batch are queued as heavy;
//   streaming group (the other warps): its share of the B row-length byte table
//     (see degree_words), then, once every block's share exists, the FLOP of
//     every row of the block's merge-path range (Algorithm 1);
//   whole block: the heavy sampled rows, taken from the queue one at a time,
//     each counted by the whole block (hash table or column bitmap in shared
//     memory); then, once f*, z* (and, for the reference design, F) are final,
//     the per-row prediction of the block's rows, the sum of the totals of the
//     blocks before it, and the exclusive scan into the offsets.
// The sampling work is latency-bound and the FLOP pass is bound by the rate
// of scattered table lookups, so the two groups overlap well; the per-row
// FLOP stays in shared memory until the prediction.  The dynamic shared memory
// is held to 128 KB so that the FLOP pass keeps a large L1.
#pragma once

#include <type_traits>

#include "common.cuh"
#include "k_dedup.cuh"
#include "k_flop.cuh"

namespace spg {

constexpr int kPredThreads = 1024;
constexpr int kPredWarps = kPredThreads / 32;
// merged items per block, at least: small problems get more blocks, so each
// block's chains of round trips are short (2D 5-point 64x64: 37 -> 29 us)
constexpr long long kPredItemsPerBlock = 1024;
static_assert(kPredThreads == kHeavyThreads, "heavy rows are counted by the whole block");

// ---- the two warp groups --------------------------------------------------------
#ifndef SPG_SAMP_WARPS
#define SPG_SAMP_WARPS 12  // measured best on GB300 among 8, 12, 16 (ER n = 2^20)
#endif
constexpr int kSampWarps = SPG_SAMP_WARPS;
constexpr int kSampThreads = kSampWarps * 32;
constexpr int kStreamWarps = kPredWarps - kSampWarps;
constexpr int kStreamThreads = kStreamWarps * 32;
constexpr int kBarSamp = 1;    // hardware barrier of the sampling group
constexpr int kBarStream = 2;  // hardware barrier of the streaming group
constexpr int kDegBatch = 3;    // table words per streaming thread loaded at once (2^20 rows: 2.7 each)
constexpr int kScanChunks = 2;  // blocks of at most this many 4096-row chunks scan before the cross-block wait

// ---- sampling group: batch limits ------------------------------------------------
constexpr int kSRows = kSampThreads;            // sampled rows per row round (one per thread)
constexpr int kSEntPer = 4;                     // A entries per thread per entry round
constexpr int kSEnts = kSampThreads * kSEntPer;  // A entries per entry round
constexpr int kSEntMax = 256;                   // rows with more entries are queued as heavy
constexpr int kSEntRound = kSEnts - kSEntMax;   // entry offsets at which entry rounds start
constexpr int kSLgSlots = 13;                   // (row, column) table of 2^13 slots
constexpr int kSSlots = 1 << kSLgSlots;
constexpr int kSProdMax = 1024;                 // rows with more products are queued as heavy
constexpr int kSProdRound = kSSlots / 2 - kSProdMax;  // product offsets at which rounds start
constexpr int kSUnroll = 8;                     // products per thread loaded at once
// product rounds of one entry round: at most kSRows rows of at most kSProdMax each
constexpr int kSMaxRounds = kSRows * kSProdMax / kSProdRound + 2;
constexpr int kSRowBits = kSRows <= 256 ? 8 : kSRows <= 512 ? 9 : 10;
constexpr int kSColBits = 32 - kSRowBits;       // key = row << kSColBits | column: needs N < 2^kSColBits
static_assert(kSRows <= (1 << kSRowBits), "row index fits the key");
static_assert(kSMaxRounds <= kSampThreads, "one round start per thread");

struct SampleSmem {
  unsigned long long r_flop[kSRows];  // FLOP of each staged row (entry round)
  int r_row[kSRows];                  // A row id of each staged row
  int r_rb[kSRows];                   // its first entry in A
  int r_eoff[kSRows];                 // exclusive prefix of the entries counted here
  int e_bs[kSEnts];                   // B row start of each entry of the round
  int e_bl[kSEnts];                   // B row length (0 once the row is queued as heavy)
  int e_poff[kSEnts];                 // exclusive prefix of e_bl
  int e_row[kSEnts];                  // staged row of each entry
  int p_start[kSMaxRounds + 1];       // first product of each product round
  int m_max;                          // last product round
  int tbl[kSSlots];                   // (row, column) keys, -1 = empty
};

// ---- dynamic shared memory ------------------------------------------------------
// [0, kOffFlopSm): the sampling group's batch (or its per-warp tables);
// [kOffFlopSm, kOffSflop): the streaming group's buffers; [kOffSflop, end): the
// FLOP of the block's first kSFlopN rows, kept until the prediction.  The
// heavy rows then use the whole space (after the FLOP is copied out).
constexpr size_t kPredDynSmem = 128 * 1024;
constexpr size_t round256(size_t b) { return (b + 255) / 256 * 256; }
constexpr size_t kOffFlopSm = round256(sizeof(SampleSmem) > (size_t)kSampWarps * kWarpTable * sizeof(int)
                                           ? sizeof(SampleSmem)
                                           : (size_t)kSampWarps * kWarpTable * sizeof(int));
constexpr size_t kOffSflop = kOffFlopSm + round256(sizeof(FlopSharedT<kStreamWarps>));
constexpr int kSFlopN = (int)((kPredDynSmem - kOffSflop) / sizeof(int));
static_assert(kOffSflop < kPredDynSmem, "groups' buffers fit");
static_assert((size_t)kBlockHashSlots * sizeof(int) <= kPredDynSmem, "heavy-row hash fits");

struct PredArgs {
  FlopArgs f;        // rows, operands, FLOP buffer, outputs, workspace, result
  DedupArgs d;       // the sample and the deduplication of its rows
  int bitmap_words;  // 32-bit words of dynamic shared memory (heavy rows' bitmap)
  int flop_out;      // f.flop is the caller's flop_row (else the workspace buffer)
};

constexpr int kListCapW = 1024;  // staged rows of the per-warp fallback

struct PredStatic {
  long long red[kPredWarps + 1];     // whole-block scans
  long long red_s[kSampWarps + 1];   // sampling-group scans
  long long bc[8];
  unsigned long long pre[4];         // f*, z*, |S| and the ratio's reciprocal, read early
  int pre_ready;                     // 1: pre[] is final and no sampled row is heavy
  int stream_fin;                    // the streaming group has finished its FLOP pass
  int s_enc, s_part;
  int s_last;
  int list[kListCapW];
  HeavySmem heavy;
};

// Candidate x of the sample: is it drawn, and which row (Sec. IV-A)?
__device__ __forceinline__ bool sample_candidate(const DedupArgs& d, long long x, int* row) {
  const uint32_t h = sample_hash32(d.seed, (uint64_t)x);
  if (d.src == kSrcBernoulli) {
    *row = (int)x;
    return (uint64_t)h < d.threshold;
  }
  *row = (int)(((uint64_t)h * (uint64_t)d.M) >> 32);
  return true;
}

// Queues a sampled row for the block-per-row pass.  The entry is row + 1 when
// its FLOP is already counted, -(row + 1) when the pass must count it too.
__device__ __forceinline__ void push_heavy(const DedupArgs& d, int row, bool flop_counted) {
  const unsigned h = atomicAdd(d.heavy_count, 1u);
  if (h < (unsigned long long)d.heavy_cap)
    flag_store(reinterpret_cast<unsigned*>(d.heavy + h), flop_counted ? (unsigned)(row + 1) : (unsigned)(-(row + 1)));
}

// Index of the last i in [lo, hi) with v[i] <= x (v non-decreasing, v[lo] <= x).
__device__ __forceinline__ int last_le(const int* v, int lo, int hi, long long x) {
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

// Sampling group, batched (B has fewer than 2^24 columns).  Adds this thread's
// share of f*, z* and |S| to f_loc, z_loc, s_loc.
__device__ void sample_batched(const DedupArgs& d, SampleSmem& sh, long long* red, long long& f_loc,
                               long long& z_loc, long long& s_loc, bool& bad) {
  constexpr int NT = kSampThreads;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, c = blockIdx.x;
  const long long c_beg = (long long)c * d.n_cand / G, c_end = (long long)(c + 1) * d.n_cand / G;
  // thread t hashes the candidates [x0, x1) of the block's slice
  const long long q = (c_end - c_beg + NT - 1) / NT;
  const long long x0 = min(c_end, c_beg + t * q), x1 = min(c_end, x0 + q);
  int cnt = 0;
  for (long long x = x0; x < x1; ++x) {
    int row;
    cnt += sample_candidate(d, x, &row);
  }
  long long total;
  const long long pre = block_excl_scan<NT, kBarSamp>(cnt, red, &total);
  if (t == 0) s_loc += total;

  for (long long R0 = 0; R0 < total; R0 += kSRows) {
    // ---- the round's rows: sample indices [R0, R0 + nr), in candidate order
    const int nr = (int)min((long long)kSRows, total - R0);
    if (pre + cnt > R0 && pre < R0 + nr) {
      long long idx = pre;
      for (long long x = x0; x < x1 && idx < R0 + nr; ++x) {
        int row;
        if (sample_candidate(d, x, &row)) {
          if (idx >= R0) sh.r_row[idx - R0] = row;
          ++idx;
        }
      }
    }
    group_sync<kBarSamp, NT>();
    // ---- stage 1: A offsets of every staged row (thread t: row t)
    int nent = 0;
    if (t < nr) {
      const int row = sh.r_row[t];
      long long rb = __ldg(d.a_rpt + row), re = __ldg(d.a_rpt + row + 1);
      if (!clamp_range(rb, re, d.nnzA)) bad = true;
      if (re - rb > kSEntMax) {
        push_heavy(d, row, false);
      } else {
        nent = (int)(re - rb);
      }
      sh.r_rb[t] = (int)rb;
    }
    long long E;
    const int eoff = (int)block_excl_scan<NT, kBarSamp>(nent, red, &E);
    if (t < nr) sh.r_eoff[t] = eoff;
    group_sync<kBarSamp, NT>();

    // ---- entry rounds: rows whose entries start in [E0, E0 + kSEntRound)
    for (long long E0 = 0; E0 < E; E0 += kSEntRound) {
      const int ia = group_count<kBarSamp, NT>(t < nr && eoff < E0);
      const int ib = group_count<kBarSamp, NT>(t < nr && eoff < E0 + kSEntRound);
      const int ea = ia < nr ? sh.r_eoff[ia] : (int)E;
      const int eb = ib < nr ? sh.r_eoff[ib] : (int)E;
      const int ne = eb - ea;  // <= kSEnts
      if (t >= ia && t < ib) sh.r_flop[t] = 0;
      group_sync<kBarSamp, NT>();
      // ---- stage 2: B range of every entry of the round (kSEntPer per thread,
      // every load of a stage in flight together)
      {
        int ii[kSEntPer], kk[kSEntPer];
#pragma unroll
        for (int u = 0; u < kSEntPer; ++u) {
          const int le = t + u * NT;
          ii[u] = 0;
          kk[u] = 0;
          if (le < ne) {
            const int g = ea + le;
            ii[u] = last_le(sh.r_eoff, ia, ib, g);
            kk[u] = __ldg(d.a_col + sh.r_rb[ii[u]] + (g - sh.r_eoff[ii[u]]));
          }
        }
        int b0[kSEntPer], b1[kSEntPer];
#pragma unroll
        for (int u = 0; u < kSEntPer; ++u) {
          b0[u] = 0;
          b1[u] = 0;
          if (t + u * NT < ne) {
            if ((unsigned)kk[u] < (unsigned long long)d.K) {
              b0[u] = __ldg(d.b_rpt + kk[u]);
              b1[u] = __ldg(d.b_rpt + kk[u] + 1);
            } else {
              bad = true;
            }
          }
        }
#pragma unroll
        for (int u = 0; u < kSEntPer; ++u) {
          const int le = t + u * NT;
          if (le < ne) {
            long long lo = b0[u], hi = b1[u];
            if (!clamp_range(lo, hi, d.nnzB)) bad = true;
            sh.e_bs[le] = (int)lo;
            sh.e_bl[le] = (int)(hi - lo);
            sh.e_row[le] = ii[u];
            atomicAdd(&sh.r_flop[ii[u]], (unsigned long long)(hi - lo));
          }
        }
      }
      group_sync<kBarSamp, NT>();
      // rows with too many products go to the heavy queue (their FLOP counted here)
      if (t >= ia && t < ib) {
        const unsigned long long fl = sh.r_flop[t];
        f_loc += (long long)fl;
        if (fl > (unsigned long long)kSProdMax) {
          push_heavy(d, sh.r_row[t], true);
          sh.r_flop[t] = ~0ull;
        }
      }
      group_sync<kBarSamp, NT>();
      // products of each entry: exclusive prefix over the round's entries
      int bl[kSEntPer];
      int bsum = 0;
#pragma unroll
      for (int u = 0; u < kSEntPer; ++u) {
        const int le = t * kSEntPer + u;
        bl[u] = (le < ne && sh.r_flop[sh.e_row[le]] != ~0ull) ? sh.e_bl[le] : 0;
        bsum += bl[u];
      }
      long long P;
      int po = (int)block_excl_scan<NT, kBarSamp>(bsum, red, &P);
#pragma unroll
      for (int u = 0; u < kSEntPer; ++u) {
        const int le = t * kSEntPer + u;
        if (le < ne) {
          sh.e_poff[le] = po;
          sh.e_bl[le] = bl[u];
        }
        po += bl[u];
      }
      if (t <= kSMaxRounds) sh.p_start[t] = 0x7fffffff;
      if (t == 0) sh.m_max = -1;
      group_sync<kBarSamp, NT>();
      // product rounds: round m holds the rows whose products start in
      // [m * kSProdRound, (m + 1) * kSProdRound), so at most kSProdRound +
      // kSProdMax products, half the table's slots.  Consecutive rows start at
      // most kSProdMax < kSProdRound products apart, so rounds 0..m_max all hold
      // a row; round m's products are [p_start[m], p_start[m + 1]) (P for the last).
      if (t >= ia && t < ib) {
        const unsigned long long fl = sh.r_flop[t];
        if (fl != ~0ull && fl > 0) {
          const int st = sh.e_poff[sh.r_eoff[t] - ea];
          const int m = st / kSProdRound;
          atomicMin(&sh.p_start[m], st);
          atomicMax(&sh.m_max, m);
        }
      }
      group_sync<kBarSamp, NT>();
      const int nrounds = sh.m_max + 1;
      for (int m = 0; m < nrounds; ++m) {
        const int pa = sh.p_start[m], pb = m + 1 < nrounds ? sh.p_start[m + 1] : (int)P;
        for (int i = t; i < kSSlots; i += NT) sh.tbl[i] = -1;
        group_sync<kBarSamp, NT>();
        // warp w takes a contiguous run of U * 32 products, lanes interleaved;
        // a lane loads kSUnroll column ids before inserting them
        const int U = (pb - pa + NT - 1) / NT;
        const int w0 = pa + warp * U * 32, w1 = min(pb, w0 + U * 32);
        int e = w0 + lane < w1 ? last_le(sh.e_poff, 0, ne, w0 + lane) : 0;
        for (int kb = 0; kb < U; kb += kSUnroll) {
          unsigned key_hi[kSUnroll];
          int col[kSUnroll];
#pragma unroll
          for (int k = 0; k < kSUnroll; ++k) {
            const int pk = w0 + lane + 32 * (kb + k);
            key_hi[k] = 0xffffffffu;
            col[k] = 0;
            if (kb + k < U && pk < w1) {
              while (e + 1 < ne && sh.e_poff[e + 1] <= pk) ++e;
              key_hi[k] = (unsigned)sh.e_row[e] << kSColBits;
              col[k] = __ldg(d.b_col + sh.e_bs[e] + (pk - sh.e_poff[e]));
            }
          }
#pragma unroll
          for (int k = 0; k < kSUnroll; ++k) {
            if (key_hi[k] != 0xffffffffu) {
              if ((unsigned)col[k] < (unsigned long long)d.N) {
                z_loc += table_insert(sh.tbl, kSLgSlots, (int)(key_hi[k] | (unsigned)col[k]));
              } else {
                bad = true;
              }
            }
          }
        }
        group_sync<kBarSamp, NT>();
      }
    }
    group_sync<kBarSamp, NT>();
  }
}

// Sampling group for B with 2^24 columns or more: each warp counts its rows
// alone (dedup_row_warp), with a table of kWarpTable slots per warp.
__device__ void sample_per_warp(const DedupArgs& d, int* tables, int* list, long long* red, long long& f_loc,
                                long long& z_loc, long long& s_loc) {
  constexpr int NT = kSampThreads;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int G = gridDim.x, c = blockIdx.x;
  int* tbl = tables + warp * kWarpTable;
  const long long c_beg = (long long)c * d.n_cand / G, c_end = (long long)(c + 1) * d.n_cand / G;
  long long base = c_beg;
  while (base < c_end) {
    // stage selected rows until the list could overflow or the slice ends; n
    // (the same in every thread) is the number staged so far
    int n = 0;
    for (;;) {
      const long long cand = base + t;
      int row = 0;
      const bool take = cand < c_end && sample_candidate(d, cand, &row);
      const unsigned bal = __ballot_sync(kFull, take);
      if (lane == 0) red[warp] = __popc(bal);
      group_sync<kBarSamp, NT>();
      int wbase = n;
      for (int w = 0; w < warp; ++w) wbase += (int)red[w];
      if (take) list[wbase + __popc(bal & ((1u << lane) - 1u))] = row;
      base += NT;
      n += group_count<kBarSamp, NT>(take);
      if (base >= c_end || n > kListCapW - NT) break;
    }
    for (int e = warp; e < n; e += kSampWarps) {
      long long flop;
      const long long nnz = dedup_row_warp(d, list[e], tbl, &flop);
      if (lane == 0) {
        f_loc += flop;
        s_loc += 1;
        if (nnz >= 0) z_loc += nnz;
      }
    }
    group_sync<kBarSamp, NT>();
  }
}

// Thread 0: claims the next heavy-queue entry and returns it (see push_heavy),
// or 0 once every queued row is taken (the queue is final when every block's
// sampling group has finished).  Waits for an entry whose writer has not
// stored it yet.  ctr_hint and cnt_hint are earlier unordered reads of
// heavy_ctr and heavy_count: both only grow during a launch, so an index below
// cnt_hint names an entry that exists, and "nothing left" is concluded only
// from the ordered reads below.
__device__ int claim_heavy_row(WsHeader* hdr, int* heavy, unsigned long long cap, unsigned G, unsigned ctr_hint,
                               unsigned cnt_hint) {
  if ((unsigned long long)ctr_hint >= min((unsigned long long)cnt_hint, cap)) {
    // maybe nothing to take: every sampling group done and every queued entry
    // claimed (one round trip instead of a claim and its checks)
    if (flag_load(&hdr->sample_done) >= G) {
      volatile WsHeader* vh = hdr;
      if ((unsigned long long)vh->heavy_ctr >= min((unsigned long long)vh->heavy_count, cap)) return 0;
    }
  }
  const unsigned h = atomicAdd(&hdr->heavy_ctr, 1u);
  const uint64_t t0 = global_ns();
  unsigned ns = 32;
  for (int it = 0; it < (1 << 26); ++it) {
    // only entries below the count queued so far exist (a clean workspace may
    // hold anything past them); an existing entry reads 0 until its writer's
    // store lands
    if (h < cap && (h < cnt_hint || h < flag_load(&hdr->heavy_count))) {
      const unsigned v = flag_load(reinterpret_cast<const unsigned*>(heavy + h));
      if (v != 0) {
        heavy[h] = 0;  // taken
        return (int)v;
      }
    }
    if (flag_load(&hdr->sample_done) >= G) {
      const unsigned long long n = min((unsigned long long)flag_load(&hdr->heavy_count), cap);
      if (h >= n) return 0;  // the entry exists otherwise; its store is on its way
    }
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) break;
  }
  atomicOr(&hdr->status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
  return 0;
}

// ---- split rows ------------------------------------------------------------------
constexpr long long kHugeProducts = 1ll << 20;  // sampled rows with more products are split
constexpr long long kPartProducts = 1ll << 17;  // products per part, at least
constexpr unsigned kPartParked = 0xffff0000u;   // part_ctr while a slot is being set up

// Warp 0: the block's next heavy work.  *part = slot * 128 + part for a part
// of a split row (-1 if none is open), else *enc = a queued row's entry (0 once
// every queued row is taken).  One round of loads, all in flight together,
// reads the split slots (one lane each) and the queue counters; a claimed
// part counts only if its slot still holds the row it was read for.
__device__ void claim_heavy_work(WsHeader* hdr, HugeSlot* hs, int* heavy, unsigned long long cap, unsigned G,
                                 int* part_out, int* enc_out) {
  const int lane = threadIdx.x & 31;
  bool open = false;
  unsigned hint = 0;
  if (hs && lane < kHugeSlots) {
    volatile HugeSlot* v = hs + lane;
    const unsigned st = v->state, pc = v->part_ctr, np = v->parts;
    open = st == 2u && pc < np;
  } else if (lane == kHugeSlots) {
    hint = reinterpret_cast<volatile WsHeader*>(hdr)->heavy_ctr;
  } else if (lane == kHugeSlots + 1) {
    hint = reinterpret_cast<volatile WsHeader*>(hdr)->heavy_count;
  }
  const unsigned ctr_hint = __shfl_sync(kFull, hint, kHugeSlots);
  const unsigned cnt_hint = __shfl_sync(kFull, hint, kHugeSlots + 1);
  unsigned m = __ballot_sync(kFull, open);
  int part = -1;
  while (m != 0 && part < 0) {
    const int s = __ffs(m) - 1;
    m &= m - 1;
    if (lane == 0) {
      const unsigned q = atomicAdd(&hs[s].part_ctr, 1u);
      __threadfence();
      // the slot may have been finished and set up again in between: the claim
      // counts only against the row now published there
      volatile HugeSlot* v = hs + s;
      if (flag_load(&hs[s].state) == 2u && q < v->parts) part = s * 128 + (int)q;
    }
    part = __shfl_sync(kFull, part, 0);
  }
  if (lane == 0) {
    *part_out = part;
    *enc_out = part >= 0 ? 0 : claim_heavy_row(hdr, heavy, cap, G, ctr_hint, cnt_hint);
  }
  __syncwarp();
}

// The whole block: sets up slot h for a row with entries [rb, re) and FLOP
// flop > kHugeProducts: up to kMaxParts parts of about equal products (at
// least kPartProducts each), cut at entry starts.
__device__ void split_row(const DedupArgs& d, HugeSlot* h, long long rb, long long re, long long flop,
                          long long* red, bool& bad) {
  const int t = threadIdx.x;
  const long long ps = max(kPartProducts, (flop + kMaxParts - 1) / kMaxParts);
  const int P = (int)min((long long)kMaxParts, (flop + ps - 1) / ps);
  long long pre = 0;
  for (long long g = rb; g < re; g += kPredThreads) {
    long long st = 0, len = 0;
    if (g + t < re) b_row(d, __ldg(d.a_col + g + t), st, len, bad);
    long long tot;
    const long long ex = block_excl_scan<kPredThreads>(len, red, &tot) + pre;
    // part k >= 1 starts at the entry whose products hold product k * ps
    if (len > 0) {
      for (long long k = max(1ll, (ex + ps - 1) / ps); k < P && k * ps < ex + len; ++k) h->bnd[k] = g + t;
    }
    pre += tot;
  }
  __threadfence();  // each writer's boundaries are visible before the slot is published
  __syncthreads();
  if (t == 0) {
    h->bnd[0] = rb;
    h->bnd[P] = re;
    h->parts = (unsigned)P;
    h->parts_done = 0;
    __threadfence();
    h->part_ctr = 0;
    __threadfence();
    flag_store(&h->state, 2u);
  }
}

// The heavy sampled rows, by the whole block: parts of split rows first, then
// rows from the queue (rows with more than kHugeProducts products are split
// into parts for all blocks), until every queued row is counted.  Returns
// whether the FLOP of the block's rows is still in sflop (the tables used
// here overwrite it, so it is moved to f.flop before the first one).  Kept
// out of line so that its registers do not weigh on the FLOP pass.
__device__ __noinline__ bool heavy_phase(const PredArgs& p, PredStatic& ss, unsigned char* pdyn, int* sflop,
                                         int i0, int i1) {
  const FlopArgs& a = p.f;
  const DedupArgs& d = p.d;
  const int t = threadIdx.x;
  const int G = gridDim.x;
  WsHeader* hdr = a.ws.hdr;
  bool flop_in_smem = true;
  unsigned* tab = reinterpret_cast<unsigned*>(pdyn);
  HugeSlot* hs = a.ws.huge;
  // the wait for other blocks' heavy rows gives up after about a second
  // without progress (a large input may legitimately keep the blocks busy
  // for longer than that in total)
  uint64_t t_start = global_ns();
  unsigned seen_done = 0;
  for (;;) {
    if (t < 32) claim_heavy_work(hdr, hs, d.heavy, (unsigned long long)d.heavy_cap, (unsigned)G, &ss.s_part, &ss.s_enc);
    __syncthreads();
    const int part = ss.s_part, enc = ss.s_enc;
    if ((part >= 0 || enc != 0) && flop_in_smem) {  // the tables below overwrite sflop: move it out first
      if (!p.flop_out)
        for (int r = i0 + t; r < min(i1, (i0 & ~3) + kSFlopN); r += kPredThreads) a.flop[r] = sflop[r - (i0 & ~3)];
      flop_in_smem = false;
      __syncthreads();
    }
    bool bad = false;
    if (part >= 0) {
      // ---- one part of a split row: its bitmap over B's columns, written whole
      HugeSlot* h = hs + (part >> 7);
      const int q = part & 127;
      unsigned* gb = a.ws.hbits + ((long long)(part >> 7) * kMaxParts + q) * a.ws.huge_words;
      const long long rb = *reinterpret_cast<volatile long long*>(&h->bnd[q]);
      const long long re = *reinterpret_cast<volatile long long*>(&h->bnd[q + 1]);
      const long long range = (long long)p.bitmap_words * 32;
      for (long long lo = 0; lo < d.N; lo += range) {
        const long long hi = min((long long)d.N, lo + range);
        const int words = (int)((hi - lo + 31) / 32);
        for (int i = t; i < words; i += kPredThreads) tab[i] = 0u;
        __syncthreads();
        heavy_count_pass<true, false>(d, rb, re, ss.heavy, tab, words, lo, hi, bad);
        for (int i = t; i < words; i += kPredThreads) gb[(lo >> 5) + i] = tab[i];
        __threadfence();  // every thread's words are visible before the part counts as done
        __syncthreads();
      }
      if (t == 0) {
        __threadfence();
        const unsigned prev = atomicAdd(&h->parts_done, 1u);
        ss.s_last = prev + 1 == *reinterpret_cast<volatile unsigned*>(&h->parts);
      }
      __syncthreads();
      if (ss.s_last) {  // the row's last part: OR the parts' bitmaps, count, free the slot
        __threadfence();
        const unsigned nparts = *reinterpret_cast<volatile unsigned*>(&h->parts);
        const unsigned* b0 = a.ws.hbits + (long long)(part >> 7) * kMaxParts * a.ws.huge_words;
        long long cnt = 0;
        const long long nw = (d.N + 31) / 32;
        for (long long i = t; i < nw; i += kPredThreads) {
          unsigned w = 0;
          for (unsigned pp = 0; pp < nparts; ++pp) w |= __ldcg(b0 + pp * a.ws.huge_words + i);
          cnt += __popc(w);
        }
        cnt = block_sum<kPredThreads>(cnt, ss.red);  // every read done before the slot is freed
        if (t == 0) {
          atomicAdd(&hdr->z_acc, (unsigned long long)cnt);
          __threadfence();
          // part_ctr stays at or above `parts`, so a late claim of this row
          // fails; the next owner parks and resets it
          flag_store(&h->state, 0u);
          atomicAdd(&hdr->heavy_done, 1u);
        }
      }
    } else if (enc != 0) {
      // ---- a queued row: counted here, or split for all blocks
      long long rb, re;
      const int row = enc > 0 ? enc - 1 : -enc - 1;
      bool pre;
      const long long flop = heavy_row_flop(d, row, ss.heavy, &rb, &re, bad, &pre);
      if (t == 0) {
        if (enc < 0) atomicAdd(&hdr->f_acc, (unsigned long long)flop);
        ss.s_part = -1;
        if (hs && flop > kHugeProducts) {
          for (int sl = 0; sl < kHugeSlots; ++sl) {
            if (atomicCAS(&hs[sl].state, 0u, 1u) == 0u) {
              hs[sl].part_ctr = kPartParked;
              __threadfence();
              ss.s_part = sl;
              break;
            }
          }
        }
      }
      __syncthreads();
      if (ss.s_part >= 0) {
        split_row(d, hs + ss.s_part, rb, re, flop, ss.red, bad);
      } else {  // small enough, or every split slot is taken: counted here
        const long long nnz = heavy_row_count(d, rb, re, flop, ss.heavy, tab, p.bitmap_words, bad, pre);
        if (t == 0) {
          atomicAdd(&hdr->z_acc, (unsigned long long)nnz);
          __threadfence();
          atomicAdd(&hdr->heavy_done, 1u);
        }
      }
    } else {
      // ---- nothing to take: leave once every queued row is counted (the
      // parts of split rows still open are taken by the blocks at them)
      if (t == 0) {
        const unsigned nh = (unsigned)min((unsigned long long)flag_load(&hdr->heavy_count),
                                          (unsigned long long)d.heavy_cap);
        const unsigned hd = flag_load(&hdr->heavy_done);
        ss.s_last = hd >= nh;
        if (!ss.s_last) {
          if (hd != seen_done) {  // progress: the limit restarts
            seen_done = hd;
            t_start = global_ns();
          }
          __nanosleep(128);
          if (global_ns() - t_start > 1000000000ull) {
            atomicOr(&hdr->status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
            ss.s_last = 1;
          }
        }
      }
      __syncthreads();
      if (ss.s_last) break;
    }
    if (__syncthreads_or(bad) && t == 0) set_status(hdr, SPGEMM_STATUS_ERR_BAD_INPUT);
  }
  return flop_in_smem;
}

template <int MODE>
__global__ void __launch_bounds__(kPredThreads, 1) k_predict(PredArgs p) {
  static_assert(MODE == kModePredict || MODE == kModeReference, "prediction modes only");
  extern __shared__ __align__(16) unsigned char pdyn[];
  __shared__ PredStatic ss;
  const FlopArgs& a = p.f;
  const DedupArgs& d = p.d;
  const int t = threadIdx.x;
  const int G = gridDim.x, c = blockIdx.x;
  WsHeader* hdr = a.ws.hdr;
  Slot* slots = a.ws.slots;
  const unsigned ep = *reinterpret_cast<volatile unsigned*>(&hdr->epoch) + 1u;
  const int M = (int)a.M;
  int* sflop = reinterpret_cast<int*>(pdyn + kOffSflop);
  FlopSharedT<kStreamWarps>& fs = *reinterpret_cast<FlopSharedT<kStreamWarps>*>(pdyn + kOffFlopSm);
  long long ftot = 0;  // streaming threads: FLOP of the finished rows they wrote
  if (t == 0) {
    ss.pre_ready = 0;
    ss.stream_fin = 0;
  }
  __syncthreads();

  if (t < kSampThreads) {
    // ---- sampling group: this block's slice of the sample candidates
    long long f_loc = 0, z_loc = 0, s_loc = 0;
    bool bad = false;
    if (d.N < (1ll << kSColBits)) {
      sample_batched(d, *reinterpret_cast<SampleSmem*>(pdyn), ss.red_s, f_loc, z_loc, s_loc, bad);
    } else {
      sample_per_warp(d, reinterpret_cast<int*>(pdyn), ss.list, ss.red_s, f_loc, z_loc, s_loc);
    }
    if (group_or<kBarSamp, kSampThreads>(bad) && t == 0) set_status(hdr, SPGEMM_STATUS_ERR_BAD_INPUT);
    const long long f = block_sum<kSampThreads, kBarSamp>(f_loc, ss.red_s);
    const long long z = block_sum<kSampThreads, kBarSamp>(z_loc, ss.red_s);
    const long long s = block_sum<kSampThreads, kBarSamp>(s_loc, ss.red_s);
    if (t == 0) {
      if (f) atomicAdd(&hdr->f_acc, (unsigned long long)f);
      if (z) atomicAdd(&hdr->z_acc, (unsigned long long)z);
      if (s) atomicAdd(&hdr->s_acc, (unsigned long long)s);
      __threadfence();
      atomicAdd(&hdr->sample_done, 1u);
      // f*, z* and |S| are final once every block's sampling group is done;
      // when no sampled row was queued as heavy, read them now, while the
      // streaming group is still busy, so that the prediction can start as
      // soon as the FLOP pass ends.  Stops polling when the streaming group
      // finishes first (the prediction phase then waits as usual).
      const uint64_t t0 = global_ns();
      for (unsigned ns = 64;;) {
        if (flag_load(&hdr->sample_done) >= (unsigned)G) {
          volatile WsHeader* vh = hdr;
          if (vh->heavy_count == 0) {
            const unsigned long long fv = vh->f_acc, zv = vh->z_acc;
            ss.pre[0] = fv;
            ss.pre[1] = zv;
            ss.pre[2] = vh->s_acc;
            ss.pre[3] = (MODE == kModePredict && fv && zv < fv) ? pred_recip_any(zv, fv) : 0;
            ss.pre_ready = 1;
          }
          break;
        }
        if (*reinterpret_cast<volatile int*>(&ss.stream_fin)) break;
        __nanosleep(ns);
        if (ns < 512) ns <<= 1;
        if (global_ns() - t0 > 1000000000ull) break;  // the prediction phase's waits report it
      }
    }
  } else {
    // ---- streaming group: the table share, then the FLOP of the block's rows
    constexpr int L = kSampThreads;  // the group's first thread
    const long long D = a.M + a.nnzA;
    const long long d0 = (long long)c * D / G, d1 = (long long)(c + 1) * D / G;
    bool bad = false;
    // the block's share of the B row-length table (all of a thread's loads
    // in flight at once)
    const long long tfirst = (long long)c * kStreamThreads + (t - L), tstride = (long long)G * kStreamThreads;
    DegreeBatch<kDegBatch> deg;
    deg.load(a.b_rpt, a.K, tfirst, tstride);
    deg.store(a.b_rpt, a.K, a.nnzB, a.ws.deg8, tfirst, tstride, bad);
    if (group_or<kBarStream, kStreamThreads>(bad) && t == L) set_status(hdr, SPGEMM_STATUS_ERR_BAD_INPUT);
    if (t == L) {  // this block's share of the table is written
      __threadfence();
      atomicAdd(&hdr->table_done, 1u);
    }
    // the warp's row bounds while the other blocks finish their shares
    const int sw = (t >> 5) - kSampWarps;
    long long wl0, wl1;
    merge_path_rows2(a.a_rpt, a.M, d0 + (d1 - d0) * sw / kStreamWarps, d0 + (d1 - d0) * (sw + 1) / kStreamWarps,
                     &wl0, &wl1);
    if (t == L) count_wait_short(&hdr->table_done, (unsigned)G, &hdr->status);
    group_sync<kBarStream, kStreamThreads>();
    bad = false;
    long long ptot = 0;
    flop_range<kModeFlop, kStreamWarps, kSampWarps, kBarStream>(a, d0, d1, c > 0, 0ull, 0ull, 0.0, fs, &fs.out,
                                                                ftot, ptot, bad, sflop, kSFlopN,
                                                                p.flop_out != 0, wl0, wl1);
    if (group_or<kBarStream, kStreamThreads>(bad) && t == L) set_status(hdr, SPGEMM_STATUS_ERR_BAD_INPUT);
    if (t == L) {
      const long long run = fs.out.run;
      const int i0 = fs.out.i0, i1 = fs.out.i1;
      long long extra_f = fs.out.extra_f;
      // the FLOP of a row that spans blocks (waits only on block c - 1)
      if (fs.out.dep) {
        long long cin = 0;
        if (flag_wait_short(&slots[c - 1].carry_flag, ep, &hdr->status)) cin = slots[c - 1].carry;
        slots[c].carry = cin + run;
        flag_store(&slots[c].carry_flag, ep);
      } else {
        slots[c].carry = i1 < M ? run : 0;
        flag_store(&slots[c].carry_flag, ep);
        if (fs.out.head_pending) {
          long long cin = 0;
          if (flag_wait_short(&slots[c - 1].carry_flag, ep, &hdr->status)) cin = slots[c - 1].carry;
          const long long v = cin + fs.out.head_known;
          sflop[i0 & 3] = (int)v;  // row i0 (sflop starts at row i0 & ~3)
          if (p.flop_out) a.flop[i0] = (int)v;
          extra_f += v;
        }
      }
      ss.bc[4] = extra_f;
      ss.bc[6] = i0;
      ss.bc[7] = i1;
      *reinterpret_cast<volatile int*>(&ss.stream_fin) = 1;
    }
  }
  __syncthreads();

  // ---- the block's FLOP total
  const int i0 = (int)ss.bc[6], i1 = (int)ss.bc[7];
  {
    const long long blk_f = block_sum<kPredThreads>(ftot, ss.red) + ss.bc[4];
    if (t == 0) {
      atomicAdd(&hdr->F_acc, (unsigned long long)blk_f);
      if (MODE == kModeReference) {  // F is needed before any prediction
        __threadfence();
        atomicAdd(&hdr->stream_done, 1u);
      }
    }
  }
  // no sampled row is heavy anywhere, and f*, z*, |S| are already known
  const bool pre = ss.pre_ready == 1;

  // ---- heavy sampled rows, by the whole block (none when `pre`)
  const bool flop_in_smem = pre ? true : heavy_phase(p, ss, pdyn, sflop, i0, i1);

  // ---- predictions and offsets of the rows [i0, i1)
  if (t == 0) {
    if (pre) {
      ss.bc[0] = (long long)ss.pre[0];
      ss.bc[1] = (long long)ss.pre[1];
      ss.bc[2] = (long long)ss.pre[2];
      ss.bc[5] = (long long)ss.pre[3];
    } else {
      count_wait_short(&hdr->sample_done, (unsigned)G, &hdr->status);  // heavy_count is final
      const unsigned nh = (unsigned)min((unsigned long long)flag_load(&hdr->heavy_count),
                                        (unsigned long long)d.heavy_cap);
      count_wait_short(&hdr->heavy_done, nh, &hdr->status);  // f* and z* are final
      volatile WsHeader* vh = hdr;
      const unsigned long long f = vh->f_acc, z = vh->z_acc;
      ss.bc[0] = (long long)f;
      ss.bc[1] = (long long)z;
      ss.bc[2] = (long long)vh->s_acc;
      ss.bc[5] = (MODE == kModePredict && f && z < f) ? (long long)pred_recip_any(z, f) : 0;
    }
    ss.bc[3] = 0;
    if (MODE == kModeReference) {  // F
      count_wait_short(&hdr->stream_done, (unsigned)G, &hdr->status);
      ss.bc[3] = (long long)*reinterpret_cast<volatile unsigned long long*>(&hdr->F_acc);
    }
  }
  __syncthreads();
  const unsigned long long fz = (unsigned long long)ss.bc[0], zz = (unsigned long long)ss.bc[1];
  const unsigned long long S = (unsigned long long)ss.bc[2], F = (unsigned long long)ss.bc[3];
  const unsigned long long R = (unsigned long long)ss.bc[5];
  const u128 zm = (u128)zz * (u128)(unsigned long long)a.M;
  const u128 den = (u128)F * (u128)S;
  const double ratio_ref = (MODE == kModeReference && F > 0 && S)
                               ? ((double)zz * (double)a.M) / ((double)F * (double)S)
                               : 0.0;
  bool sat = false;
  // the prediction of one row from its FLOP: ceil(flop * z* / f*), or flop
  // when f* = 0 (empty sample) or z* = f*; F32 (f* < 2^32) picks the 32-bit
  // exact ceiling, with R the matching reciprocal (pred_recip_any)
  auto predict = [&](int v, auto f32) -> int {
    if (MODE == kModePredict) {
      if (fz == 0 || zz >= fz) return v;
      if constexpr (decltype(f32)::value) {
        return pred_ceil32((uint32_t)v, (uint32_t)zz, (uint32_t)fz, (uint32_t)R);
      } else {
        return pred_fixed((uint32_t)v, zz, fz, R);
      }
    }
    return S == 0 ? v : pred_reference((uint32_t)v, zm, den, ratio_ref, &sat);
  };
  const bool f32 = fz < (1ull << 32);
  // pass 1: every prediction of the block's rows, once; it replaces the FLOP
  // in sflop (row r at sflop[r - base0] while the FLOP is there) or goes to
  // f.pred.  Thread t takes rows base0 + 4t .. + 3 of each chunk of
  // kPredThreads * 4 rows (base0 = i0 rounded down to a multiple of 4), as
  // pass 2 does.  The block total is published as soon as it is known; a
  // block of at most kScanChunks chunks then scans them while the blocks
  // before it publish theirs, keeping each thread's exclusive prefixes in
  // registers, so that only the stores remain after the wait.
  static_assert(kRowsPerThread == 4, "vector stores of 4 rows");
  constexpr int kChunkRows = kPredThreads * kRowsPerThread;
  const int base0 = i0 & ~3;
  const int s_hi = flop_in_smem ? min(i1, base0 + kSFlopN) : i0;  // rows [i0, s_hi) live in sflop
  const int nchunks = i1 > base0 ? (i1 - base0 + kChunkRows - 1) / kChunkRows : 0;
  const bool early = nchunks <= kScanChunks;
  auto pred_rows_t = [&](int r0, auto f32t) -> long long {  // predictions of rows r0 .. r0 + 3 in place; their sum
    long long l = 0;
    if (r0 >= i0 && r0 + 3 < s_hi) {  // all four in sflop: one 16-byte load and store
      int4* p4 = reinterpret_cast<int4*>(sflop + (r0 - base0));
      int4 x = *p4;
      x.x = predict(x.x, f32t);
      x.y = predict(x.y, f32t);
      x.z = predict(x.z, f32t);
      x.w = predict(x.w, f32t);
      *p4 = x;
      return (long long)x.x + x.y + x.z + x.w;
    }
#pragma unroll
    for (int u = 0; u < kRowsPerThread; ++u) {
      const int r = r0 + u;
      if (r >= i0 && r < i1) {
        const bool in_s = r < s_hi;
        const int q = predict(in_s ? sflop[r - base0] : a.flop[r], f32t);
        if (in_s) sflop[r - base0] = q; else a.pred[r] = q;
        l += q;
      }
    }
    return l;
  };
  long long lsum[kScanChunks];  // early: the thread's sum over its rows of each chunk
  long long loc = 0;
  // the whole pass for one arithmetic path (f32 is the same for every row)
  auto pass1 = [&](auto f32t) {
    if (early) {
#pragma unroll
      for (int ch = 0; ch < kScanChunks; ++ch) {
        lsum[ch] = ch < nchunks ? pred_rows_t(base0 + ch * kChunkRows + t * kRowsPerThread, f32t) : 0;
        loc += lsum[ch];
      }
    } else {
      for (int rb = base0; rb < i1; rb += kChunkRows) loc += pred_rows_t(rb + t * kRowsPerThread, f32t);
    }
  };
  if (f32) {
    pass1(std::true_type{});
  } else {
    pass1(std::false_type{});
  }
  const long long blk_p = block_sum<kPredThreads>(loc, ss.red);
  if (t == 0) {  // the total with its epoch in one word (and in full when it needs 32 bits or more)
    slots[c].total = blk_p;
    const unsigned lo = blk_p < 0xffffffffll ? (unsigned)blk_p : 0xffffffffu;
    if (lo == 0xffffffffu) __threadfence();
    word_store(&slots[c].tot_ep, ((unsigned long long)ep << 32) | lo);
  }
  long long ex_c[kScanChunks];  // early: exclusive prefix, within the block, of the thread's rows per chunk
  if (early) {
    long long run_b = 0;
#pragma unroll
    for (int ch = 0; ch < kScanChunks; ++ch) {
      ex_c[ch] = 0;
      if (ch < nchunks) {  // the same for the whole block
        long long tot;
        ex_c[ch] = block_excl_scan<kPredThreads>(lsum[ch], ss.red, &tot) + run_b;
        run_b += tot;
      }
    }
  }
  // the predictions of rows r0 .. r0 + 3 (from sflop or f.pred), 0 outside the block
  auto load_rows = [&](int r0, int* v) {
    if (r0 >= i0 && r0 + 3 < s_hi) {
      const int4 x = *reinterpret_cast<const int4*>(sflop + (r0 - base0));
      v[0] = x.x;
      v[1] = x.y;
      v[2] = x.z;
      v[3] = x.w;
      return (long long)x.x + x.y + x.z + x.w;
    }
    long long l = 0;
#pragma unroll
    for (int u = 0; u < kRowsPerThread; ++u) {
      const int r = r0 + u;
      v[u] = (r >= i0 && r < i1) ? (r < s_hi ? sflop[r - base0] : a.pred[r]) : 0;
      l += v[u];
    }
    return l;
  };
  // their stores: predictions, and offsets from ex (16-byte stores when all
  // four rows belong to the block)
  const bool vec = ((reinterpret_cast<uintptr_t>(a.pred) | reinterpret_cast<uintptr_t>(a.offsets)) & 15) == 0;
  auto store_pred = [&](int r0, const int* v) {
    if (vec && r0 >= i0 && r0 + 3 < i1) {
      *reinterpret_cast<int4*>(a.pred + r0) = make_int4(v[0], v[1], v[2], v[3]);
    } else {
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u)
        if (r0 + u >= i0 && r0 + u < i1) a.pred[r0 + u] = v[u];
    }
  };
  auto store_offsets = [&](int r0, const int* v, long long ex) {
    long long o[kRowsPerThread];
#pragma unroll
    for (int u = 0; u < kRowsPerThread; ++u) {
      o[u] = ex;
      ex += v[u];
    }
    if (vec && r0 >= i0 && r0 + 3 < i1) {
      *reinterpret_cast<longlong2*>(a.offsets + r0) = make_longlong2(o[0], o[1]);
      *reinterpret_cast<longlong2*>(a.offsets + r0 + 2) = make_longlong2(o[2], o[3]);
    } else {
#pragma unroll
      for (int u = 0; u < kRowsPerThread; ++u)
        if (r0 + u >= i0 && r0 + u < i1) a.offsets[r0 + u] = o[u];
    }
  };
  // early: the predictions do not depend on the other blocks, so they are
  // stored while the blocks before this one publish their totals
  if (early) {
#pragma unroll
    for (int ch = 0; ch < kScanChunks; ++ch) {
      if (ch < nchunks) {
        const int r0 = base0 + ch * kChunkRows + t * kRowsPerThread;
        int v[kRowsPerThread];
        load_rows(r0, v);
        store_pred(r0, v);
      }
    }
  }
  long long ppart = 0;
  for (int q = t; q < c; q += kPredThreads) ppart += slot_total(&slots[q], ep, &hdr->status);
  const long long before = block_sum<kPredThreads>(ppart, ss.red);  // predicted nnz of blocks 0 .. c-1
  if (c == G - 1 && t == 0) {
    a.offsets[a.M] = before + blk_p;
    a.res->pred_total = before + blk_p;
  }
  // every status bit of this block is set by now (saturation comes from pass 1)
  if (__syncthreads_or(sat) && t == 0) set_status(hdr, SPGEMM_STATUS_WARN_SATURATED);

  // ---- the block is done with the header and the other blocks' slots: the
  // last block to get here writes the result record and resets the header
  // while the blocks store their offsets
  if (t == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(&hdr->done, 1u);
    if (prev == (unsigned)G - 1) {
      __threadfence();
      volatile WsHeader* vh = hdr;
      unsigned st = vh->status;
      if (MODE == kModePredict ? fz == 0 : S == 0) st |= SPGEMM_STATUS_WARN_EMPTY_SAMPLE;
      a.res->flop_total = (long long)vh->F_acc;
      a.res->flop_s = (long long)fz;
      a.res->nnz_s = (long long)zz;
      a.res->n_sampled = (long long)S;
      a.res->status = (int)st;
      vh->f_acc = 0;
      vh->z_acc = 0;
      vh->s_acc = 0;
      vh->F_acc = 0;
      vh->heavy_count = 0;
      vh->status = 0;
      vh->table_done = 0;
      vh->sample_done = 0;
      vh->heavy_ctr = 0;
      vh->heavy_done = 0;
      vh->stream_done = 0;
      vh->done = 0;
      __threadfence();
      vh->epoch = ep;
    }
  }
  // pass 2: the offsets (with the predictions, for a block of more chunks)
  if (early) {
#pragma unroll
    for (int ch = 0; ch < kScanChunks; ++ch) {
      if (ch < nchunks) {
        const int r0 = base0 + ch * kChunkRows + t * kRowsPerThread;
        int v[kRowsPerThread];
        load_rows(r0, v);
        store_offsets(r0, v, before + ex_c[ch]);
      }
    }
  } else {
    long long run = before;
    for (int rb = base0; rb < i1; rb += kChunkRows) {
      const int r0 = rb + t * kRowsPerThread;
      int v[kRowsPerThread];
      long long tot;
      const long long ex = block_excl_scan<kPredThreads>(load_rows(r0, v), ss.red, &tot) + run;
      store_pred(r0, v);
      store_offsets(r0, v, ex);
      run += tot;
    }
  }
}

}  // namespace spg
