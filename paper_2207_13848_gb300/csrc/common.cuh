// Device helpers shared by the kernels of the structure predictor: the sample
// hash, exact integer rounding, warp/block scans, inter-block flags with
// bounded waits, and the workspace layout.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/spgemm_predict.h"

namespace spg {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xffffffffu;

// Maximum number of thread blocks of one inter-block (persistent) launch; one
// 64-byte slot per block lives in the workspace.
constexpr int kMaxSlots = 4096;

// ---------------------------------------------------------------------------
// Workspace layout.  Everything here starts at zero (the caller zero-fills the
// workspace once) and every successful call returns it to zero, except `epoch`,
// which only grows: a flag counts as set when it equals the epoch of the
// current launch, so flags never need clearing.
// ---------------------------------------------------------------------------
struct alignas(128) WsHeader {
  unsigned long long f_acc;  // sum of sampled flop (f*)
  unsigned long long z_acc;  // sum of sampled nnz (z*)
  unsigned long long s_acc;  // number of sampled rows (|S|)
  unsigned long long F_acc;  // total flop (F) where a kernel accumulates it
  unsigned int heavy_count;  // rows queued for the block-per-row pass
  unsigned int status;       // SPGEMM_STATUS_* bits (atomicOr)
  unsigned int epoch;        // flag epoch of the previous completed launch
  unsigned int done;         // blocks finished in the current launch
  // progress counters of the single-launch predictor (k_predict)
  unsigned int table_done;   // blocks whose share of the B row-length table is written
  unsigned int sample_done;  // blocks whose sampled rows are counted or queued
  unsigned int heavy_ctr;    // heavy-queue entries claimed
  unsigned int heavy_done;   // heavy rows counted
  unsigned int stream_done;  // blocks whose FLOP pass is finished
  unsigned int pad[19];
};
static_assert(sizeof(WsHeader) == 256, "workspace header layout");

struct alignas(64) Slot {
  unsigned int carry_flag;  // = epoch when `carry` is valid
  unsigned int total_flag;  // = epoch when `total` is valid
  unsigned int ftot_flag;   // = epoch when `ftot` is valid
  unsigned int pad0;
  long long carry;  // partial FLOP of the row open at the block's end
  long long total;  // sum of the block's per-row values (pred or nnz)
  long long ftot;   // sum of the block's complete-row FLOP
  unsigned long long tot_ep;  // (epoch << 32) | total, or | 0xffffffff when total
                              // needs 32 bits or more (then read `total`)
  unsigned long long pool;    // numeric product, pool mode: entries taken from stripe s (slot s)
  long long pad1;
};

// A sampled row with very many products is split by its entries into parts
// that several blocks count at once, each into a shared-memory bitmap over B's
// columns that it writes out whole to its own bitmap in the workspace; the
// block that finishes the row's last part ORs the parts' bitmaps and counts.
constexpr int kHugeSlots = 8;    // split rows in progress at once
constexpr int kMaxParts = 8;     // parts of one split row
struct alignas(64) HugeSlot {
  unsigned int state;       // 0 free, 1 being set up, 2 parts claimable
  unsigned int parts;       // number of parts
  unsigned int part_ctr;    // parts claimed (parked high while being set up)
  unsigned int parts_done;  // parts counted
  long long bnd[kMaxParts + 1];  // part p = A entries [bnd[p], bnd[p + 1])
};

struct Workspace {
  WsHeader* hdr;
  Slot* slots;
  int* heavy;            // [M] rows queued for the block-per-row deduplication
  int* flop_buf;         // [M] per-row FLOP when the caller gives no flop_row buffer
  unsigned char* deg8;   // [K] B row lengths capped at kDegEscape (see k_degree_table)
  HugeSlot* huge;        // [kHugeSlots] split rows (when carved with N > 0)
  unsigned int* hbits;   // [kHugeSlots][kMaxParts][huge_words] the parts' bitmaps over B's columns
  long long huge_words;  // words of one bitmap (0 when not carved)
};

// B row lengths of at least kDegEscape are read from B.rpt instead of the table.
constexpr int kDegEscape = 255;

constexpr size_t ws_round(size_t b) { return ((b + 255) / 256) * 256; }
constexpr long long ws_huge_words(int64_t N) { return N > 0 ? (N + 2047) / 2048 * 64 : 0; }

// Bytes for M rows of A, K columns of A (= rows of B) and N columns of B (the
// split-row bitmaps; N = 0 leaves them out).  The regions that must read as
// zero when a call starts (header, block slots, split-row slots) sit at fixed
// offsets, so a workspace left clean by one call is clean for any later call
// whose operands it is large enough for, whatever their shapes; the regions
// whose place depends on M, K and N are written by a call before it reads them
// (the heavy-row queue is read only below the count of entries queued).
constexpr size_t ws_bytes_for(int64_t M, int64_t K, int64_t N = 0) {
  const size_t m = (size_t)(M > 0 ? M : 1), k = (size_t)(K > 0 ? K : 1);
  size_t b = sizeof(WsHeader) + sizeof(Slot) * kMaxSlots + sizeof(HugeSlot) * kHugeSlots + 2 * ws_round(m * 4) +
             ws_round(k + 16);
  if (N > 0) b += (size_t)kHugeSlots * kMaxParts * (size_t)ws_huge_words(N) * 4;
  return b;
}

inline Workspace ws_carve(void* base, int64_t M, int64_t K = 0, int64_t N = 0) {
  const size_t m = (size_t)(M > 0 ? M : 1), k = (size_t)(K > 0 ? K : 1);
  char* p = static_cast<char*>(base);
  Workspace w;
  w.hdr = reinterpret_cast<WsHeader*>(p);
  p += sizeof(WsHeader);
  w.slots = reinterpret_cast<Slot*>(p);
  p += sizeof(Slot) * kMaxSlots;
  w.huge = N > 0 ? reinterpret_cast<HugeSlot*>(p) : nullptr;
  p += sizeof(HugeSlot) * kHugeSlots;
  w.heavy = reinterpret_cast<int*>(p);
  p += ws_round(m * 4);
  w.flop_buf = reinterpret_cast<int*>(p);
  p += ws_round(m * 4);
  w.deg8 = reinterpret_cast<unsigned char*>(p);
  p += ws_round(k + 16);
  w.hbits = N > 0 ? reinterpret_cast<unsigned int*>(p) : nullptr;
  w.huge_words = ws_huge_words(N);
  return w;
}

// ---------------------------------------------------------------------------
// Sample hash: SplitMix64 (Steele, Lea, Flood, OOPSLA 2014).  The state of the
// generator started at `seed` after k steps is seed + k * gamma with gamma =
// 0x9e3779b97f4a7c15; an output is the state passed through the finaliser
// (xor-shift 30, multiply 0xbf58476d1ce4e5b9, xor-shift 27, multiply
// 0x94d049bb133111eb, xor-shift 31).  h32(seed, x) takes output x + 1's high
// half.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t sample_hash32(uint64_t seed, uint64_t x) {
  uint64_t s = seed + (x + 1ull) * 0x9e3779b97f4a7c15ull;
  s ^= s >> 30;
  s *= 0xbf58476d1ce4e5b9ull;
  s ^= s >> 27;
  s *= 0x94d049bb133111ebull;
  s ^= s >> 31;
  return (uint32_t)(s >> 32);
}

// ---------------------------------------------------------------------------
// Exact rounding of the per-row prediction without integer division: q is
// estimated in double precision, then moved to the exact ceiling with 128-bit
// products (the estimate is off by at most one for q < 2^32, so the loops run
// at most a couple of times; they are bounded regardless).
// ---------------------------------------------------------------------------
typedef unsigned __int128 u128;

// ceil(v * z / f) for 0 < v < 2^31, 0 < z <= f < 2^63 (so the result is <= v).
__device__ __forceinline__ int pred_proposed(uint32_t v, uint64_t z, uint64_t f, double ratio) {
  if (v == 0) return 0;
  const u128 num = (u128)v * z;
  uint64_t q = (uint64_t)((double)v * ratio);
  if (q > v) q = v;
#pragma unroll 1
  for (int it = 0; it < 8 && (u128)q * f < num; ++it) ++q;
#pragma unroll 1
  for (int it = 0; it < 8 && q > 0 && (u128)(q - 1) * f >= num; ++it) --q;
  return (int)q;
}

// The same ceiling without floating point, for a whole launch's rows: R =
// floor(z * 2^64 / f) is prepared once (pred_recip, for 0 < z < f); then
// q = floor(v * R / 2^64) is floor(v * z / f) or one less, and the exact ceiling
// is q, q + 1 or q + 2, decided by two 128-bit comparisons with v * z.
__host__ __device__ __forceinline__ uint64_t pred_recip(uint64_t z, uint64_t f) {
  return (uint64_t)(((u128)z << 64) / (u128)f);
}
// pred_recip without a 128-bit division: a double estimate, then the exact
// correction from the 128-bit remainder (the estimate is within 2^13 of R, so
// one more double step and a final +-1 adjustment are exact).
__host__ __device__ __forceinline__ uint64_t pred_recip_fast(uint64_t z, uint64_t f) {
  const double ratio = (double)z / (double)f;                       // in [0, 1)
  uint64_t R = ratio >= 1.0 ? ~0ull : (uint64_t)(ratio * 18446744073709551616.0);
  const u128 num = (u128)z << 64;
  // r = num - R * f, signed; |r| < 2^14 * f
  const u128 prod = (u128)R * f;
  if (prod <= num) {
    const u128 r = num - prod;
    R += (uint64_t)((double)r / (double)f);
  } else {
    const u128 r = prod - num;
    R -= (uint64_t)((double)r / (double)f) + 1;
  }
  // final exact adjustment: R * f <= num < (R + 1) * f
#pragma unroll 1
  for (int it = 0; it < 4 && (u128)R * f > num; ++it) --R;
#pragma unroll 1
  for (int it = 0; it < 4 && (u128)(R + 1) * f <= num; ++it) ++R;
  return R;
}

__host__ __device__ __forceinline__ int pred_fixed(uint32_t v, uint64_t z, uint64_t f, uint64_t R) {
#ifdef __CUDA_ARCH__
  uint64_t q = __umul64hi((uint64_t)v, R);
#else
  uint64_t q = (uint64_t)(((u128)v * R) >> 64);
#endif
  if (f < (1ull << 32)) {  // then v * z and (q + 2) * f stay below 2^64
    const uint64_t num = (uint64_t)v * z;
    if (q * f >= num) return (int)q;
    ++q;
    if (q * f >= num) return (int)q;
    return (int)(q + 1);
  }
  const u128 num = (u128)v * z;
  if ((u128)q * f >= num) return (int)q;
  ++q;
  if ((u128)q * f >= num) return (int)q;
  return (int)(q + 1);
}

// ceil(v * z / f) for f < 2^32 (and z < f), with R32 = floor(z * 2^32 / f):
// v * R32 / 2^32 <= v * z / f < v * R32 / 2^32 + v / 2^32, and v < 2^32, so
// q = floor(v * R32 / 2^32) is floor(v * z / f) or one less; the remainder
// v * z - q * f (64-bit products of 32-bit operands, in [0, 2f)) settles it.
__host__ __device__ __forceinline__ uint32_t pred_recip32(uint32_t z, uint32_t f) {
  return (uint32_t)(((uint64_t)z << 32) / f);
}
__host__ __device__ __forceinline__ int pred_ceil32(uint32_t v, uint32_t z, uint32_t f, uint32_t R32) {
#ifdef __CUDA_ARCH__
  uint32_t q = __umulhi(v, R32);
#else
  uint32_t q = (uint32_t)(((uint64_t)v * R32) >> 32);
#endif
  uint64_t r = (uint64_t)v * z - (uint64_t)q * f;
  if (r >= f) {
    ++q;
    r -= f;
  }
  return (int)(q + (r != 0));
}
// The reciprocal that pred_fast takes (z < f): 32-bit when f < 2^32, else 64.64.
__host__ __device__ __forceinline__ uint64_t pred_recip_any(uint64_t z, uint64_t f) {
  return f < (1ull << 32) ? pred_recip32((uint32_t)z, (uint32_t)f) : pred_recip_fast(z, f);
}
// ceil(v * z / f) for z < f, with R = pred_recip_any(z, f).
__host__ __device__ __forceinline__ int pred_fast(uint32_t v, uint64_t z, uint64_t f, uint64_t R) {
  return f < (1ull << 32) ? pred_ceil32(v, (uint32_t)z, (uint32_t)f, (uint32_t)R) : pred_fixed(v, z, f, R);
}

// ceil(v * zm / den) for the reference design: zm = z * M (< 2^94),
// den = F * |S| (< 2^94).  Saturates at 2^31 - 1 and reports it via *sat.
__device__ __forceinline__ int pred_reference(uint32_t v, u128 zm, u128 den, double ratio,
                                              bool* sat) {
  if (v == 0) return 0;
  const double est = (double)v * ratio;
  if (est > 2147483700.0) {
    *sat = true;
    return 2147483647;
  }
  const u128 num = (u128)v * zm;
  uint64_t q = (uint64_t)est;
#pragma unroll 1
  for (int it = 0; it < 8 && (u128)q * den < num; ++it) ++q;
#pragma unroll 1
  for (int it = 0; it < 8 && q > 0 && (u128)(q - 1) * den >= num; ++it) --q;
  if (q > 2147483647ull) {
    *sat = true;
    return 2147483647;
  }
  return (int)q;
}

// ---------------------------------------------------------------------------
// Warp and block scans / reductions (int64).
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(kFull, v, o);
    if (lane >= o) v += n;
  }
  return v;
}

// ---------------------------------------------------------------------------
// Thread groups: the NT threads of warps [WOFF, WOFF + NT/32) of a block,
// synchronised by hardware barrier BAR (0 = the whole block, __syncthreads).
// Every thread of the group must reach each call.
// ---------------------------------------------------------------------------
template <int BAR, int NT>
__device__ __forceinline__ void group_sync() {
  if (BAR == 0) {
    __syncthreads();
  } else {
    asm volatile("bar.sync %0, %1;" ::"r"(BAR), "r"(NT) : "memory");
  }
}

// Number of threads of the group with p true (a barrier, like __syncthreads_count).
template <int BAR, int NT>
__device__ __forceinline__ int group_count(bool p) {
  if (BAR == 0) return __syncthreads_count(p);
  unsigned n;
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n bar.red.popc.u32 %0, %2, %3, q;\n}"
      : "=r"(n)
      : "r"((unsigned)p), "r"(BAR), "r"(NT)
      : "memory");
  return (int)n;
}

template <int BAR, int NT>
__device__ __forceinline__ bool group_or(bool p) {
  if (BAR == 0) return __syncthreads_or(p);
  return group_count<BAR, NT>(p) != 0;
}

// Group-wide exclusive scan of one value per thread; returns the exclusive
// prefix and writes the group total to *total.  `sm` needs NT/32 + 1 entries.
template <int NT, int BAR = 0, int WOFF = 0>
__device__ __forceinline__ long long block_excl_scan(long long v, long long* sm, long long* total) {
  constexpr int NW = NT / 32;
  const int lane = threadIdx.x & 31, w = (int)(threadIdx.x >> 5) - WOFF;
  long long inc = warp_incl_scan(v);
  if (lane == 31) sm[w] = inc;
  group_sync<BAR, NT>();
  if (w == 0) {
    long long t = lane < NW ? sm[lane] : 0;
    long long ti = warp_incl_scan(t);
    if (lane < NW) sm[lane] = ti - t;
    if (lane == NW - 1) sm[NW] = ti;
  }
  group_sync<BAR, NT>();
  long long r = sm[w] + inc - v;
  *total = sm[NW];
  group_sync<BAR, NT>();
  return r;
}

template <int NT, int BAR = 0, int WOFF = 0>
__device__ __forceinline__ long long block_sum(long long v, long long* sm) {
  long long t;
  block_excl_scan<NT, BAR, WOFF>(v, sm, &t);
  return t;
}

// ---------------------------------------------------------------------------
// Inter-block flags: release/acquire at GPU scope, bounded waits.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void flag_store(unsigned int* p, unsigned int v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned int flag_load(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void word_store(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long word_load(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits until *p == want; gives up after about one second (or 2^26 polls),
// sets SPGEMM_STATUS_ERR_TIMEOUT and returns false.
__device__ __noinline__ bool flag_wait(const unsigned int* p, unsigned int want,
                                       unsigned int* status) {
  if (flag_load(p) == want) return true;
  const uint64_t t0 = global_ns();
  unsigned ns = 32;
  for (int it = 0; it < (1 << 26); ++it) {
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    if (flag_load(p) == want) return true;
    if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) break;
  }
  atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
  return false;
}

// flag_wait for waits expected to be short: polls every 64 ns or so.
__device__ __noinline__ bool flag_wait_short(const unsigned int* p, unsigned int want,
                                             unsigned int* status) {
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (flag_load(p) == want) return true;
    __nanosleep(64);
    if ((it & 255) == 255 && global_ns() - t0 > 1000000000ull) break;
  }
  atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
  return false;
}

// count_wait for waits expected to be short: polls every 64 ns or so.
__device__ __noinline__ bool count_wait_short(const unsigned int* p, unsigned int want,
                                              unsigned int* status) {
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    if (flag_load(p) >= want) return true;
    __nanosleep(64);
    if ((it & 255) == 255 && global_ns() - t0 > 1000000000ull) break;
  }
  atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
  return false;
}

// The block total published in slot->tot_ep for epoch ep (one load in the
// common case); polls every 64 ns or so and gives up like flag_wait.
__device__ __noinline__ long long slot_total(const Slot* slot, unsigned ep, unsigned int* status) {
  const uint64_t t0 = global_ns();
  for (int it = 0; it < (1 << 26); ++it) {
    const unsigned long long w = word_load(&slot->tot_ep);
    if ((unsigned)(w >> 32) == ep) {
      const unsigned lo = (unsigned)w;
      return lo != 0xffffffffu ? (long long)lo : *reinterpret_cast<const volatile long long*>(&slot->total);
    }
    __nanosleep(64);
    if ((it & 255) == 255 && global_ns() - t0 > 1000000000ull) break;
  }
  atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
  return 0;
}

// Waits until *p >= want (a counter that only grows within a launch); gives up
// like flag_wait.
__device__ __noinline__ bool count_wait(const unsigned int* p, unsigned int want, unsigned int* status) {
  if (flag_load(p) >= want) return true;
  const uint64_t t0 = global_ns();
  unsigned ns = 32;
  for (int it = 0; it < (1 << 26); ++it) {
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
    if (flag_load(p) >= want) return true;
    if ((it & 63) == 63 && global_ns() - t0 > 1000000000ull) break;
  }
  atomicOr(status, (unsigned)SPGEMM_STATUS_ERR_TIMEOUT);
  return false;
}

__device__ __forceinline__ void set_status(WsHeader* h, unsigned bits) { atomicOr(&h->status, bits); }

// Byte table of B's row lengths: deg8[k] = min(B.rpt[k+1] - B.rpt[k], kDegEscape).
// Lookups into this 1-byte table replace the pair of B.rpt loads per nonzero
// in the FLOP pass (fewer L2 sectors and more L1 reuse); kDegEscape means
// "read B.rpt".  Offsets out of range give 0 and set *bad.  Thread `first` of
// `nthreads` writes the 4-row words first, first + nthreads, ...
// The table word of rows [k0, k0 + 4) from v[u] = B.rpt[k0 + u] (u <= 4, entries past K unused).
__device__ __forceinline__ unsigned degree_word(const int* v, long long k0, long long K, long long nnzB,
                                                bool& bad) {
  unsigned word = 0;
  long long prev = v[0];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    if (k0 + u < K) {
      const long long next = v[u + 1];
      long long d = next - prev;
      if (d < 0 || prev < 0 || next > nnzB) {
        bad = true;
        d = 0;
      }
      word |= (unsigned)(d < kDegEscape ? d : kDegEscape) << (8 * u);
      prev = next;
    }
  }
  return word;
}

__device__ __forceinline__ void degree_words(const int* b_rpt, long long K, long long nnzB,
                                             unsigned char* deg8, long long first, long long nthreads,
                                             bool& bad) {
  for (long long k0 = first * 4; k0 < K; k0 += nthreads * 4) {
    int v[5];
#pragma unroll
    for (int u = 0; u < 5; ++u) v[u] = k0 + u <= K ? __ldg(b_rpt + k0 + u) : 0;
    *reinterpret_cast<unsigned*>(deg8 + k0) = degree_word(v, k0, K, nnzB, bad);
  }
}

// degree_words with the loads of the thread's first NB words issued at once:
// load() reads their B.rpt entries, store() writes those words and then the
// thread's remaining ones.
template <int NB>
struct DegreeBatch {
  int v[NB][5];
  __device__ __forceinline__ void load(const int* b_rpt, long long K, long long first, long long nthreads) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const long long k0 = (first + b * nthreads) * 4;
#pragma unroll
      for (int u = 0; u < 5; ++u) v[b][u] = k0 + u <= K ? __ldg(b_rpt + k0 + u) : 0;
    }
  }
  __device__ __forceinline__ void store(const int* b_rpt, long long K, long long nnzB, unsigned char* deg8,
                                        long long first, long long nthreads, bool& bad) {
#pragma unroll
    for (int b = 0; b < NB; ++b) {
      const long long k0 = (first + b * nthreads) * 4;
      if (k0 < K) *reinterpret_cast<unsigned*>(deg8 + k0) = degree_word(v[b], k0, K, nnzB, bad);
    }
    degree_words(b_rpt, K, nnzB, deg8, first + NB * nthreads, nthreads, bad);
  }
};

__global__ void k_degree_table(const int* b_rpt, long long K, long long nnzB, unsigned char* deg8,
                               WsHeader* hdr) {
  bool bad = false;
  degree_words(b_rpt, K, nnzB, deg8, (long long)blockIdx.x * blockDim.x + threadIdx.x,
               (long long)gridDim.x * blockDim.x, bad);
  if (bad) atomicOr(&hdr->status, (unsigned)SPGEMM_STATUS_ERR_BAD_INPUT);
}

// Clamp a row range [b, e) read from untrusted offsets into [0, nnz].
__device__ __forceinline__ bool clamp_range(long long& b, long long& e, long long nnz) {
  bool ok = (b >= 0) & (e >= b) & (e <= nnz);
  if (b < 0) b = 0;
  if (b > nnz) b = nnz;
  if (e > nnz) e = nnz;
  if (e < b) e = b;
  return ok;
}

}  // namespace spg
