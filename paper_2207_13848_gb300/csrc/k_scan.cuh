// Ordered per-row scans over co-resident blocks (exact nnz -> offsets for the
// symbolic phase; sampled-row flags -> ascending sample ids), CSR validation,
// and the finalisation of the sampling-only call.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace spg {

constexpr int kScanThreads = 512;
constexpr int kScanRows = 4;  // rows per thread per step

// Values: exact nnz per row; output: offsets (M + 1 entries).
struct ScanNnz {
  const int* vals;
  long long* offsets;
  __device__ int value(long long r) const { return vals[r]; }
  __device__ void emit(long long r, long long excl, int) const { offsets[r] = excl; }
  __device__ void finish(long long n, long long total, spgemm_result_t* res) const {
    offsets[n] = total;
    res->pred_total = total;
  }
};

// Values: exact nnz per row of a numeric product; output: the exact CSR's
// offsets (M + 1 entries).  The result record keeps its fields.
struct ScanNumNnz {
  const int* vals;
  long long* offsets;
  __device__ int value(long long r) const { return vals[r]; }
  __device__ void emit(long long r, long long excl, int) const { offsets[r] = excl; }
  __device__ void finish(long long n, long long total, spgemm_numeric_result_t*) const { offsets[n] = total; }
};

// Values: 1 if the candidate is in the sample; output: its row id at position excl.
struct ScanSample {
  int mode;
  uint64_t seed, threshold;
  long long M;
  int* ids;
  long long capacity;
  __device__ int value(long long r) const {
    if (mode == SPGEMM_SAMPLE_BERNOULLI) return (uint64_t)sample_hash32(seed, (uint64_t)r) < threshold ? 1 : 0;
    return 1;
  }
  __device__ void emit(long long r, long long excl, int v) const {
    if (!v || excl >= capacity) return;
    if (mode == SPGEMM_SAMPLE_BERNOULLI)
      ids[excl] = (int)r;
    else
      ids[excl] = (int)(((uint64_t)sample_hash32(seed, (uint64_t)r) * (uint64_t)M) >> 32);
  }
  __device__ void finish(long long, long long total, spgemm_result_t* res) const {
    res->n_sampled = total;
  }
};

// Block c takes items [c*n/G, (c+1)*n/G): sums them, publishes the sum, adds the
// sums of blocks 0..c-1 (bounded waits) and writes the exclusive prefixes.
// The last block to finish copies the workspace accumulators into *res
// (flop_total = flop_s = f_acc, nnz_s = z_acc, n_sampled = s_acc unless the
// source writes it) and resets them; a numeric result record only gains the
// status bits.
template <class Src, bool SYMBOLIC, class Res = spgemm_result_t>
__global__ void __launch_bounds__(kScanThreads) k_scan_rows(Src src, long long n, Workspace ws, Res* res) {
  __shared__ long long red[kScanThreads / 32 + 1];
  const int t = threadIdx.x, G = gridDim.x, c = blockIdx.x;
  WsHeader* hdr = ws.hdr;
  const unsigned ep = *reinterpret_cast<volatile unsigned*>(&hdr->epoch) + 1u;
  const long long b = (long long)c * n / G, e = (long long)(c + 1) * n / G;
  long long loc = 0;
  for (long long r = b + t; r < e; r += kScanThreads) loc += src.value(r);
  const long long blk = block_sum<kScanThreads>(loc, red);
  if (t == 0) {
    ws.slots[c].total = blk;
    flag_store(&ws.slots[c].total_flag, ep);
  }
  long long pp = 0;
  for (int q = t; q < c; q += kScanThreads)
    if (flag_wait(&ws.slots[q].total_flag, ep, &hdr->status))
      pp += *reinterpret_cast<volatile long long*>(&ws.slots[q].total);
  long long run = block_sum<kScanThreads>(pp, red);
  for (long long rb = b; rb < e; rb += (long long)kScanThreads * kScanRows) {
    const long long r0 = rb + (long long)t * kScanRows;
    int v[kScanRows];
    long long l = 0;
#pragma unroll
    for (int u = 0; u < kScanRows; ++u) {
      v[u] = (r0 + u < e) ? src.value(r0 + u) : 0;
      l += v[u];
    }
    long long tot;
    long long ex = block_excl_scan<kScanThreads>(l, red, &tot) + run;
#pragma unroll
    for (int u = 0; u < kScanRows; ++u) {
      if (r0 + u < e) src.emit(r0 + u, ex, v[u]);
      ex += v[u];
    }
    run += tot;
  }
  if (c == G - 1 && t == 0) src.finish(n, run, res);
  __syncthreads();
  if (t == 0) {
    __threadfence();
    if (atomicAdd(&hdr->done, 1u) == (unsigned)G - 1) {
      __threadfence();
      volatile WsHeader* vh = hdr;
      if constexpr (std::is_same<Res, spgemm_result_t>::value) {
        if (SYMBOLIC) {
          res->flop_total = (long long)vh->f_acc;
          res->flop_s = (long long)vh->f_acc;
          res->nnz_s = (long long)vh->z_acc;
          res->n_sampled = (long long)vh->s_acc;
        } else {
          res->flop_total = 0;
          res->flop_s = 0;
          res->nnz_s = 0;
          res->pred_total = 0;
        }
        res->status = (int)vh->status;
      } else {
        res->status |= (int)vh->status;
      }
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

// Finalisation of spgemm_predict_cr: one thread copies the accumulators.
__global__ void k_finalize_cr(Workspace ws, spgemm_result_t* res) {
  volatile WsHeader* vh = ws.hdr;
  unsigned st = vh->status;
  if (vh->f_acc == 0) st |= SPGEMM_STATUS_WARN_EMPTY_SAMPLE;
  res->flop_total = 0;
  res->flop_s = (long long)vh->f_acc;
  res->nnz_s = (long long)vh->z_acc;
  res->n_sampled = (long long)vh->s_acc;
  res->pred_total = 0;
  res->status = (int)st;
  vh->f_acc = 0;
  vh->z_acc = 0;
  vh->s_acc = 0;
  vh->F_acc = 0;
  vh->heavy_count = 0;
  vh->status = 0;
}

// CSR validation: one warp per row.  Offsets in range and non-decreasing,
// rpt[0] = 0 and rpt[rows] = nnz, ids in [0, cols), rows strictly increasing.
constexpr int kValThreads = 256;
__global__ void __launch_bounds__(kValThreads) k_validate(long long rows, long long cols, long long nnz,
                                                         const int* rpt, const int* col, Workspace ws,
                                                         spgemm_result_t* res) {
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * kValThreads + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * kValThreads) >> 5;
  unsigned st = 0;
  if (gw == 0 && lane == 0) {
    if (__ldg(rpt) != 0 || (long long)__ldg(rpt + rows) != nnz) st |= SPGEMM_STATUS_ERR_BAD_INPUT;
  }
  for (long long r = gw; r < rows; r += nwarps) {
    long long b = __ldg(rpt + r), e = __ldg(rpt + r + 1);
    if (b < 0 || e < b || e > nnz) {
      st |= SPGEMM_STATUS_ERR_BAD_INPUT;
      continue;
    }
    for (long long j = b + lane; j < e; j += 32) {
      const int x = __ldg(col + j);
      if (x < 0 || (long long)x >= cols) st |= SPGEMM_STATUS_ERR_BAD_INPUT;
      if (j + 1 < e && __ldg(col + j + 1) <= x) st |= SPGEMM_STATUS_WARN_UNSORTED;
    }
  }
  st = __reduce_or_sync(kFull, st);
  if (lane == 0 && st) atomicOr(&ws.hdr->status, st);
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&ws.hdr->done, 1u) == gridDim.x - 1) {
      __threadfence();
      volatile WsHeader* vh = ws.hdr;
      res->flop_total = 0;
      res->flop_s = 0;
      res->nnz_s = 0;
      res->n_sampled = 0;
      res->pred_total = 0;
      res->status = (int)vh->status;
      vh->status = 0;
      vh->done = 0;
    }
  }
}

}  // namespace spg
