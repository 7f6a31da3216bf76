// Roofline calibration for the FLOP pass: the same memory access pattern
// (a stream of column ids with one scattered one-byte table lookup per id)
// with nothing else, so that its rate is the ceiling of the pass on this
// device.  The paper has no counterpart; the benchmark times it beside the
// prediction.
#pragma once

#include "common.cuh"

namespace spg {

constexpr int kProbeThreads = 1024;
constexpr int kProbeItems = 16;  // ids per lane per step (four 16-byte loads)

// Warp w of the grid takes the aligned 512-id steps [w0, w1) of col; ids past
// the last whole step are looked up one per thread.  Ids outside [0, tab_n)
// count as zero.  The sum of the looked-up bytes goes to *out.
__global__ void __launch_bounds__(kProbeThreads, 1)
    k_lookup_probe(const int* __restrict__ col, long long n, const unsigned char* tab, long long tab_n,
                   unsigned long long* out) {
  constexpr int SUB = 32 * kProbeItems;
  const int lane = threadIdx.x & 31;
  const long long gw = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nw = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long nsteps = n / SUB;
  const long long w0 = gw * nsteps / nw * SUB, w1 = (gw + 1) * nsteps / nw * SUB;
  unsigned acc = 0;
  for (long long s = w0; s < w1; s += SUB) {
    int c[kProbeItems];
#pragma unroll
    for (int h = 0; h < kProbeItems / 4; ++h) {
      const int4 x = __ldg(reinterpret_cast<const int4*>(col + s + 4 * lane + 128 * h));
      c[4 * h] = x.x;
      c[4 * h + 1] = x.y;
      c[4 * h + 2] = x.z;
      c[4 * h + 3] = x.w;
    }
    unsigned l[kProbeItems];
#pragma unroll
    for (int u = 0; u < kProbeItems; ++u) l[u] = (unsigned)c[u] < (unsigned long long)tab_n ? tab[c[u]] : 0u;
#pragma unroll
    for (int u = 0; u < kProbeItems; ++u) acc += l[u];
  }
  for (long long j = nsteps * SUB + (long long)blockIdx.x * blockDim.x + threadIdx.x; j < n;
       j += (long long)gridDim.x * blockDim.x) {
    const int cc = __ldg(col + j);
    acc += (unsigned)cc < (unsigned long long)tab_n ? tab[cc] : 0u;
  }
  acc = __reduce_add_sync(kFull, acc);
  if (lane == 0) atomicAdd(out, (unsigned long long)acc);
}

}  // namespace spg
