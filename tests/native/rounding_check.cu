// Host-side check of the exact per-row rounding helpers of the CUDA library
// (common.cuh): pred_recip_fast must equal floor(z * 2^64 / f) computed by
// 128-bit division, and pred_fixed must equal ceil(v * z / f), on random and
// edge operands; so must pred_fast with pred_recip_any (the 32-bit reciprocal
// floor(z * 2^32 / f) when f < 2^32).  Built by nvcc as host code only; prints "ok N" or the first
// mismatch and exits non-zero.
#include <cstdio>
#include <cstdint>
#include "../../paper_2207_13848_gb300/csrc/common.cuh"

using spg::u128;

static uint64_t rng_state = 0x243F6A8885A308D3ull;
static uint64_t next64() {  // xorshift64*
  rng_state ^= rng_state >> 12;
  rng_state ^= rng_state << 25;
  rng_state ^= rng_state >> 27;
  return rng_state * 0x2545F4914F6CDD1Dull;
}

static int check(uint64_t z, uint64_t f, uint32_t v) {
  const uint64_t R = spg::pred_recip_fast(z, f);
  const uint64_t Rx = (uint64_t)(((u128)z << 64) / f);
  if (R != Rx) {
    printf("recip mismatch z=%llu f=%llu got %llu want %llu\n", (unsigned long long)z, (unsigned long long)f,
           (unsigned long long)R, (unsigned long long)Rx);
    return 1;
  }
  const u128 num = (u128)v * z;
  const uint64_t want = (uint64_t)((num + f - 1) / f);
  const int got = spg::pred_fixed(v, z, f, R);
  if ((uint64_t)got != want) {
    printf("ceil mismatch v=%u z=%llu f=%llu got %d want %llu\n", v, (unsigned long long)z, (unsigned long long)f, got,
           (unsigned long long)want);
    return 1;
  }
  // the path the prediction kernel takes: 32-bit reciprocal when f < 2^32
  const uint64_t Ra = spg::pred_recip_any(z, f);
  const uint64_t Rw = f < (1ull << 32) ? (uint64_t)(((u128)z << 32) / f) : Rx;
  const int got2 = spg::pred_fast(v, z, f, Ra);
  if (Ra != Rw || (uint64_t)got2 != want) {
    printf("fast-path mismatch v=%u z=%llu f=%llu R %llu (want %llu) got %d want %llu\n", v, (unsigned long long)z,
           (unsigned long long)f, (unsigned long long)Ra, (unsigned long long)Rw, got2, (unsigned long long)want);
    return 1;
  }
  return 0;
}

int main() {
  long n = 0;
  // edges: z close to f, f near 2^32 (both arithmetic paths), near 2^63, tiny
  const uint64_t fs[] = {1, 2, 3, 7, 1000, (1ull << 32) - 1, 1ull << 32, (1ull << 32) + 1, 1ull << 40,
                         (1ull << 62) + 12345, (1ull << 63) - 1};
  const uint32_t vs[] = {0, 1, 2, 3, 255, 65536, 2147483647u};
  for (uint64_t f : fs) {
    const uint64_t zs[] = {0, 1, f / 2, f > 1 ? f - 1 : 0, f / 3, (f / 7) * 5};
    for (uint64_t z : zs) {
      if (z >= f && f > 1) continue;
      if (z >= f) continue;
      for (uint32_t v : vs) {
        if (check(z, f, v)) return 1;
        ++n;
      }
    }
  }
  for (int i = 0; i < 2000000; ++i) {
    const int bits = 1 + (int)(next64() % 63);
    uint64_t f = next64() >> (64 - bits);
    if (f < 2) f = 2;
    const uint64_t z = next64() % f;
    const uint32_t v = (uint32_t)(next64() >> 33);
    if (check(z, f, v)) return 1;
    ++n;
  }
  // the 32-bit path: f < 2^32, large v, z near f
  for (int i = 0; i < 1000000; ++i) {
    const int bits = 1 + (int)(next64() % 32);
    uint64_t f = next64() >> (64 - bits);
    if (f < 2) f = 2;
    const uint64_t z = (i & 1) ? f - 1 - next64() % (f < 64 ? f : 64) : next64() % f;
    const uint32_t v = (i & 2) ? 2147483647u - (uint32_t)(next64() % 1024) : (uint32_t)(next64() >> 33);
    if (check(z, f, v)) return 1;
    ++n;
  }
  printf("ok %ld\n", n);
  return 0;
}
