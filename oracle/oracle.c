/*
 * CPU oracle for the sampled-compression-ratio predictor of the output structure
 * of a sparse matrix product C = A*B (Du et al., arXiv 2207.13848).
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load or call this code.  It
 * includes nothing from the GPU library and the GPU library includes nothing from
 * it; the only thing the two sides share is the seeded synthetic inputs.
 *
 * The code is deliberately plain: one loop per definition, exact integer
 * arithmetic (64-bit sums, unsigned 128-bit products and quotients), no blocking,
 * no fusion.  Each routine names the passage of the paper it follows.  OpenMP,
 * when compiled in, only splits the outer row loop into static chunks, as the
 * paper's own implementation does (Sec. V-A, V-B); results do not depend on it.
 *
 * Notation (Table I, Sec. II-A): A is M x K, B is K x N, C = A*B is M x N.
 * CSR arrays (Sec. II-B): rpt (row offsets, M+1 entries) and col (column ids).
 * Values are never read: the method counts structural products and structural
 * nonzeros only.
 *
 * Readings of the paper fixed here (each marked "reading" below):
 *  - sample_num = min(0.003 M, 300) is floored, i.e. floor(3M/1000), and at least 1.
 *  - the random row of a draw is (h * M) >> 32 for a 32-bit uniform h, so it lies in [0, M).
 *  - the per-row prediction flop_i / CR is rounded up: ceil(flop_i * z / f).
 *  - an empty sample (f* = 0) leaves CR undefined; the prediction falls back to
 *    flop_i (the upper-bound method) and the status carries ORC_WARN_EMPTY_SAMPLE.
 *  - the reference design's per-row prediction is saturated at 2^31 - 1, with
 *    ORC_WARN_SATURATED in the status.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_WARN_EMPTY_SAMPLE 1
#define ORC_WARN_SATURATED 2

typedef unsigned __int128 u128;

/* ---------------------------------------------------------------------------
 * Counter-based random numbers for the row sample.
 *
 * SplitMix64 (G. L. Steele, D. Lea, C. H. Flood, "Fast splittable pseudorandom
 * number generators", OOPSLA 2014): the state advances by the odd constant
 * gamma = 0x9e3779b97f4a7c15 and every state is passed through the 64-bit
 * finaliser with shifts 30, 27, 31 and multipliers 0xbf58476d1ce4e5b9 and
 * 0x94d049bb133111eb.  orc_splitmix64(seed, k) is the k-th output (k >= 1) of
 * the generator whose initial state is `seed`.
 * ------------------------------------------------------------------------- */
uint64_t orc_splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + k * 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

/* h32(seed, x): the high 32 bits of output x+1 of SplitMix64 seeded with `seed`. */
uint32_t orc_h32(uint64_t seed, uint64_t x) {
  return (uint32_t)(orc_splitmix64(seed, x + 1) >> 32);
}

/* ---------------------------------------------------------------------------
 * Algorithm 1 (Sec. V-A): FLOP of every output row and the total FLOP(C).
 * flop_i = sum over j in A's row i of (B.rpt[A.col[j]+1] - B.rpt[A.col[j]]).
 * Returns total_flop.
 * ------------------------------------------------------------------------- */
int64_t orc_flop_per_row(int64_t M, const int32_t* a_rpt, const int32_t* a_col,
                         const int32_t* b_rpt, int64_t* flop_out) {
  int64_t total_flop = 0;
  int64_t i;
#pragma omp parallel for schedule(static) reduction(+ : total_flop)
  for (i = 0; i < M; ++i) {
    int64_t local_flop = 0;
    for (int64_t j = a_rpt[i]; j < a_rpt[i + 1]; ++j) {
      int32_t k = a_col[j];
      local_flop += (int64_t)b_rpt[k + 1] - (int64_t)b_rpt[k];
    }
    flop_out[i] = local_flop;
    total_flop += local_flop;
  }
  return total_flop;
}

/* ---------------------------------------------------------------------------
 * Exact nnz of output rows (the "precise method", Sec. I; the per-row count of
 * Algorithm 2's hash loop, Sec. V-B).  nnz_i is the number of distinct column
 * ids among all products of row i: |union over k in A_i of cols(B_k)|.
 *
 * The paper counts them with an open-addressing hash table; the count does not
 * depend on how duplicates are detected, so this routine uses the textbook dense
 * marker: mark[c] holds the stamp of the last row that produced column c.
 * Stamps are unique per row visit, so no clearing is needed between rows.
 *
 * rows == NULL means every row 0..nrows-1; otherwise rows[0..nrows) lists the
 * rows to count (repeats allowed).  Returns the sum of the counts.
 * ------------------------------------------------------------------------- */
int64_t orc_row_nnz(int64_t N, const int32_t* a_rpt, const int32_t* a_col,
                    const int32_t* b_rpt, const int32_t* b_col,
                    const int32_t* rows, int64_t nrows, int64_t* nnz_out) {
  int64_t total = 0;
  int failed = 0;
#pragma omp parallel reduction(+ : total) reduction(| : failed)
  {
    int64_t* mark = (int64_t*)malloc((size_t)(N > 0 ? N : 1) * sizeof(int64_t));
    if (!mark) {
      failed = 1;
    } else {
      for (int64_t c = 0; c < N; ++c) mark[c] = -1;
      int64_t r;
#pragma omp for schedule(static)
      for (r = 0; r < nrows; ++r) {
        int64_t i = rows ? rows[r] : r;
        int64_t stamp = r; /* unique for this visit */
        int64_t local_nnz = 0;
        for (int64_t j = a_rpt[i]; j < a_rpt[i + 1]; ++j) {
          int32_t k = a_col[j];
          for (int64_t t = b_rpt[k]; t < b_rpt[k + 1]; ++t) {
            int32_t c = b_col[t];
            if (mark[c] != stamp) {
              mark[c] = stamp;
              local_nnz += 1;
            }
          }
        }
        nnz_out[r] = local_nnz;
        total += local_nnz;
      }
      free(mark);
    }
  }
  return failed ? -1 : total;
}

/* ---------------------------------------------------------------------------
 * Row sampling (Sec. IV-A: a fraction p of A's rows; B is used whole).
 *
 * Bernoulli mode (the workloads' "ratio of rows chosen by a counter hash of
 * (seed, row)"): row i is sampled iff h32(seed, i) < threshold, with threshold
 * in [0, 2^32]; 2^32 samples every row.  Writes the sampled rows in ascending
 * order and returns |S|.
 * ------------------------------------------------------------------------- */
int64_t orc_sample_bernoulli(int64_t M, uint64_t seed, uint64_t threshold, int32_t* ids_out) {
  int64_t n = 0;
  for (int64_t i = 0; i < M; ++i)
    if ((uint64_t)orc_h32(seed, (uint64_t)i) < threshold) ids_out[n++] = (int32_t)i;
  return n;
}

/* sample_num = min(0.003 M, 300) of Algorithm 2 (Sec. V-B).  Reading: floored
 * (the paper prints 140 samples for M = 46835), and at least 1 when M > 0. */
int64_t orc_paper_sample_num(int64_t M) {
  if (M <= 0) return 0;
  int64_t s = (3 * M) / 1000;
  if (s > 300) s = 300;
  if (s < 1) s = 1;
  return s;
}

/* Algorithm 2's draws (Sec. V-B): draw r picks row rid = M * rand[r].  Reading:
 * rand[r] is the 32-bit uniform h32(seed, r) / 2^32, so rid = (h32 * M) >> 32,
 * which is always in [0, M).  Draws are with replacement; a row drawn twice is
 * counted twice.  Writes sample_num row ids in draw order. */
int64_t orc_sample_paper_draw(int64_t M, uint64_t seed, int64_t sample_num, int32_t* ids_out) {
  for (int64_t r = 0; r < sample_num; ++r)
    ids_out[r] = (int32_t)(((uint64_t)orc_h32(seed, (uint64_t)r) * (uint64_t)M) >> 32);
  return sample_num;
}

/* ceil(a / b) for b > 0, exact. */
static u128 ceil_div_u128(u128 a, u128 b) { return (a + b - 1) / b; }

/* ---------------------------------------------------------------------------
 * The proposed method (Sec. IV-D, Eq. 4; Algorithm 2, Sec. V-B).
 *   f* = sum over sampled rows of flop_i     (sample_flop)
 *   z* = sum over sampled rows of nnz_i      (sample_nnz)
 *   r* = f* / z*                              (sampled compression ratio)
 *   pred_i = flop_i / r*, rounded up = ceil(flop_i * z* / f*)
 *   offsets = exclusive scan of pred (M+1 entries), Z2* = F * z* / f*.
 * Inputs: the sample `ids` (|S| = n_ids entries, repeats allowed).
 * Outputs: flop[M], pred[M], offsets[M+1]; scalars[0..5] =
 *   {F, f*, z*, |S|, pred_total, status}.
 * Returns 0, or -1 if a work buffer could not be allocated.
 * ------------------------------------------------------------------------- */
int orc_predict(int64_t M, int64_t N, const int32_t* a_rpt, const int32_t* a_col,
                const int32_t* b_rpt, const int32_t* b_col, const int32_t* ids, int64_t n_ids,
                int64_t* flop, int64_t* pred, int64_t* offsets, int64_t* scalars) {
  int64_t F = orc_flop_per_row(M, a_rpt, a_col, b_rpt, flop);
  int64_t* nnz_s = (int64_t*)malloc((size_t)(n_ids > 0 ? n_ids : 1) * sizeof(int64_t));
  if (!nnz_s) return -1;
  int64_t z = orc_row_nnz(N, a_rpt, a_col, b_rpt, b_col, ids, n_ids, nnz_s);
  free(nnz_s);
  if (z < 0) return -1;
  int64_t f = 0;
  for (int64_t r = 0; r < n_ids; ++r) f += flop[ids[r]];
  int64_t status = 0;
  if (f == 0) status |= ORC_WARN_EMPTY_SAMPLE;
  offsets[0] = 0;
  for (int64_t i = 0; i < M; ++i) {
    int64_t p;
    if (f == 0)
      p = flop[i];
    else
      p = (int64_t)ceil_div_u128((u128)(uint64_t)flop[i] * (u128)(uint64_t)z, (u128)(uint64_t)f);
    pred[i] = p;
    offsets[i + 1] = offsets[i] + p;
  }
  scalars[0] = F;
  scalars[1] = f;
  scalars[2] = z;
  scalars[3] = n_ids;
  scalars[4] = offsets[M];
  scalars[5] = status;
  return 0;
}

/* ---------------------------------------------------------------------------
 * The reference design (Sec. IV-C, Eq. 2): Z1* = z* / p with p = |S| / M,
 * predicted CR1 = F / Z1*, pred1_i = flop_i / CR1 rounded up
 *   = ceil(flop_i * z* * M / (F * |S|)),
 * saturated at 2^31 - 1.  Same outputs as orc_predict.
 * ------------------------------------------------------------------------- */
int orc_predict_reference(int64_t M, int64_t N, const int32_t* a_rpt, const int32_t* a_col,
                          const int32_t* b_rpt, const int32_t* b_col, const int32_t* ids,
                          int64_t n_ids, int64_t* flop, int64_t* pred, int64_t* offsets,
                          int64_t* scalars) {
  int64_t F = orc_flop_per_row(M, a_rpt, a_col, b_rpt, flop);
  int64_t* nnz_s = (int64_t*)malloc((size_t)(n_ids > 0 ? n_ids : 1) * sizeof(int64_t));
  if (!nnz_s) return -1;
  int64_t z = orc_row_nnz(N, a_rpt, a_col, b_rpt, b_col, ids, n_ids, nnz_s);
  free(nnz_s);
  if (z < 0) return -1;
  int64_t f = 0;
  for (int64_t r = 0; r < n_ids; ++r) f += flop[ids[r]];
  int64_t status = 0;
  if (n_ids == 0) status |= ORC_WARN_EMPTY_SAMPLE;
  offsets[0] = 0;
  for (int64_t i = 0; i < M; ++i) {
    int64_t p;
    if (n_ids == 0) {
      p = flop[i];
    } else if (flop[i] == 0) {
      p = 0; /* F == 0 implies every flop_i == 0 */
    } else {
      u128 num = (u128)(uint64_t)flop[i] * (u128)(uint64_t)z * (u128)(uint64_t)M;
      u128 den = (u128)(uint64_t)F * (u128)(uint64_t)n_ids;
      u128 q = ceil_div_u128(num, den);
      if (q > (u128)2147483647) {
        q = 2147483647;
        status |= ORC_WARN_SATURATED;
      }
      p = (int64_t)q;
    }
    pred[i] = p;
    offsets[i + 1] = offsets[i] + p;
  }
  scalars[0] = F;
  scalars[1] = f;
  scalars[2] = z;
  scalars[3] = n_ids;
  scalars[4] = offsets[M];
  scalars[5] = status;
  return 0;
}

/* ---------------------------------------------------------------------------
 * Exact output structure (the precise method / symbolic phase, Sec. I):
 * nnz_i for every row, offsets = exclusive scan, returns Z = NNZ(C).
 * ------------------------------------------------------------------------- */
int64_t orc_symbolic_exact(int64_t M, int64_t N, const int32_t* a_rpt, const int32_t* a_col,
                           const int32_t* b_rpt, const int32_t* b_col, int64_t* nnz,
                           int64_t* offsets) {
  int64_t Z = orc_row_nnz(N, a_rpt, a_col, b_rpt, b_col, NULL, M, nnz);
  if (Z < 0) return -1;
  offsets[0] = 0;
  for (int64_t i = 0; i < M; ++i) offsets[i + 1] = offsets[i] + nnz[i];
  return Z;
}

/* ---------------------------------------------------------------------------
 * Numeric product C = A*B: the numeric phase that the predicted structure
 * allocates memory for (Sec. I; the consumer of the prediction, outside the
 * paper's own experiments).  Row i of C holds every column reached by a
 * product of A's row i with the rows of B, with the value sum_k a_ik * b_kc.
 * Textbook row-wise (Gustavson) product with a dense accumulator: each product
 * is formed in double precision from the single-precision inputs (exact: 24-bit
 * by 24-bit mantissas), summed in double, and the row's columns are written in
 * ascending order.  For every entry it also writes the sum of |a_ik * b_kc| and
 * the number of products, which bound the rounding of a single-precision sum.
 * c_rpt holds the exact offsets (orc_symbolic_exact).  Returns the number of
 * entries written, or -1 when the accumulator could not be allocated.
 * ------------------------------------------------------------------------- */
static int orc_cmp_i32(const void* x, const void* y) {
  const int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
  return (a > b) - (a < b);
}

int64_t orc_spgemm_numeric(int64_t M, int64_t N, const int32_t* a_rpt, const int32_t* a_col,
                           const float* a_val, const int32_t* b_rpt, const int32_t* b_col,
                           const float* b_val, const int64_t* c_rpt, int32_t* c_col, double* c_val,
                           double* c_abs, int32_t* c_terms) {
  int64_t total = 0;
  int failed = 0;
#pragma omp parallel reduction(+ : total) reduction(| : failed)
  {
    const size_t n_alloc = (size_t)(N > 0 ? N : 1);
    double* acc = (double*)malloc(n_alloc * sizeof(double));
    double* acc_abs = (double*)malloc(n_alloc * sizeof(double));
    int32_t* terms = (int32_t*)malloc(n_alloc * sizeof(int32_t));
    int64_t* mark = (int64_t*)malloc(n_alloc * sizeof(int64_t));
    int32_t* list = (int32_t*)malloc(n_alloc * sizeof(int32_t));
    if (!acc || !acc_abs || !terms || !mark || !list) {
      failed = 1;
    } else {
      for (int64_t c = 0; c < N; ++c) mark[c] = -1;
      int64_t i;
#pragma omp for schedule(static)
      for (i = 0; i < M; ++i) {
        int64_t n = 0;
        for (int64_t j = a_rpt[i]; j < a_rpt[i + 1]; ++j) {
          const int32_t k = a_col[j];
          const double a = (double)a_val[j];
          for (int64_t t = b_rpt[k]; t < b_rpt[k + 1]; ++t) {
            const int32_t c = b_col[t];
            const double prod = a * (double)b_val[t];
            if (mark[c] != i) {
              mark[c] = i;
              acc[c] = 0.0;
              acc_abs[c] = 0.0;
              terms[c] = 0;
              list[n++] = c;
            }
            acc[c] += prod;
            acc_abs[c] += prod < 0.0 ? -prod : prod;
            terms[c] += 1;
          }
        }
        qsort(list, (size_t)n, sizeof(int32_t), orc_cmp_i32);
        const int64_t o = c_rpt[i];
        for (int64_t q = 0; q < n; ++q) {
          const int32_t c = list[q];
          c_col[o + q] = c;
          c_val[o + q] = acc[c];
          c_abs[o + q] = acc_abs[c];
          c_terms[o + q] = terms[c];
        }
        total += n;
      }
    }
    free(acc);
    free(acc_abs);
    free(terms);
    free(mark);
    free(list);
  }
  return failed ? -1 : total;
}

/* Number of OpenMP threads a parallel region uses (1 without OpenMP). */
int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
