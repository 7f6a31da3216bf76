// C ABI of the structure predictor: argument checks on the host, then the
// launches of each entry point on the caller's stream.  No allocation, no
// synchronisation.
#include <atomic>
#include <cstdio>
#include <mutex>

#include "common.cuh"
#include "k_dedup.cuh"
#include "k_flop.cuh"
#include "k_scan.cuh"

using namespace spg;

namespace {

constexpr long long kIdxMax = 2147483647ll;
constexpr int kDegThreads = 256;

// Per-device launch limits, computed once per device.
struct DeviceLimits {
  int sms = 0;
  int flop_blocks_per_sm = 0;
  int scan_blocks_per_sm = 0;
  int dedup_blocks_per_sm = 0;
  int heavy_dyn_smem = 0;
  int heavy_bitmap_words = 0;
  bool ok = false;
};

// Events of the profiling hook (spgemm_set_profile_events).
std::atomic<cudaEvent_t> g_prof_before{nullptr};
std::atomic<cudaEvent_t> g_prof_after{nullptr};

void prof_mark(bool after, cudaStream_t st) {
  cudaEvent_t e = after ? g_prof_after.load() : g_prof_before.load();
  if (e) cudaEventRecord(e, st);
}

constexpr int kMaxDevices = 64;
DeviceLimits g_limits[kMaxDevices];
std::once_flag g_once[kMaxDevices];

size_t dedup_dyn_smem() { return (size_t)kDedupWarps * kWarpTable * sizeof(int); }

void init_limits(int dev, DeviceLimits* L) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return;
  L->sms = p.multiProcessorCount;
  // heavy pass: as much shared memory as the block can take for the bitmap
  const int static_smem = (int)sizeof(HeavySmem);
  int dyn = (int)p.sharedMemPerBlockOptin - static_smem - 1024;
  dyn = (dyn / 4096) * 4096;
  if (dyn < kBlockHashSlots * 4) return;
  L->heavy_dyn_smem = dyn;
  L->heavy_bitmap_words = dyn / 4;
  if (cudaFuncSetAttribute(k_dedup_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess) return;
  if (cudaFuncSetAttribute(k_dedup_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dedup_dyn_smem()) != cudaSuccess) return;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_flop_pred<kModePredict>, kFlopThreads, 0) != cudaSuccess) return;
  int b2 = 0, b3 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_flop_pred<kModeReference>, kFlopThreads, 0);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, k_flop_pred<kModeFlop>, kFlopThreads, 0);
  L->flop_blocks_per_sm = min(b, min(b2, b3));
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_scan_rows<ScanNnz, true>, kScanThreads, 0) != cudaSuccess) return;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_scan_rows<ScanSample, false>, kScanThreads, 0);
  L->scan_blocks_per_sm = min(b, b2);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_dedup_rows, kDedupThreads, dedup_dyn_smem()) != cudaSuccess) return;
  L->dedup_blocks_per_sm = b;
  L->ok = L->flop_blocks_per_sm > 0 && L->scan_blocks_per_sm > 0 && L->dedup_blocks_per_sm > 0;
}

const DeviceLimits* limits() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::call_once(g_once[dev], init_limits, dev, &g_limits[dev]);
  return g_limits[dev].ok ? &g_limits[dev] : nullptr;
}

bool csr_ok(const spgemm_csr_t* m) {
  if (!m || m->rows < 0 || m->cols < 0 || m->nnz < 0) return false;
  if (!m->rpt) return false;
  if (m->nnz > 0 && !m->col) return false;
  return true;
}

bool csr_fits(const spgemm_csr_t* m) {
  return m->rows < kIdxMax && m->cols < kIdxMax && m->nnz <= kIdxMax && m->rows + m->nnz < (1ll << 32);
}

int check_pair(const spgemm_csr_t* A, const spgemm_csr_t* B, void* ws, size_t ws_bytes,
               spgemm_result_t* res) {
  if (!csr_ok(A) || !csr_ok(B) || !res || !ws) return SPGEMM_ERR_INVALID_ARG;
  if (A->cols != B->rows) return SPGEMM_ERR_DIM_MISMATCH;
  if (!csr_fits(A) || !csr_fits(B)) return SPGEMM_ERR_TOO_LARGE;
  if (ws_bytes < ws_bytes_for(A->rows, A->cols)) return SPGEMM_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return SPGEMM_ERR_WORKSPACE;
  return SPGEMM_OK;
}

// Candidates of the sample: rows (Bernoulli) or draws (the paper's rule).
int sample_candidates(const spgemm_config_t* cfg, long long M, long long* n_cand) {
  if (!cfg || cfg->reserved0 != 0) return SPGEMM_ERR_INVALID_ARG;
  if (cfg->mode == SPGEMM_SAMPLE_BERNOULLI) {
    if (cfg->threshold > (1ull << 32)) return SPGEMM_ERR_INVALID_ARG;
    *n_cand = M;
    return SPGEMM_OK;
  }
  if (cfg->mode == SPGEMM_SAMPLE_PAPER_DRAW) {
    long long s = cfg->sample_num;
    if (s < 0 || s > M) return SPGEMM_ERR_INVALID_ARG;
    if (s == 0 && M > 0) {
      s = (3 * M) / 1000;  // min(0.003 M, 300), floored, at least one draw
      if (s > 300) s = 300;
      if (s < 1) s = 1;
    }
    *n_cand = s;
    return SPGEMM_OK;
  }
  return SPGEMM_ERR_INVALID_ARG;
}

DedupArgs dedup_args(const spgemm_csr_t* A, const spgemm_csr_t* B, const Workspace& w) {
  DedupArgs d;
  d.M = A->rows;
  d.K = A->cols;
  d.N = B->cols;
  d.nnzA = A->nnz;
  d.nnzB = B->nnz;
  d.a_rpt = A->rpt;
  d.a_col = A->col;
  d.b_rpt = B->rpt;
  d.b_col = B->col;
  d.src = kSrcAllRows;
  d.seed = 0;
  d.threshold = 0;
  d.n_cand = A->rows;
  d.nnz_out = nullptr;
  d.ws = w;
  d.heavy_cap = A->rows;
  d.heavy_case = nullptr;
  d.case_id = 0;
  return d;
}

int grid_for(long long work, long long per_block, long long cap) {
  long long g = (work + per_block - 1) / per_block;
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  if (g > kMaxSlots) g = kMaxSlots;
  return (int)g;
}

// Queues the two deduplication passes over the candidates in `d`.
int launch_dedup(const DeviceLimits* L, const DedupArgs& d, cudaStream_t st) {
  if (d.n_cand <= 0) return SPGEMM_OK;
  const int g1 = grid_for(d.n_cand, kDedupThreads, (long long)L->sms * L->dedup_blocks_per_sm);
  if (d.src == kSrcAllRows) prof_mark(false, st);
  k_dedup_rows<<<g1, kDedupThreads, dedup_dyn_smem(), st>>>(d);
  if (d.src == kSrcAllRows) prof_mark(true, st);
  k_dedup_heavy<<<L->sms, kHeavyThreads, L->heavy_dyn_smem, st>>>(d, L->heavy_bitmap_words);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

// flop_row may be null in predict mode (the per-row FLOP is then not stored);
// the other modes keep it in the workspace when the caller gives no buffer.
FlopArgs flop_args(const spgemm_csr_t* A, const spgemm_csr_t* B, const Workspace& w, int* flop,
                   int* pred, int64_t* offsets, spgemm_result_t* res, bool flop_optional) {
  FlopArgs f;
  f.M = A->rows;
  f.K = A->cols;
  f.nnzA = A->nnz;
  f.nnzB = B->nnz;
  f.a_rpt = A->rpt;
  f.a_col = A->col;
  f.b_rpt = B->rpt;
  f.deg8 = w.deg8;
  f.flop = flop ? flop : (flop_optional ? nullptr : w.flop_buf);
  f.vec_ok = ((reinterpret_cast<uintptr_t>(A->col) | reinterpret_cast<uintptr_t>(B->rpt)) & 15) == 0;
  f.pred = pred;
  f.offsets = reinterpret_cast<long long*>(offsets);
  f.ws = w;
  f.res = res;
  return f;
}

template <int MODE>
int launch_flop(const DeviceLimits* L, const FlopArgs& f, cudaStream_t st) {
  if (f.K > 0) {
    const int gd = grid_for((f.K + 3) / 4, kDegThreads, (long long)L->sms * 8);
    k_degree_table<<<gd, kDegThreads, 0, st>>>(f.b_rpt, f.K, f.nnzB, f.ws.deg8, f.ws.hdr);
  }
  const long long D = f.M + f.nnzA;
  const int g = grid_for(D, 4096, (long long)L->sms * L->flop_blocks_per_sm);
  prof_mark(false, st);
  k_flop_pred<MODE><<<g, kFlopThreads, 0, st>>>(f);
  prof_mark(true, st);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

template <class Src, bool SYM>
int launch_scan(const DeviceLimits* L, const Src& src, long long n, const Workspace& w,
                spgemm_result_t* res, cudaStream_t st) {
  const int g = grid_for(n, (long long)kScanThreads * kScanRows * 2, (long long)L->sms * L->scan_blocks_per_sm);
  k_scan_rows<Src, SYM><<<g, kScanThreads, 0, st>>>(src, n, w, res);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

int predict_common(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_config_t* cfg,
                   int32_t* pred_row, int64_t* offsets, int32_t* flop_row, spgemm_result_t* res,
                   void* ws, size_t ws_bytes, void* stream, bool reference) {
  int rc = check_pair(A, B, ws, ws_bytes, res);
  if (rc) return rc;
  if (!offsets || (!pred_row && A->rows > 0)) return SPGEMM_ERR_INVALID_ARG;
  long long n_cand = 0;
  if ((rc = sample_candidates(cfg, A->rows, &n_cand))) return rc;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = ws_carve(ws, A->rows);
  DedupArgs d = dedup_args(A, B, w);
  d.src = cfg->mode == SPGEMM_SAMPLE_BERNOULLI ? kSrcBernoulli : kSrcDraws;
  d.seed = cfg->seed;
  d.threshold = cfg->threshold;
  d.n_cand = n_cand;
  if ((rc = launch_dedup(L, d, st))) return rc;
  FlopArgs f = flop_args(A, B, w, flop_row, pred_row, offsets, res, !reference);
  return reference ? launch_flop<kModeReference>(L, f, st) : launch_flop<kModePredict>(L, f, st);
}

// ---- scratch for spgemm_predict_structure_static --------------------------------
// The workspace of a problem with SPGEMM_STATIC_MAX_ROWS rows and columns in A, as one file-scope
// device array.  In host code the name is only a stand-in for the device
// object: its device address comes from cudaGetSymbolAddress, looked up once per
// device below and passed to the kernels.
constexpr size_t kStaticHeaderBytes = sizeof(WsHeader) + sizeof(Slot) * kMaxSlots;
constexpr size_t kStaticRowBytes = ((size_t)SPGEMM_STATIC_MAX_ROWS * 4 + 255) / 256 * 256;
constexpr size_t kStaticDegBytes = ((size_t)SPGEMM_STATIC_MAX_ROWS + 16 + 255) / 256 * 256;
constexpr size_t kStaticBytes = kStaticHeaderBytes + 2 * kStaticRowBytes + kStaticDegBytes;
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

void* g_static_ptr[kMaxDevices];
cudaError_t g_static_err[kMaxDevices];
std::once_flag g_static_once[kMaxDevices];

void init_static_scratch(int dev) {
  void* p = nullptr;
  g_static_err[dev] = cudaGetSymbolAddress(&p, g_static_scratch);
  g_static_ptr[dev] = g_static_err[dev] == cudaSuccess ? p : nullptr;
}

}  // namespace

extern "C" {

size_t spgemm_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B) {
  (void)B;
  if (!A || A->rows < 0) return 0;
  return ws_bytes_for(A->rows, A->cols);
}

int spgemm_flop_per_row(const spgemm_csr_t* A, const spgemm_csr_t* B, int32_t* flop_row,
                        spgemm_result_t* res, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_pair(A, B, ws, ws_bytes, res);
  if (rc) return rc;
  if (!flop_row && A->rows > 0) return SPGEMM_ERR_INVALID_ARG;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  Workspace w = ws_carve(ws, A->rows);
  FlopArgs f = flop_args(A, B, w, flop_row, nullptr, nullptr, res, false);
  return launch_flop<kModeFlop>(L, f, static_cast<cudaStream_t>(stream));
}

int spgemm_predict_cr(const spgemm_csr_t* A, const spgemm_csr_t* B, const spgemm_config_t* cfg,
                      spgemm_result_t* res, void* ws, size_t ws_bytes, void* stream) {
  int rc = check_pair(A, B, ws, ws_bytes, res);
  if (rc) return rc;
  long long n_cand = 0;
  if ((rc = sample_candidates(cfg, A->rows, &n_cand))) return rc;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = ws_carve(ws, A->rows);
  DedupArgs d = dedup_args(A, B, w);
  d.src = cfg->mode == SPGEMM_SAMPLE_BERNOULLI ? kSrcBernoulli : kSrcDraws;
  d.seed = cfg->seed;
  d.threshold = cfg->threshold;
  d.n_cand = n_cand;
  if ((rc = launch_dedup(L, d, st))) return rc;
  k_finalize_cr<<<1, 1, 0, st>>>(w, res);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

int spgemm_predict_structure(const spgemm_csr_t* A, const spgemm_csr_t* B,
                             const spgemm_config_t* cfg, int32_t* pred_row, int64_t* offsets,
                             int32_t* flop_row, spgemm_result_t* res, void* ws, size_t ws_bytes,
                             void* stream) {
  return predict_common(A, B, cfg, pred_row, offsets, flop_row, res, ws, ws_bytes, stream, false);
}

int spgemm_predict_reference(const spgemm_csr_t* A, const spgemm_csr_t* B,
                             const spgemm_config_t* cfg, int32_t* pred_row, int64_t* offsets,
                             int32_t* flop_row, spgemm_result_t* res, void* ws, size_t ws_bytes,
                             void* stream) {
  return predict_common(A, B, cfg, pred_row, offsets, flop_row, res, ws, ws_bytes, stream, true);
}

int spgemm_symbolic_exact(const spgemm_csr_t* A, const spgemm_csr_t* B, int32_t* nnz_row,
                          int64_t* offsets, spgemm_result_t* res, void* ws, size_t ws_bytes,
                          void* stream) {
  int rc = check_pair(A, B, ws, ws_bytes, res);
  if (rc) return rc;
  if (!offsets || (!nnz_row && A->rows > 0)) return SPGEMM_ERR_INVALID_ARG;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = ws_carve(ws, A->rows);
  DedupArgs d = dedup_args(A, B, w);
  d.nnz_out = nnz_row;
  if ((rc = launch_dedup(L, d, st))) return rc;
  ScanNnz src{nnz_row, reinterpret_cast<long long*>(offsets)};
  return launch_scan<ScanNnz, true>(L, src, A->rows, w, res, st);
}

int spgemm_sample_rows(int64_t rows, const spgemm_config_t* cfg, int32_t* ids, int64_t capacity,
                       spgemm_result_t* res, void* ws, size_t ws_bytes, void* stream) {
  if (rows < 0 || rows >= kIdxMax || !res || !ws || capacity < 0 || (capacity > 0 && !ids))
    return SPGEMM_ERR_INVALID_ARG;
  if (ws_bytes < ws_bytes_for(rows, 0) || (reinterpret_cast<uintptr_t>(ws) & 255)) return SPGEMM_ERR_WORKSPACE;
  long long n_cand = 0;
  int rc = sample_candidates(cfg, rows, &n_cand);
  if (rc) return rc;
  if (cfg->mode == SPGEMM_SAMPLE_PAPER_DRAW && n_cand > capacity) return SPGEMM_ERR_INVALID_ARG;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  Workspace w = ws_carve(ws, rows);
  ScanSample src{cfg->mode, cfg->seed, cfg->threshold, rows, ids, capacity};
  return launch_scan<ScanSample, false>(L, src, n_cand, w, res, static_cast<cudaStream_t>(stream));
}

int spgemm_validate_csr(const spgemm_csr_t* A, spgemm_result_t* res, void* ws, size_t ws_bytes,
                        void* stream) {
  if (!csr_ok(A) || !res || !ws) return SPGEMM_ERR_INVALID_ARG;
  if (!csr_fits(A)) return SPGEMM_ERR_TOO_LARGE;
  if (ws_bytes < ws_bytes_for(A->rows, 0) || (reinterpret_cast<uintptr_t>(ws) & 255)) return SPGEMM_ERR_WORKSPACE;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  Workspace w = ws_carve(ws, A->rows);
  const int g = grid_for(A->rows, kValThreads / 32, (long long)L->sms * 8);
  k_validate<<<g, kValThreads, 0, static_cast<cudaStream_t>(stream)>>>(A->rows, A->cols, A->nnz, A->rpt, A->col, w, res);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

int spgemm_predict_structure_static(const spgemm_csr_t* A, const spgemm_csr_t* B,
                                    const spgemm_config_t* cfg, int32_t* pred_row,
                                    int64_t* offsets, int32_t* flop_row, spgemm_result_t* res,
                                    void* stream) {
  if (!csr_ok(A)) return SPGEMM_ERR_INVALID_ARG;
  if (A->rows > SPGEMM_STATIC_MAX_ROWS || A->cols > SPGEMM_STATIC_MAX_ROWS) return SPGEMM_ERR_STATIC_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SPGEMM_ERR_CUDA;
  std::call_once(g_static_once[dev], init_static_scratch, dev);
  void* ws = g_static_ptr[dev];
  if (!ws) return SPGEMM_ERR_CUDA;
  if (ws_bytes_for(A->rows, A->cols) > kStaticBytes) return SPGEMM_ERR_STATIC_CAPACITY;
  // Header, per-block slots and flag epoch start from zero on every call.
  if (cudaMemsetAsync(ws, 0, kStaticHeaderBytes, static_cast<cudaStream_t>(stream)) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  return predict_common(A, B, cfg, pred_row, offsets, flop_row, res, ws, kStaticBytes, stream, false);
}

int spgemm_set_profile_events(void* before, void* after) {
  g_prof_before.store(static_cast<cudaEvent_t>(before));
  g_prof_after.store(static_cast<cudaEvent_t>(after));
  return SPGEMM_OK;
}

const char* spgemm_status_string(int code) {
  switch (code) {
    case SPGEMM_OK: return "ok";
    case SPGEMM_ERR_INVALID_ARG: return "invalid argument";
    case SPGEMM_ERR_DIM_MISMATCH: return "A.cols != B.rows";
    case SPGEMM_ERR_WORKSPACE: return "workspace too small or not 256-byte aligned";
    case SPGEMM_ERR_CUDA: return "CUDA launch or query failed";
    case SPGEMM_ERR_TOO_LARGE: return "size exceeds the int32 index range";
    case SPGEMM_ERR_STATIC_CAPACITY:
      return "A.rows or A.cols exceeds the static scratch of spgemm_predict_structure_static (SPGEMM_STATIC_MAX_ROWS)";
    case SPGEMM_STATUS_WARN_EMPTY_SAMPLE: return "warning: empty sample, prediction fell back to FLOP";
    case SPGEMM_STATUS_WARN_SATURATED: return "warning: a prediction saturated at 2^31-1";
    case SPGEMM_STATUS_WARN_UNSORTED: return "warning: a row is not strictly increasing";
    case SPGEMM_STATUS_ERR_BAD_INPUT: return "error: an offset or column id is out of range";
    case SPGEMM_STATUS_ERR_TIMEOUT: return "error: an inter-block wait timed out";
    default: break;
  }
  if (code > 0 && (code & (SPGEMM_STATUS_ERR_BAD_INPUT | SPGEMM_STATUS_ERR_TIMEOUT)))
    return "error: several status bits set";
  if (code > 0) return "warning: several status bits set";
  return "unknown code";
}

}  // extern "C"
