// C ABI of the structure predictor: argument checks on the host, then the
// launches of each entry point on the caller's stream.  No allocation, no
// synchronisation.
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "k_batch.cuh"
#include "k_numeric.cuh"
#include "k_dedup.cuh"
#include "k_flop.cuh"
#include "k_predict.cuh"
#include "k_probe.cuh"
#include "k_scan.cuh"

using namespace spg;

static_assert(sizeof(spgemm_csr_t) == 40, "spgemm_csr_t layout");
static_assert(sizeof(spgemm_config_t) == 32, "spgemm_config_t layout");
static_assert(sizeof(spgemm_result_t) == 48, "spgemm_result_t layout");
static_assert(sizeof(spgemm_batch_item_t) == 144, "spgemm_batch_item_t layout");
static_assert(sizeof(spgemm_batch_tuning_t) == 32, "spgemm_batch_tuning_t layout");
static_assert(sizeof(spgemm_batch_plan_t) == 88, "spgemm_batch_plan_t layout");

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
  // batched prediction
  int kb_sample_blocks_per_sm[3] = {0, 0, 0};  // warp tables of 512, 1024, 2048 slots
  int kb_flop_blocks_per_sm = 0;
  int kb_heavy_dyn_smem = 0;
  int kb_heavy_bitmap_words = 0;
  int kb_all_blocks_per_sm = 0;
  // single-launch predictor
  int pred_blocks_per_sm = 0;
  int pred_dyn_smem = 0;
  // numeric product (the consumer)
  int num_blocks_per_sm = 0;
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
  // batched prediction
  cudaFuncAttributes fa;
  if (cudaFuncGetAttributes(&fa, kb_heavy) != cudaSuccess) return;
  int kdyn = (int)p.sharedMemPerBlockOptin - (int)fa.sharedSizeBytes - 1024;
  kdyn = (kdyn / 4096) * 4096;
  if (kdyn < kBlockHashSlots * 4) return;
  if (cudaFuncSetAttribute(kb_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, kdyn) != cudaSuccess) return;
  L->kb_heavy_dyn_smem = kdyn;
  L->kb_heavy_bitmap_words = kdyn / 4;
  const void* samplers[3] = {(const void*)kb_sample<512>, (const void*)kb_sample<1024>, (const void*)kb_sample<2048>};
  for (int i = 0; i < 3; ++i) {
    const int sm = kDedupWarps * (512 << i) * (int)sizeof(int);
    if (cudaFuncSetAttribute(samplers[i], cudaFuncAttributeMaxDynamicSharedMemorySize, sm) != cudaSuccess) return;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, samplers[i], kDedupThreads, sm) != cudaSuccess) return;
    L->kb_sample_blocks_per_sm[i] = b;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kb_flop, kFlopThreads, 0) != cudaSuccess) return;
  L->kb_flop_blocks_per_sm = b;
  // the batch as one persistent launch: one block per SM
  const int adyn = (int)kAllDynSmem;
  if (cudaFuncSetAttribute(kb_all<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, adyn) != cudaSuccess) return;
  if (cudaFuncSetAttribute(kb_all<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, adyn) != cudaSuccess) return;
  if (cudaFuncSetAttribute(kb_all<2048>, cudaFuncAttributeMaxDynamicSharedMemorySize, adyn) != cudaSuccess) return;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kb_all<512>, kAllThreads, adyn) != cudaSuccess) return;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, kb_all<1024>, kAllThreads, adyn) != cudaSuccess) return;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, kb_all<2048>, kAllThreads, adyn) != cudaSuccess) return;
  L->kb_all_blocks_per_sm = min(b, min(b2, b3));
  // single-launch predictor: a fixed 128 KB of dynamic shared memory (the rest
  // of the SM's 256 KB stays L1 for the FLOP pass)
  const int pdyn = (int)kPredDynSmem;
  if (cudaFuncSetAttribute(k_predict<kModePredict>, cudaFuncAttributeMaxDynamicSharedMemorySize, pdyn) != cudaSuccess) return;
  if (cudaFuncSetAttribute(k_predict<kModeReference>, cudaFuncAttributeMaxDynamicSharedMemorySize, pdyn) != cudaSuccess) return;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_predict<kModePredict>, kPredThreads, pdyn) != cudaSuccess) return;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_predict<kModeReference>, kPredThreads, pdyn) != cudaSuccess) return;
  L->pred_blocks_per_sm = min(b, b2);
  L->pred_dyn_smem = pdyn;
  // numeric product
  if (cudaFuncSetAttribute(k_numeric_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNumRowsSmem) != cudaSuccess) return;
  if (cudaFuncSetAttribute(k_numeric_heavy, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNumHeavySmem) != cudaSuccess) return;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_numeric_rows, kNumThreads, kNumRowsSmem) != cudaSuccess) return;
  L->num_blocks_per_sm = b;
  L->ok = L->pred_blocks_per_sm > 0 && L->num_blocks_per_sm > 0 && L->flop_blocks_per_sm > 0 && L->scan_blocks_per_sm > 0 && L->dedup_blocks_per_sm > 0 &&
          L->kb_flop_blocks_per_sm > 0 && L->kb_all_blocks_per_sm > 0 && L->kb_sample_blocks_per_sm[0] > 0 &&
          L->kb_sample_blocks_per_sm[1] > 0 && L->kb_sample_blocks_per_sm[2] > 0;
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
  if (ws_bytes < ws_bytes_for(A->rows, A->cols, B->cols)) return SPGEMM_ERR_WORKSPACE;
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
  d.status = &w.hdr->status;
  d.heavy_count = &w.hdr->heavy_count;
  d.heavy = w.heavy;
  d.heavy_cap = A->rows;
  d.heavy_base = 0;
  d.heavy_thr = kWarpCap;
  d.big_count = nullptr;
  d.big_thr = 0;
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

template <class Src, bool SYM, class Res = spgemm_result_t>
int launch_scan(const DeviceLimits* L, const Src& src, long long n, const Workspace& w, Res* res,
                cudaStream_t st) {
  const int g = grid_for(n, (long long)kScanThreads * kScanRows * 2, (long long)L->sms * L->scan_blocks_per_sm);
  k_scan_rows<Src, SYM, Res><<<g, kScanThreads, 0, st>>>(src, n, w, res);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

// One cooperative launch of the single-launch predictor over the operands of
// pa (all blocks co-resident).
template <int MODE>
int launch_predict(const DeviceLimits* L, const PredArgs& pa, cudaStream_t st) {
  const long long D = pa.f.M + pa.f.nnzA;
  long long g = (D + kPredItemsPerBlock - 1) / kPredItemsPerBlock;
  const long long cap = std::min<long long>((long long)L->sms * L->pred_blocks_per_sm, kMaxSlots);
  if (g < 1) g = 1;
  if (g > cap) g = cap;
  cudaLaunchConfig_t lc = {};
  lc.gridDim = dim3((unsigned)g);
  lc.blockDim = dim3(kPredThreads);
  lc.dynamicSmemBytes = (size_t)L->pred_dyn_smem;
  lc.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  lc.attrs = at;
  lc.numAttrs = 1;
  prof_mark(false, st);
  const cudaError_t e = cudaLaunchKernelEx(&lc, k_predict<MODE>, pa);
  prof_mark(true, st);
  return e == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
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
  Workspace w = ws_carve(ws, A->rows, A->cols, B->cols);
  DedupArgs d = dedup_args(A, B, w);
  d.src = cfg->mode == SPGEMM_SAMPLE_BERNOULLI ? kSrcBernoulli : kSrcDraws;
  d.seed = cfg->seed;
  d.threshold = cfg->threshold;
  d.n_cand = n_cand;
  PredArgs pa;
  pa.f = flop_args(A, B, w, flop_row, pred_row, offsets, res, false);
  pa.d = d;
  pa.bitmap_words = L->pred_dyn_smem / 4;
  pa.flop_out = flop_row != nullptr;
  return reference ? launch_predict<kModeReference>(L, pa, st) : launch_predict<kModePredict>(L, pa, st);
}

// ---- scratch for spgemm_predict_structure_static --------------------------------
// The workspace of a problem with SPGEMM_STATIC_MAX_ROWS rows and columns in A, as one file-scope
// device array.  In host code the name is only a stand-in for the device
// object: its device address comes from cudaGetSymbolAddress, looked up once per
// device below and passed to the kernels.
constexpr size_t kStaticHeaderBytes = sizeof(WsHeader) + sizeof(Slot) * kMaxSlots;
constexpr size_t kStaticBytes = ws_bytes_for(SPGEMM_STATIC_MAX_ROWS, SPGEMM_STATIC_MAX_ROWS, SPGEMM_STATIC_MAX_ROWS);
static_assert(kStaticBytes >= kStaticHeaderBytes + 2 * (size_t)SPGEMM_STATIC_MAX_ROWS * 4 + (size_t)SPGEMM_STATIC_MAX_ROWS,
              "the scratch holds the header, the row queue, the FLOP buffer and the byte table");
static __device__ __align__(256) unsigned char g_static_scratch[kStaticBytes];

void* g_static_ptr[kMaxDevices];
cudaError_t g_static_err[kMaxDevices];
std::once_flag g_static_once[kMaxDevices];

void init_static_scratch(int dev) {
  void* p = nullptr;
  g_static_err[dev] = cudaGetSymbolAddress(&p, g_static_scratch);
  g_static_ptr[dev] = g_static_err[dev] == cudaSuccess ? p : nullptr;
  if (g_static_err[dev] != cudaSuccess) cudaGetLastError();
}

// ---- batched prediction ---------------------------------------------------------
constexpr int kDefTile = 16384, kMinTile = 4096, kMaxTile = 1 << 24;
constexpr int kDefChunk = 32768, kMinChunk = 4096, kMaxChunk = 1 << 24;
constexpr int kDefTable = 1024;

size_t r256(size_t b) { return (b + 255) / 256 * 256; }
size_t r16(size_t b) { return (b + 15) / 16 * 16; }

// Regions of the batch workspace, in order.  [cases, slots) is the plan copied
// from the host; the deg8 tables follow the heavy-row queue.
struct BatchLayout {
  size_t hdr, acc, cases, tile_case, chunk_case, tab_case, slots, heavy, deg, total;
  size_t plan_bytes() const { return slots - cases; }
};

BatchLayout batch_layout(long long n, long long tiles, long long chunks, long long tab_blocks,
                         long long heavy_cap, long long deg_bytes) {
  BatchLayout l;
  size_t p = 0;
  l.hdr = p;
  p += r256(sizeof(BatchHeader));
  l.acc = p;
  p += r256(sizeof(CaseAcc) * (size_t)n);
  l.cases = p;
  p += r256(sizeof(BatchCase) * (size_t)n);
  l.tile_case = p;
  p += r256(4 * (size_t)tiles);
  l.chunk_case = p;
  p += r256(4 * (size_t)(chunks > 0 ? chunks : 1));
  l.tab_case = p;
  p += r256(4 * (size_t)(tab_blocks > 0 ? tab_blocks : 1));
  l.slots = p;
  p += sizeof(Slot) * (size_t)tiles;
  l.heavy = p;
  p += r256(4 * (size_t)(heavy_cap > 0 ? heavy_cap : 1));
  l.deg = p;
  p += r256((size_t)deg_bytes);
  l.total = p;
  return l;
}

int resolve_tuning(const spgemm_batch_tuning_t* in, const DeviceLimits* L, spgemm_batch_tuning_t* out) {
  spgemm_batch_tuning_t t{};
  if (in) t = *in;
  if (t.reserved[0] || t.reserved[1]) return SPGEMM_ERR_INVALID_ARG;
  if (t.tile_items == 0) t.tile_items = kDefTile;
  if (t.warp_table == 0) t.warp_table = kDefTable;
  if (t.heavy_threshold == 0) t.heavy_threshold = t.warp_table / 2;
  if (t.sample_chunk == 0) t.sample_chunk = kDefChunk;
  if (t.flop_blocks_per_sm == 0 && L) t.flop_blocks_per_sm = L->kb_flop_blocks_per_sm;
  if (t.launches == 0) t.launches = 4;
  if (t.launches != 1 && t.launches != 4) return SPGEMM_ERR_INVALID_ARG;
  if (t.tile_items < kMinTile || t.tile_items > kMaxTile) return SPGEMM_ERR_INVALID_ARG;
  if (t.warp_table != 512 && t.warp_table != 1024 && t.warp_table != 2048) return SPGEMM_ERR_INVALID_ARG;
  if (t.heavy_threshold < 32 || t.heavy_threshold > t.warp_table / 2) return SPGEMM_ERR_INVALID_ARG;
  if (t.sample_chunk < kMinChunk || t.sample_chunk > kMaxChunk || t.sample_chunk % 256) return SPGEMM_ERR_INVALID_ARG;
  if (t.flop_blocks_per_sm < 0 || (L && (t.flop_blocks_per_sm < 1 || t.flop_blocks_per_sm > L->kb_flop_blocks_per_sm)))
    return SPGEMM_ERR_INVALID_ARG;
  *out = t;
  return SPGEMM_OK;
}

// Host checks of one case, as spgemm_predict_structure makes them.
int check_item(const spgemm_batch_item_t& it, long long* n_cand) {
  const spgemm_csr_t* A = &it.A;
  const spgemm_csr_t* B = &it.B;
  if (!csr_ok(A) || !csr_ok(B) || !it.res) return SPGEMM_ERR_INVALID_ARG;
  if (A->cols != B->rows) return SPGEMM_ERR_DIM_MISMATCH;
  if (!csr_fits(A) || !csr_fits(B)) return SPGEMM_ERR_TOO_LARGE;
  if (!it.offsets || (!it.pred_row && A->rows > 0)) return SPGEMM_ERR_INVALID_ARG;
  return sample_candidates(&it.cfg, A->rows, n_cand);
}

long long tiles_of(const spgemm_batch_item_t& it, long long tile) {
  const long long D = it.A.rows + it.A.nnz;
  const long long t = (D + tile - 1) / tile;
  return t > 0 ? t : 1;
}
long long tab_blocks_of(const spgemm_batch_item_t& it) {
  return (it.A.cols + kTabRowsPerBlock - 1) / kTabRowsPerBlock;
}

// Totals of a batch under tile size `tile` and chunk size `chunk`; returns the
// first failing case's code (and index) or SPGEMM_OK.
struct BatchTotals {
  long long rows = 0, cand = 0, tiles = 0, chunks = 0, tab = 0, deg = 0;
};
int batch_totals(const spgemm_batch_item_t* items, int n, long long tile, long long chunk, BatchTotals* T,
                 int* bad) {
  BatchTotals t;
  for (int i = 0; i < n; ++i) {
    long long nc = 0;
    const int rc = check_item(items[i], &nc);
    if (rc) {
      *bad = i;
      return rc;
    }
    t.rows += items[i].A.rows;
    t.cand += nc;
    t.tiles += tiles_of(items[i], tile);
    t.tab += tab_blocks_of(items[i]);
    t.deg += (long long)r16((size_t)items[i].A.cols + 16);
  }
  t.chunks = (t.cand + chunk - 1) / chunk;
  if (t.rows >= kIdxMax || t.tiles >= kIdxMax || t.tab >= kIdxMax) return SPGEMM_ERR_TOO_LARGE;
  *T = t;
  return SPGEMM_OK;
}

BatchLayout layout_of(const BatchTotals& t, int n) {
  return batch_layout(n, t.tiles, t.chunks, t.tab, t.cand, t.deg);
}

BatchArgs batch_args(const spgemm_batch_plan_t* plan, void* ws) {
  const BatchLayout l = batch_layout(plan->n_cases, plan->total_tiles, plan->total_chunks,
                                     plan->total_table_blocks, plan->total_candidates, 0);
  char* base = static_cast<char*>(ws);
  BatchArgs b;
  b.hdr = reinterpret_cast<BatchHeader*>(base + l.hdr);
  b.cases = reinterpret_cast<const BatchCase*>(base + l.cases);
  b.acc = reinterpret_cast<CaseAcc*>(base + l.acc);
  b.slots = reinterpret_cast<Slot*>(base + l.slots);
  b.tile_case = reinterpret_cast<const int*>(base + l.tile_case);
  b.chunk_case = reinterpret_cast<const int*>(base + l.chunk_case);
  b.tab_case = reinterpret_cast<const int*>(base + l.tab_case);
  b.heavy = reinterpret_cast<int*>(base + l.heavy);
  b.n_cases = plan->n_cases;
  b.total_tiles = (int)plan->total_tiles;
  b.total_cand = plan->total_candidates;
  b.total_chunks = plan->total_chunks;
  b.sample_chunk = plan->tuning.sample_chunk;
  b.heavy_cap = plan->total_candidates;
  b.total_tab_blocks = plan->total_table_blocks;
  b.heavy_thr = plan->tuning.heavy_threshold;
  return b;
}

// Queues the batch: counters reset, then one cooperative launch of kb_all
// (tuning.launches = 1) or the four launches.  ev (optional, 5 events) is
// recorded before the first launch and after each phase: tables, sampled rows,
// heavy rows, FLOP (with one launch, all four after it).
int launch_batch(const DeviceLimits* L, const spgemm_batch_plan_t* plan, void* ws, cudaStream_t st,
                 cudaEvent_t* ev) {
  const BatchArgs b = batch_args(plan, ws);
  if (cudaMemsetAsync(b.hdr, 0, kBatchCounterBytes, st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  if (plan->tuning.launches == 1) {
    if (ev) cudaEventRecord(ev[0], st);
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3((unsigned)std::min<long long>((long long)L->sms * L->kb_all_blocks_per_sm, kMaxSlots));
    lc.blockDim = dim3(kAllThreads);
    lc.dynamicSmemBytes = kAllDynSmem;
    lc.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    lc.attrs = at;
    lc.numAttrs = 1;
    const int words = (int)(kAllDynSmem / sizeof(unsigned));
    prof_mark(false, st);
    const int wt = plan->tuning.warp_table;
    const cudaError_t e = wt == 512    ? cudaLaunchKernelEx(&lc, kb_all<512>, b, words)
                          : wt == 1024 ? cudaLaunchKernelEx(&lc, kb_all<1024>, b, words)
                                       : cudaLaunchKernelEx(&lc, kb_all<2048>, b, words);
    prof_mark(true, st);
    if (ev)
      for (int i = 1; i < 5; ++i) cudaEventRecord(ev[i], st);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return SPGEMM_ERR_CUDA;
    }
    return SPGEMM_OK;
  }
  if (ev) cudaEventRecord(ev[0], st);
  if (plan->total_table_blocks > 0)
    kb_tables<<<(unsigned)plan->total_table_blocks, kTabThreads, 0, st>>>(b);
  if (ev) cudaEventRecord(ev[1], st);
  if (plan->total_chunks > 0) {
    const int ti = plan->tuning.warp_table == 512 ? 0 : plan->tuning.warp_table == 1024 ? 1 : 2;
    const long long cap = (long long)L->sms * L->kb_sample_blocks_per_sm[ti];
    const int g = (int)std::min<long long>(plan->total_chunks, cap);
    const size_t sm = (size_t)kDedupWarps * plan->tuning.warp_table * sizeof(int);
    if (ti == 0) kb_sample<512><<<g, kDedupThreads, sm, st>>>(b);
    else if (ti == 1) kb_sample<1024><<<g, kDedupThreads, sm, st>>>(b);
    else kb_sample<2048><<<g, kDedupThreads, sm, st>>>(b);
    if (ev) cudaEventRecord(ev[2], st);
    kb_heavy<<<L->sms, kHeavyThreads, L->kb_heavy_dyn_smem, st>>>(b, L->kb_heavy_bitmap_words);
  } else if (ev) {
    cudaEventRecord(ev[2], st);
  }
  if (ev) cudaEventRecord(ev[3], st);
  const long long cap = (long long)L->sms * plan->tuning.flop_blocks_per_sm;
  const int g = (int)std::min<long long>(plan->total_tiles, cap);
  prof_mark(false, st);
  kb_flop<<<g, kFlopThreads, 0, st>>>(b);
  prof_mark(true, st);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

int batch_prepare(const spgemm_batch_item_t* items, int n, const spgemm_batch_tuning_t* tuning,
                  spgemm_batch_plan_t* plan, void* ws, size_t ws_bytes, void* host_staging,
                  size_t staging_bytes, int* bad_item, cudaStream_t st) {
  if (!items || n <= 0 || n > SPGEMM_BATCH_MAX_CASES || !plan || !ws) return SPGEMM_ERR_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(ws) & 255) return SPGEMM_ERR_WORKSPACE;
  // host checks first (tuning ranges, every case), then the device limits
  spgemm_batch_tuning_t tu;
  int rc = resolve_tuning(tuning, nullptr, &tu);
  if (rc) return rc;
  BatchTotals T;
  int bad = -1;
  if ((rc = batch_totals(items, n, tu.tile_items, tu.sample_chunk, &T, &bad))) {
    if (bad_item && bad >= 0) *bad_item = bad;
    return rc;
  }
  const BatchLayout l = layout_of(T, n);
  if (ws_bytes < l.total) return SPGEMM_ERR_WORKSPACE;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  if ((rc = resolve_tuning(&tu, L, &tu))) return rc;
  std::vector<unsigned char> own;
  unsigned char* buf = static_cast<unsigned char*>(host_staging);
  if (buf) {
    if (staging_bytes < l.plan_bytes()) return SPGEMM_ERR_INVALID_ARG;
  } else {
    own.resize(l.plan_bytes());
    buf = own.data();
  }
  char* dev = static_cast<char*>(ws);
  BatchCase* cs = reinterpret_cast<BatchCase*>(buf);
  int* tile_case = reinterpret_cast<int*>(buf + (l.tile_case - l.cases));
  int* chunk_case = reinterpret_cast<int*>(buf + (l.chunk_case - l.cases));
  int* tab_case = reinterpret_cast<int*>(buf + (l.tab_case - l.cases));
  long long row = 0, cand = 0, tile = 0, tab = 0, ch = 0;
  size_t deg = l.deg;
  for (int i = 0; i < n; ++i) {
    const spgemm_batch_item_t& it = items[i];
    long long nc = 0;
    sample_candidates(&it.cfg, it.A.rows, &nc);
    BatchCase& c = cs[i];
    c.a_rpt = it.A.rpt;
    c.a_col = it.A.col;
    c.b_rpt = it.B.rpt;
    c.b_col = it.B.col;
    c.M = it.A.rows;
    c.K = it.A.cols;
    c.N = it.B.cols;
    c.nnzA = it.A.nnz;
    c.nnzB = it.B.nnz;
    c.seed = it.cfg.seed;
    c.threshold = it.cfg.threshold;
    c.n_cand = nc;
    c.cand_off = cand;
    c.row_base = row;
    c.tab_blk0 = tab;
    c.pred = it.pred_row;
    c.offsets = reinterpret_cast<long long*>(it.offsets);
    c.flop = it.flop_row;
    c.res = it.res;
    c.deg8 = reinterpret_cast<unsigned char*>(dev + deg);
    c.src = it.cfg.mode == SPGEMM_SAMPLE_BERNOULLI ? kSrcBernoulli : kSrcDraws;
    c.vec_ok = ((reinterpret_cast<uintptr_t>(it.A.col) | reinterpret_cast<uintptr_t>(it.B.rpt)) & 15) == 0;
    const long long nt = tiles_of(it, tu.tile_items);
    c.tile0 = (int)tile;
    c.ntiles = (int)nt;
    for (long long q = 0; q < nt; ++q) tile_case[tile + q] = i;
    const long long nb = tab_blocks_of(it);
    for (long long q = 0; q < nb; ++q) tab_case[tab + q] = i;
    // chunks whose first candidate falls in this case
    for (; ch < T.chunks && ch * (long long)tu.sample_chunk < cand + nc; ++ch) chunk_case[ch] = i;
    row += it.A.rows;
    cand += nc;
    tile += nt;
    tab += nb;
    deg += r16((size_t)it.A.cols + 16);
  }
  if (cudaMemcpyAsync(dev + l.cases, buf, l.plan_bytes(), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return SPGEMM_ERR_CUDA;
  if (cudaMemsetAsync(dev + l.acc, 0, sizeof(CaseAcc) * (size_t)n, st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  // the tile slots of this plan may lie where another plan kept other data:
  // their flags start from zero
  if (cudaMemsetAsync(dev + l.slots, 0, sizeof(Slot) * (size_t)T.tiles, st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  if (!host_staging && cudaStreamSynchronize(st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  spgemm_batch_plan_t p{};
  p.n_cases = n;
  p.total_rows = T.rows;
  p.total_candidates = T.cand;
  p.total_tiles = T.tiles;
  p.total_chunks = T.chunks;
  p.total_table_blocks = T.tab;
  p.ws_bytes = l.total;
  p.tuning = tu;
  *plan = p;
  return SPGEMM_OK;
}

// ---- numeric product into a given allocation (the consumer of the prediction)

int numeric_check(const spgemm_csr_t* A, const float* a_val, const spgemm_csr_t* B, const float* b_val,
                  const void* c_col, const void* c_val, int64_t c_capacity, const int64_t* row_start,
                  const int32_t* nnz_row, const spgemm_numeric_result_t* res, void* ws, size_t ws_bytes) {
  if (!csr_ok(A) || !csr_ok(B) || !res || !ws) return SPGEMM_ERR_INVALID_ARG;
  if ((A->nnz > 0 && !a_val) || (B->nnz > 0 && !b_val)) return SPGEMM_ERR_INVALID_ARG;
  if (A->rows > 0 && (!nnz_row || !row_start)) return SPGEMM_ERR_INVALID_ARG;
  if (c_capacity < 0 || (c_capacity > 0 && (!c_col || !c_val))) return SPGEMM_ERR_INVALID_ARG;
  if (A->cols != B->rows) return SPGEMM_ERR_DIM_MISMATCH;
  if (!csr_fits(A) || !csr_fits(B)) return SPGEMM_ERR_TOO_LARGE;
  // the documented size (as for every other call), although only the part for
  // A's rows and columns is used here
  if (ws_bytes < ws_bytes_for(A->rows, A->cols, B->cols)) return SPGEMM_ERR_WORKSPACE;
  if ((reinterpret_cast<uintptr_t>(ws) & 255) != 0) return SPGEMM_ERR_WORKSPACE;
  return SPGEMM_OK;
}

NumArgs numeric_args(const spgemm_csr_t* A, const float* a_val, const spgemm_csr_t* B, const float* b_val,
                     const int64_t* alloc, int32_t* c_col, float* c_val, int64_t c_capacity,
                     int64_t* row_start, int32_t* nnz_row, spgemm_numeric_result_t* res, const Workspace& w) {
  NumArgs a;
  a.M = A->rows;
  a.K = B->rows;
  a.N = B->cols;
  a.nnzA = A->nnz;
  a.nnzB = B->nnz;
  a.a_rpt = A->rpt;
  a.a_col = A->col;
  a.a_val = a_val;
  a.b_rpt = B->rpt;
  a.b_col = B->col;
  a.b_val = b_val;
  a.alloc = reinterpret_cast<const long long*>(alloc);
  a.c_col = c_col;
  a.c_val = c_val;
  a.alloc_cap = c_capacity;
  // pool mode: about one stripe per 64 K entries, at most kPoolStripes
  a.pool_stripes = (int)std::max<long long>(1, std::min<long long>(kPoolStripes, c_capacity >> 16));
  a.slots = w.slots;
  a.row_start = reinterpret_cast<long long*>(row_start);
  a.nnz_row = nnz_row;
  a.out_rpt = nullptr;
  a.out_col = nullptr;
  a.out_val = nullptr;
  a.out_cap = 0;
  a.mode = kNumInto;
  a.heavy_count = &w.hdr->heavy_count;
  a.heavy = w.heavy;
  a.heavy_cap = A->rows;
  a.status = &w.hdr->status;
  a.res = res;
  return a;
}

// Warp-per-row pass, block-per-row pass over the rows it queued, finish;
// the compaction first moves the rows that fitted.
int launch_numeric(const DeviceLimits* L, const NumArgs& a, cudaStream_t st) {
  if (a.M > 0) {
    if (a.mode == kNumCompact) k_numeric_move<<<L->sms * 8, kMoveThreads, 0, st>>>(a);
    const int g = grid_for(a.M, kNumWarps, (long long)L->sms * L->num_blocks_per_sm);
    k_numeric_rows<<<g, kNumThreads, kNumRowsSmem, st>>>(a);
    k_numeric_heavy<<<L->sms, kNumHeavyThreads, kNumHeavySmem, st>>>(a);
  }
  k_numeric_finish<<<1, 1, 0, st>>>(a, a.status);
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t spgemm_workspace_size(const spgemm_csr_t* A, const spgemm_csr_t* B) {
  (void)B;
  if (!A || A->rows < 0) return 0;
  return ws_bytes_for(A->rows, A->cols, B ? B->cols : A->cols);
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

int spgemm_numeric_into(const spgemm_csr_t* A, const float* a_val, const spgemm_csr_t* B,
                        const float* b_val, const int64_t* alloc_offsets, int32_t* c_col,
                        float* c_val, int64_t c_capacity, int64_t* row_start, int32_t* nnz_row,
                        spgemm_numeric_result_t* res, void* ws, size_t ws_bytes, void* stream) {
  int rc = numeric_check(A, a_val, B, b_val, c_col, c_val, c_capacity, row_start, nnz_row, res, ws, ws_bytes);
  if (rc) return rc;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = ws_carve(ws, A->rows);
  if (cudaMemsetAsync(res, 0, sizeof(*res), st) != cudaSuccess) return SPGEMM_ERR_CUDA;
  const NumArgs a = numeric_args(A, a_val, B, b_val, alloc_offsets, c_col, c_val, c_capacity, row_start, nnz_row,
                                 res, w);
  return launch_numeric(L, a, st);
}

int spgemm_numeric_compact(const spgemm_csr_t* A, const float* a_val, const spgemm_csr_t* B,
                           const float* b_val, const int32_t* c_col, const float* c_val, int64_t c_capacity,
                           const int64_t* row_start, const int32_t* nnz_row, int64_t* out_rpt, int32_t* out_col,
                           float* out_val, int64_t out_capacity, spgemm_numeric_result_t* res, void* ws,
                           size_t ws_bytes, void* stream) {
  int rc = numeric_check(A, a_val, B, b_val, c_col, c_val, c_capacity, row_start, nnz_row, res, ws, ws_bytes);
  if (rc) return rc;
  if (!out_rpt || out_capacity < 0 || (out_capacity > 0 && (!out_col || !out_val))) return SPGEMM_ERR_INVALID_ARG;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Workspace w = ws_carve(ws, A->rows);
  // the allocation, row_start and nnz_row are only read here
  NumArgs a = numeric_args(A, a_val, B, b_val, nullptr, const_cast<int32_t*>(c_col), const_cast<float*>(c_val),
                           c_capacity, const_cast<int64_t*>(row_start), const_cast<int32_t*>(nnz_row), res, w);
  a.mode = kNumCompact;
  a.out_rpt = reinterpret_cast<const long long*>(out_rpt);
  a.out_col = out_col;
  a.out_val = out_val;
  a.out_cap = out_capacity;
  ScanNumNnz src{nnz_row, reinterpret_cast<long long*>(out_rpt)};
  if ((rc = launch_scan<ScanNumNnz, false, spgemm_numeric_result_t>(L, src, A->rows, w, res, st))) return rc;
  return launch_numeric(L, a, st);
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
  // Every host check comes first, so that a rejected call has queued nothing.
  if (!csr_ok(A) || !csr_ok(B) || !res) return SPGEMM_ERR_INVALID_ARG;
  if (A->cols != B->rows) return SPGEMM_ERR_DIM_MISMATCH;
  if (!csr_fits(A) || !csr_fits(B)) return SPGEMM_ERR_TOO_LARGE;
  if (!offsets || (!pred_row && A->rows > 0)) return SPGEMM_ERR_INVALID_ARG;
  long long n_cand = 0;
  int rc = sample_candidates(cfg, A->rows, &n_cand);
  if (rc) return rc;
  if (A->rows > SPGEMM_STATIC_MAX_ROWS || A->cols > SPGEMM_STATIC_MAX_ROWS || B->cols > SPGEMM_STATIC_MAX_ROWS)
    return SPGEMM_ERR_STATIC_CAPACITY;
  if (ws_bytes_for(A->rows, A->cols, B->cols) > kStaticBytes) return SPGEMM_ERR_STATIC_CAPACITY;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return SPGEMM_ERR_CUDA;
  }
  std::call_once(g_static_once[dev], init_static_scratch, dev);
  void* ws = g_static_ptr[dev];
  if (!ws) return SPGEMM_ERR_CUDA;
  if (!limits()) return SPGEMM_ERR_CUDA;
  // Header, per-block slots and flag epoch, the heavy-row queue and the
  // split-row slots (present when B has columns) start from zero on every call
  // (a call that ended with an error may have left them dirty).
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Workspace w = ws_carve(ws, A->rows, A->cols, B->cols);
  bool ok = cudaMemsetAsync(ws, 0, kStaticHeaderBytes, st) == cudaSuccess &&
            cudaMemsetAsync(w.heavy, 0, (size_t)(A->rows > 0 ? A->rows : 1) * sizeof(int), st) == cudaSuccess;
  if (ok && w.huge) ok = cudaMemsetAsync(w.huge, 0, sizeof(HugeSlot) * kHugeSlots, st) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();  // leave no error behind for the next call to find
    return SPGEMM_ERR_CUDA;
  }
  return predict_common(A, B, cfg, pred_row, offsets, flop_row, res, ws, kStaticBytes, stream, false);
}

size_t spgemm_batch_workspace_size(const spgemm_batch_item_t* items, int32_t n) {
  if (!items || n <= 0 || n > SPGEMM_BATCH_MAX_CASES) return 0;
  BatchTotals T;
  int bad = -1;
  if (batch_totals(items, n, kMinTile, kMinChunk, &T, &bad)) return 0;
  return layout_of(T, n).total;
}

size_t spgemm_batch_staging_size(const spgemm_batch_item_t* items, int32_t n) {
  if (!items || n <= 0 || n > SPGEMM_BATCH_MAX_CASES) return 0;
  BatchTotals T;
  int bad = -1;
  if (batch_totals(items, n, kMinTile, kMinChunk, &T, &bad)) return 0;
  return layout_of(T, n).plan_bytes();
}

int spgemm_batch_prepare(const spgemm_batch_item_t* items, int32_t n,
                         const spgemm_batch_tuning_t* tuning, spgemm_batch_plan_t* plan,
                         void* ws, size_t ws_bytes, void* host_staging, size_t staging_bytes,
                         int32_t* bad_item, void* stream) {
  int bad = -1;
  const int rc = batch_prepare(items, n, tuning, plan, ws, ws_bytes, host_staging, staging_bytes, &bad,
                               static_cast<cudaStream_t>(stream));
  if (rc && bad_item && bad >= 0) *bad_item = bad;
  return rc;
}

int spgemm_predict_batch(const spgemm_batch_plan_t* plan, void* ws, size_t ws_bytes, void* stream) {
  if (!plan || !ws || plan->n_cases <= 0 || plan->total_tiles <= 0) return SPGEMM_ERR_INVALID_ARG;
  if (ws_bytes < plan->ws_bytes || (reinterpret_cast<uintptr_t>(ws) & 255)) return SPGEMM_ERR_WORKSPACE;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  spgemm_batch_tuning_t tu;
  if (resolve_tuning(&plan->tuning, L, &tu)) return SPGEMM_ERR_INVALID_ARG;
  return launch_batch(L, plan, ws, static_cast<cudaStream_t>(stream), nullptr);
}

int spgemm_batch_autotune(const spgemm_batch_item_t* items, int32_t n, void* ws, size_t ws_bytes,
                          int32_t reps, spgemm_batch_tuning_t* best, float* best_ms,
                          spgemm_batch_plan_t* plan, void* stream) {
  if (!best || !plan || reps < 1 || reps > 1000) return SPGEMM_ERR_INVALID_ARG;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t ev[5];
  for (int i = 0; i < 5; ++i)
    if (cudaEventCreate(&ev[i]) != cudaSuccess) return SPGEMM_ERR_CUDA;
  // median over `reps` runs of the time between events a and b
  auto measure = [&](const spgemm_batch_tuning_t& tu, int a, int b, float* out) -> int {
    int rc = batch_prepare(items, n, &tu, plan, ws, ws_bytes, nullptr, 0, nullptr, st);
    if (rc) return rc;
    if ((rc = launch_batch(L, plan, ws, st, ev))) return rc;
    std::vector<float> ts;
    for (int r = 0; r < reps; ++r) {
      if ((rc = launch_batch(L, plan, ws, st, ev))) return rc;
      if (cudaEventSynchronize(ev[4]) != cudaSuccess) return SPGEMM_ERR_CUDA;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[a], ev[b]) != cudaSuccess) return SPGEMM_ERR_CUDA;
      ts.push_back(ms);
    }
    std::sort(ts.begin(), ts.end());
    *out = ts[ts.size() / 2];
    return SPGEMM_OK;
  };
  int rc = SPGEMM_OK;
  spgemm_batch_tuning_t cur{};
  float t_best = 0.f;
  // 1) the sampled-row passes: table size, heavy threshold, chunk size
  bool first = true;
  const int tables[3] = {512, 1024, 2048};
  const int chunks[3] = {8192, 32768, 131072};
  for (int ti = 0; ti < 3 && !rc; ++ti) {
    for (int hi = 0; hi < 2 && !rc; ++hi) {
      for (int ci = 0; ci < 3 && !rc; ++ci) {
        spgemm_batch_tuning_t tu{};
        tu.launches = 4;  // phases timed apart
        tu.warp_table = tables[ti];
        tu.heavy_threshold = hi == 0 ? tables[ti] / 4 : tables[ti] / 2;
        tu.sample_chunk = chunks[ci];
        float ms = 0.f;
        if ((rc = measure(tu, 1, 3, &ms))) break;
        if (first || ms < t_best) {
          cur = tu;
          t_best = ms;
          first = false;
        }
      }
    }
  }
  // 2) the FLOP pass: tile size and blocks per SM
  first = true;
  const int tiles[5] = {4096, 8192, 16384, 32768, 65536};
  spgemm_batch_tuning_t pick = cur;
  for (int ti = 0; ti < 5 && !rc; ++ti) {
    for (int bps = L->kb_flop_blocks_per_sm; bps >= 1 && bps >= L->kb_flop_blocks_per_sm - 2 && !rc; --bps) {
      spgemm_batch_tuning_t tu = cur;
      tu.tile_items = tiles[ti];
      tu.flop_blocks_per_sm = bps;
      float ms = 0.f;
      if ((rc = measure(tu, 3, 4, &ms))) break;
      if (first || ms < t_best) {
        pick = tu;
        t_best = ms;
        first = false;
      }
    }
  }
  // 3) the pick, end to end, in both forms; the faster is kept and the workspace
  // left prepared with it
  float total = 0.f;
  if (!rc) rc = measure(pick, 0, 4, &total);
  if (!rc) {
    spgemm_batch_tuning_t one = pick;
    one.launches = 1;
    float t1 = 0.f;
    if (!(rc = measure(one, 0, 4, &t1)) && t1 < total) {
      pick = one;
      total = t1;
    }
    if (!rc && pick.launches == 4) rc = measure(pick, 0, 4, &total);  // leave the workspace prepared with the pick
  }
  for (int i = 0; i < 5; ++i) cudaEventDestroy(ev[i]);
  if (rc) return rc;
  *best = pick;
  if (best_ms) *best_ms = total;
  return SPGEMM_OK;
}

int spgemm_predict_many(const spgemm_batch_item_t* items, int32_t n, void* const* ws, const size_t* ws_bytes,
                        int32_t* bad_item, void* stream) {
  if (!items || n < 0 || (n > 0 && (!ws || !ws_bytes))) return SPGEMM_ERR_INVALID_ARG;
  for (int32_t i = 0; i < n; ++i) {
    const spgemm_batch_item_t& it = items[i];
    const int rc = predict_common(&it.A, &it.B, &it.cfg, it.pred_row, it.offsets, it.flop_row, it.res, ws[i],
                                  ws_bytes[i], stream, false);
    if (rc != SPGEMM_OK) {
      if (bad_item) *bad_item = i;
      return rc;
    }
  }
  return SPGEMM_OK;
}

int spgemm_lookup_probe(const int32_t* col, int64_t n, const uint8_t* table, int64_t table_bytes,
                        uint64_t* out, void* stream) {
  if (n < 0 || table_bytes < 0 || !out) return SPGEMM_ERR_INVALID_ARG;
  if (n > 0 && (!col || (reinterpret_cast<uintptr_t>(col) & 15) != 0)) return SPGEMM_ERR_INVALID_ARG;
  if (table_bytes > 0 && !table) return SPGEMM_ERR_INVALID_ARG;
  const DeviceLimits* L = limits();
  if (!L) return SPGEMM_ERR_CUDA;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(out, 0, sizeof(uint64_t), st) != cudaSuccess) {
    cudaGetLastError();
    return SPGEMM_ERR_CUDA;
  }
  k_lookup_probe<<<L->sms, kProbeThreads, 0, st>>>(col, n, table, table_bytes,
                                                   reinterpret_cast<unsigned long long*>(out));
  return cudaGetLastError() == cudaSuccess ? SPGEMM_OK : SPGEMM_ERR_CUDA;
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
      return "A.rows, A.cols or B.cols exceeds the static scratch of spgemm_predict_structure_static (SPGEMM_STATIC_MAX_ROWS)";
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
