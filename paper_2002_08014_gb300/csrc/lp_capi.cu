// C ABI and round scheduler of the LocalPower library.
//
// The host side drives Alg. 1 round by round on one CUDA stream:
//   round start   Z = orth(Y)                          (cholqr2, batch 1)
//   local steps   Z_i = orth(Y_i) (j > 1, batch m)      (cholqr2)
//                 P = A^T (A Z_i) per row segment       (fused step kernel)
//                 Y_i = (1/s_i) sum of P over i's slots (reduce)
//   aggregation   D_i (sign / OPT, skipped when p_t = 1) then Y = sum_i p_i Y_i D_i
//   output        Z_T = orth(Y), optionally Rayleigh-Ritz
// Device state is FP32 d x K blocks (K = k rounded up to 8, 16 or 32, padding
// columns zero); the k x k factorisations run inside the kernels (FP32 with an
// FP64 Cholesky fallback for small pivots; FP64 Ritz matrix).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lp_internal.cuh"

using lp::Segment;

struct lp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0;
  size_t used = 0;
  int sms = 0;
  std::string err;

  // partitions
  int m = 0;
  int64_t d = 0, ld = 0, n = 0;
  lp_dtype dtype = LP_F32;
  std::vector<int64_t> rows, row_off;
  void* dA = nullptr;
  size_t dA_bytes = 0;
  float* dScales = nullptr;
  float smax2 = 1.f;  // FP8: the largest squared row scale (the tensor-core kernel's W scale)
  int base = 0;

  // step-kernel schedule
  int grid = 0;
  int nslots = 0;
  Segment* dSegs = nullptr;
  int* dSegPtr = nullptr;
  int* dSlotBegin = nullptr;
  float* dInvS = nullptr;
  float* dW = nullptr;

  // tensor-core step schedule (BF16 partitions): one segment list per cluster
  bool tc_ready = false;
  lp::TcPlan tc;
  int nslots_tc = 0;
  Segment* dSegsTc = nullptr;
  int* dSegPtrTc = nullptr;
  int* dSlotBeginTc = nullptr;

  // streaming tensor-core step (BF16 plane or hi/lo planes): plans per padded k
  // (index 0, 1, 2 for K = 8, 16, 32; state 0 = not planned, 1 = ready, -1 = none)
  int planes = 0;  // 1 for LP_BF16, 2 for LP_F32_BF16X2, 0 otherwise
  lp::TcsPlan tcs[3];
  int tcs_state[3] = {0, 0, 0};
  int tcs_G = 0;  // clusters the device segment table below was built for
  int nslots_tcs = 0;
  int max_slots[3] = {0, 0, 0};  // most slots of one partition, per path (SIMT, resident, streaming)
  Segment* dSegsTcs = nullptr;
  int* dSegPtrTcs = nullptr;
  int* dSlotBeginTcs = nullptr;
  const lp::TcsPlan* tcs_cur = nullptr;

  int path = 0;  // step kernel of the current solve / step (lp_stats::path)
  lp::TcsTuning tuning;
  bool prefer_resident = false;  // set by lp_autotune for LP_BF16 data

  // Independent problems sharing this context's partitions (the batch runner's
  // groups): problem q owns partitions [prob_begin[q], prob_begin[q + 1]), has
  // its own start block, bases, weights s_i / n_q, aggregate and result.  An
  // ordinary context is one problem.
  int nprob = 1;
  std::vector<int> prob_begin;
  std::vector<int64_t> prob_n;
  int* dPartProb = nullptr;   // partition -> problem
  int* dPartBase = nullptr;   // partition -> its problem's base partition
  int* dProbBegin = nullptr;  // nprob + 1 partition offsets
  double* dProbN = nullptr;   // rows per problem (the Ritz values' scale)

  // per-round records (LP_FLAG_TRACE): Z_t blocks and per-partition residuals
  float* dTraceZ = nullptr;
  double* dTraceRho = nullptr;
  size_t trace_z_bytes = 0, trace_rho_bytes = 0;
  int traced_rounds = 0;  // rounds recorded by the last solve (0: none)

  // CUDA graph of the last solve's launch sequence, replayed while its key matches
  uint64_t gen = 1;  // bumped whenever buffers, plans or tuning change
  std::vector<int64_t> graph_key;
  cudaGraphExec_t graph_exec = nullptr;
  lp_stats graph_stats{};
  int graph_step_ev_used = 0;

  // solve state (capacity in K)
  int Kcap = 0;
  float *dP = nullptr, *dYl = nullptr, *dZl = nullptr, *dY = nullptr, *dZ = nullptr, *dG = nullptr, *dMZ = nullptr;
  double *dZout = nullptr, *dSigma = nullptr, *dStage = nullptr;
  size_t stage_bytes = 0;
  int* dStatus = nullptr;

  // last solve
  bool solved = false;
  int k = 0;
  bool ritz = false;
  lp_stats stats{};
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> step_ev;
  int step_ev_used = 0;
};

namespace {

thread_local std::string g_create_err;

lp_status fail(lp_ctx* c, lp_status st, const std::string& msg) {
  if (c) c->err = msg;
  else g_create_err = msg;
  return st;
}

lp_status cuda_fail(lp_ctx* c, cudaError_t e, const char* what) {
  return fail(c, LP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define LP_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

// Device allocation against the context's budget.  Nothing is allocated on failure.
template <typename T>
lp_status dalloc(lp_ctx* c, T** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) / 256 * 256;
  if (c->budget && c->used + bytes > c->budget)
    return fail(c, LP_ERR_OOM, "HBM budget exceeded: need " + std::to_string(bytes) + " more bytes, budget " +
                                   std::to_string(c->budget) + ", in use " + std::to_string(c->used));
  void* q = nullptr;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    (void)cudaGetLastError();
    return fail(c, LP_ERR_OOM, std::string("cudaMalloc of ") + std::to_string(bytes) + " bytes failed: " +
                                   cudaGetErrorString(e));
  }
  c->used += bytes;
  *p = static_cast<T*>(q);
  return LP_OK;
}

template <typename T>
void dfree(lp_ctx* c, T*& p, size_t bytes) {
  if (p) {
    cudaFree(p);
    if (bytes == 0) bytes = 16;
    c->used -= (bytes + 255) / 256 * 256;
    p = nullptr;
  }
}

enum Path { PATH_SIMT = 0, PATH_TC = 1, PATH_TCS = 2 };
// What LP_KERNEL_DEFAULT means for the tensor-core step.
constexpr int kDefaultTcKernel = LP_KERNEL_PAIR;
// lp_stats::path code of the pass-split pair kernel (it shares PATH_TCS's tables).
constexpr int kReportedPathPair = 3;

// Tensor-core step kernels accumulate a segment's A^T W in TMEM, and the tensor
// cores round that FP32 accumulator toward zero on every MMA, so a long chain
// shrinks the result a little (about half an ulp per MMA).  Their segments are
// cut into pieces of at most this many rows (32 tiles, 256 accumulating MMAs
// per entry); the reduction adds the pieces with round-to-nearest.
constexpr int64_t kTcChainRows = 4096;

// Most segments any step kernel's table can have for `workers` workers: each
// worker's row range is cut at partition ends and into kTcChainRows pieces.
int64_t max_segments(int64_t workers, int64_t m, int64_t n) { return workers + m + n / kTcChainRows + 1; }

// Launches of the SIMT step per local step (0: no SIMT kernel for the shape).
int simt_launches(int d, int64_t ld, lp_dtype dtype, int K) {
  return lp::step_simt_smem(d, ld, dtype, K, nullptr) != 0 ? 1 : 0;
}

int kcap_of(int k) { return k <= 8 ? 8 : (k <= 16 ? 16 : 32); }
// Algorithmic bytes per element of A (both planes for LP_F32_BF16X2).
size_t elem_bytes(lp_dtype t) { return (t == LP_F32 || t == LP_F32_BF16X2) ? 4 : (t == LP_BF16 ? 2 : 1); }
// Bytes per stored element of one plane.
size_t plane_bytes(lp_dtype t) { return t == LP_F32_BF16X2 ? 2 : elem_bytes(t); }

// Forget the captured solve graph (buffers, plans or tuning changed).
void drop_graph(lp_ctx* c) {
  if (c->graph_exec) cudaGraphExecDestroy(c->graph_exec);
  c->graph_exec = nullptr;
  c->graph_key.clear();
  c->gen++;
}

struct StateSizes {
  size_t P, Yl, Y, G, stage;
};
StateSizes state_sizes(const lp_ctx* c, int K) {
  StateSizes s;
  s.P = size_t(max_segments(c->sms, c->m, c->n)) * c->d * K * 4;
  s.Yl = size_t(c->m) * c->d * K * 4;
  s.Y = size_t(c->nprob) * c->d * K * 4;
  s.G = size_t(c->m) * K * K * 4;
  s.stage = size_t(c->m) * c->d * K * 8;
  return s;
}

void free_state(lp_ctx* c) {
  if (!c->Kcap) return;
  StateSizes s = state_sizes(c, c->Kcap);
  dfree(c, c->dP, s.P);
  dfree(c, c->dYl, s.Yl);
  dfree(c, c->dZl, s.Yl);
  dfree(c, c->dY, s.Y);
  dfree(c, c->dZ, s.Y);
  dfree(c, c->dMZ, s.Y);
  dfree(c, c->dG, s.G);
  dfree(c, c->dZout, size_t(c->nprob) * c->d * LP_MAX_K * 8);
  dfree(c, c->dSigma, size_t(c->nprob) * LP_MAX_K * 8);
  dfree(c, c->dStage, c->stage_bytes);
  c->stage_bytes = 0;
  c->Kcap = 0;
  dfree(c, c->dTraceZ, c->trace_z_bytes);
  dfree(c, c->dTraceRho, c->trace_rho_bytes);
  c->trace_z_bytes = c->trace_rho_bytes = 0;
  c->traced_rounds = 0;
}

lp_status ensure_state(lp_ctx* c, int K) {
  if (c->Kcap >= K) return LP_OK;
  drop_graph(c);
  free_state(c);
  StateSizes s = state_sizes(c, K);
  lp_status st;
  if ((st = dalloc(c, &c->dP, s.P)) || (st = dalloc(c, &c->dYl, s.Yl)) || (st = dalloc(c, &c->dZl, s.Yl)) ||
      (st = dalloc(c, &c->dY, s.Y)) || (st = dalloc(c, &c->dZ, s.Y)) || (st = dalloc(c, &c->dMZ, s.Y)) ||
      (st = dalloc(c, &c->dG, s.G)) || (st = dalloc(c, &c->dZout, size_t(c->nprob) * c->d * LP_MAX_K * 8)) ||
      (st = dalloc(c, &c->dSigma, size_t(c->nprob) * LP_MAX_K * 8)) || (st = dalloc(c, &c->dStage, s.stage))) {
    c->Kcap = K;  // free what was allocated
    free_state(c);
    return st;
  }
  c->stage_bytes = s.stage;
  c->Kcap = K;
  return LP_OK;
}

void free_partitions(lp_ctx* c) {
  drop_graph(c);
  dfree(c, c->dA, c->dA_bytes);
  dfree(c, c->dScales, size_t(c->n) * 4);
  dfree(c, c->dSegs, (size_t(c->grid) + c->m) * sizeof(Segment));
  dfree(c, c->dSegPtr, (size_t(c->grid) + 1) * 4);
  dfree(c, c->dSlotBegin, (size_t(c->m) + 1) * 4);
  dfree(c, c->dInvS, size_t(c->m) * 4);
  dfree(c, c->dW, size_t(c->m) * 4);
  dfree(c, c->dSegsTc, size_t(max_segments(c->tc.nclusters, c->m, c->n)) * sizeof(Segment));
  dfree(c, c->dSegPtrTc, (size_t(c->tc.nclusters) + 1) * 4);
  dfree(c, c->dSlotBeginTc, (size_t(c->m) + 1) * 4);
  dfree(c, c->dSegsTcs, size_t(max_segments(c->sms, c->m, c->n)) * sizeof(Segment));
  dfree(c, c->dSegPtrTcs, (size_t(c->sms) + 1) * 4);
  dfree(c, c->dSlotBeginTcs, (size_t(c->m) + 1) * 4);
  free_state(c);
  dfree(c, c->dPartProb, size_t(c->m) * 4);
  dfree(c, c->dPartBase, size_t(c->m) * 4);
  dfree(c, c->dProbBegin, (size_t(c->nprob) + 1) * 4);
  dfree(c, c->dProbN, size_t(c->nprob) * 8);
  c->nprob = 1;
  c->prob_begin.clear();
  c->prob_n.clear();
  c->nslots_tc = 0;
  c->tc_ready = false;
  c->nslots_tcs = 0;
  c->tcs_G = 0;
  c->tcs_state[0] = c->tcs_state[1] = c->tcs_state[2] = 0;
  c->tcs_cur = nullptr;
  c->planes = 0;
  c->m = 0;
  c->n = 0;
  c->dA_bytes = 0;
  c->solved = false;
}

// Copy a d x k (or batch of) FP64 array from `space` to the device staging buffer.
lp_status stage_in(lp_ctx* c, const double* src, size_t count, lp_ptr_space space, const double** dev) {
  if (space == LP_DEVICE) {
    *dev = src;
    return LP_OK;
  }
  if (count * 8 > c->stage_bytes) return fail(c, LP_ERR_INVALID, "staging buffer too small");
  LP_CUDA(cudaMemcpyAsync(c->dStage, src, count * 8, cudaMemcpyHostToDevice, c->stream));
  *dev = c->dStage;
  return LP_OK;
}

// Contiguous row ranges for G workers (CTAs or clusters): worker g owns rows
// [g n / G, (g+1) n / G), cut at partition ends and, when max_rows > 0, into
// pieces of at most max_rows rows; one output slot per piece.  Partition i's
// slots are the contiguous range [slot_begin[i], slot_begin[i+1]).
void build_segments(const lp_ctx* c, int G, std::vector<Segment>& segs, std::vector<int>& seg_ptr,
                    std::vector<int>& slot_begin, int64_t max_rows = 0) {
  const int64_t n = c->n;
  const int m = c->m;
  segs.clear();
  seg_ptr.assign(G + 1, 0);
  slot_begin.assign(m + 1, 0);
  int part = 0;
  for (int g = 0; g < G; ++g) {
    seg_ptr[g] = static_cast<int>(segs.size());
    int64_t r0 = n * g / G, r1 = n * (g + 1) / G;
    while (r0 < r1) {
      while (c->row_off[part] + c->rows[part] <= r0) ++part;
      const int64_t pend = c->row_off[part] + c->rows[part];
      int64_t e = std::min(r1, pend);
      if (max_rows > 0) e = std::min(e, r0 + max_rows);
      Segment s;
      s.row0 = r0;
      s.row1 = e;
      s.part = part;
      s.slot = static_cast<int>(segs.size());
      segs.push_back(s);
      r0 = e;
    }
  }
  seg_ptr[G] = static_cast<int>(segs.size());
  const int nslots = static_cast<int>(segs.size());
  int s = 0;
  for (int i = 0; i < m; ++i) {
    while (s < nslots && segs[s].part < i) ++s;
    slot_begin[i] = s;
  }
  slot_begin[m] = nslots;
}

// Event record that also works inside a stream capture: there a plain record is
// only a dependency edge, so timing events become external event-record nodes.
cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  const cudaError_t q = cudaStreamIsCapturing(s, &cs);
  if (q != cudaSuccess) return q;
  return cudaEventRecordWithFlags(e, s, cs == cudaStreamCaptureStatusActive ? cudaEventRecordExternal
                                                                             : cudaEventRecordDefault);
}

int max_slots_in(const std::vector<int>& slot_begin) {
  int mx = 0;
  for (size_t i = 0; i + 1 < slot_begin.size(); ++i) mx = std::max(mx, slot_begin[i + 1] - slot_begin[i]);
  return mx;
}

int reported_path(const lp_ctx* c) {
  return c->path == PATH_TCS && c->tcs_cur && c->tcs_cur->pair ? kReportedPathPair : c->path;
}

const int* slot_begin_of(const lp_ctx* c) {
  return c->path == PATH_TCS ? c->dSlotBeginTcs : c->path == PATH_TC ? c->dSlotBeginTc : c->dSlotBegin;
}

lp_status launch_step(lp_ctx* c, int K, const float* Z, int64_t z_stride, bool timing) {
  lp::StepArgs a;
  a.A = c->dA;
  a.ld = c->ld;
  a.d = static_cast<int>(c->d);
  a.scales = c->dScales;
  a.segs = c->dSegs;
  a.seg_ptr = c->dSegPtr;
  a.Z = Z;
  a.z_stride = z_stride;
  a.P = c->dP;
  a.grid = c->grid;
  a.status = c->dStatus;
  if (timing) {
    const size_t need = size_t(c->step_ev_used) + 2;
    while (c->step_ev.size() < need) {
      cudaEvent_t e;
      LP_CUDA(cudaEventCreate(&e));
      c->step_ev.push_back(e);
    }
    LP_CUDA(record_event(c->step_ev[c->step_ev_used], c->stream));
  }
  cudaError_t e;
  if (c->path == PATH_TCS && c->tcs_cur->pair)
    e = lp::launch_step_pair(*c->tcs_cur, c->dSegsTcs, c->dSegPtrTcs, Z, z_stride, c->dP, static_cast<int>(c->d),
                             c->dStatus, c->stream);
  else if (c->path == PATH_TCS && c->tcs_cur->fp8)
    e = lp::launch_step_tcs8(*c->tcs_cur, c->dSegsTcs, c->dSegPtrTcs, Z, z_stride, c->dP, static_cast<int>(c->d),
                             c->dScales, c->smax2, c->dStatus, c->stream);
  else if (c->path == PATH_TCS)
    e = lp::launch_step_tcs(*c->tcs_cur, c->dSegsTcs, c->dSegPtrTcs, Z, z_stride, c->dP, static_cast<int>(c->d),
                            c->dStatus, c->stream);
  else if (c->path == PATH_TC)
    e = lp::launch_step_tc(c->tc, c->dSegsTc, c->dSegPtrTc, Z, z_stride, c->dP, static_cast<int>(c->d), c->dStatus,
                           c->stream);
  else
    e = lp::launch_step_simt(a, c->dtype, K, c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "fused power-step launch");
  if (timing) {
    LP_CUDA(record_event(c->step_ev[c->step_ev_used + 1], c->stream));
    c->step_ev_used += 2;
  }
  c->stats.step_launches++;
  c->stats.kernel_launches++;
  c->stats.a_bytes += double(c->n) * double(c->d) * double(elem_bytes(c->dtype)) +
                      (c->dtype == LP_FP8_E4M3 ? 4.0 * double(c->n) : 0.0);
  return LP_OK;
}

lp_status check_launch(lp_ctx* c, cudaError_t e, const char* what) {
  if (e != cudaSuccess) return cuda_fail(c, e, what);
  c->stats.kernel_launches++;
  return LP_OK;
}

}  // namespace

void lp::set_no_context_error(const char* msg) { g_create_err = msg; }

// =============================================================================
extern "C" {

lp_status lp_create(lp_ctx** out, int device, size_t hbm_budget_bytes, void* cuda_stream) {
  if (!out) return fail(nullptr, LP_ERR_INVALID, "out is NULL");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    (void)cudaGetLastError();
    return fail(nullptr, LP_ERR_CUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  if (device < 0 || device >= ndev) return fail(nullptr, LP_ERR_INVALID, "device index out of range");
  lp_ctx* c = new (std::nothrow) lp_ctx();
  if (!c) return fail(nullptr, LP_ERR_OOM, "host allocation failed");
  c->device = device;
  c->budget = hbm_budget_bytes;
  e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) {
    if (cuda_stream) {
      c->stream = static_cast<cudaStream_t>(cuda_stream);
    } else {
      e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
      c->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&c->ev1);
  if (e == cudaSuccess && dalloc(c, &c->dStatus, 16) != LP_OK) e = cudaErrorMemoryAllocation;
  if (e != cudaSuccess) {
    std::string msg = std::string("context setup failed: ") + cudaGetErrorString(e);
    lp_destroy(c);
    return fail(nullptr, LP_ERR_CUDA, msg);
  }
  *out = c;
  return LP_OK;
}

void lp_destroy(lp_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  free_partitions(c);
  dfree(c, c->dStatus, 16);
  drop_graph(c);
  for (cudaEvent_t e : c->step_ev) cudaEventDestroy(e);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* lp_last_error(const lp_ctx* c) { return c ? c->err.c_str() : g_create_err.c_str(); }

lp_status lp_load_partitions(lp_ctx* c, int m, const int64_t* rows, int64_t d, lp_dtype dtype,
                             const void* const* parts, const float* const* row_scales, lp_ptr_space space) {
  return lp::load_pitched(c, m, rows, d, d, dtype, parts, row_scales, space);
}

}  // extern "C"

// Buffers, segment tables, plans and weights for m partitions of the given row
// counts (n in total), or - for the same shapes as loaded now - the existing ones
// (*reused).  The caller then copies the data into c->dA (and c->dScales).
static lp_status setup_partitions(lp_ctx* c, int m, const int64_t* rows, int64_t d, lp_dtype dtype, int64_t n,
                                  bool* reused) {
  LP_CUDA(cudaSetDevice(c->device));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  // New data of the same shapes (m, rows, d, dtype) go into the existing buffers:
  // allocations, segment tables, tensor maps, tuning and captured graphs stay.
  const bool reuse = c->dA && c->m == m && c->d == d && c->dtype == dtype && c->n == n &&
                     std::equal(rows, rows + m, c->rows.begin());
  if (!reuse) {
    free_partitions(c);
  } else {
    c->solved = false;  // the last result belongs to the old data
    c->traced_rounds = 0;
  }

  const bool split = dtype == LP_F32_BF16X2;
  if (split) {
    lp::TcsPlan probe;
    if (!lp::tcs_plan(static_cast<int>(d), 8, 2, c->sms, lp::TcsTuning{}, &probe))
      return fail(c, LP_ERR_UNSUPPORTED, "split-plane storage has no tensor-core kernel for d=" + std::to_string(d));
  }
  const size_t eb = plane_bytes(dtype);  // bytes per stored element of one plane
  const int nplanes = split ? 2 : 1;
  const int64_t per16 = 16 / static_cast<int64_t>(eb);
  c->m = m;
  c->d = d;
  c->ld = (d + per16 - 1) / per16 * per16;
  c->n = n;
  c->dtype = dtype;
  c->planes = dtype == LP_BF16 ? 1 : (split ? 2 : 0);
  c->rows.assign(rows, rows + m);
  c->row_off.resize(m);
  int64_t o = 0;
  for (int i = 0; i < m; ++i) {
    c->row_off[i] = o;
    o += rows[i];
  }
  c->base = static_cast<int>(std::max_element(c->rows.begin(), c->rows.end()) - c->rows.begin());

  lp_status st;
  if (!reuse) {
  // Row segments of the SIMT step kernel: CTA g owns rows [g n / G, (g+1) n / G), cut at partition ends.
  const int64_t min_rows = 32;
  c->grid = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->sms, n / min_rows)));
  std::vector<Segment> segs;
  std::vector<int> seg_ptr, slot_begin;
  build_segments(c, c->grid, segs, seg_ptr, slot_begin);
  c->nslots = static_cast<int>(segs.size());
  c->max_slots[PATH_SIMT] = max_slots_in(slot_begin);
  // Tensor-core step kernel (BF16): one segment table per cluster of CTAs.
  std::vector<Segment> segs_tc;
  std::vector<int> seg_ptr_tc, slot_begin_tc;
  c->tc_ready = false;
  if (dtype == LP_BF16 && lp::tc_plan(static_cast<int>(d), LP_MAX_K, c->sms, &c->tc)) {
    const int G = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(c->tc.nclusters, (n + 127) / 128)));
    c->tc.nclusters = G;
    build_segments(c, G, segs_tc, seg_ptr_tc, slot_begin_tc, kTcChainRows);
    c->nslots_tc = static_cast<int>(segs_tc.size());
    c->max_slots[PATH_TC] = max_slots_in(slot_begin_tc);
    c->tc_ready = true;
  }
  std::vector<float> invs(m), w(m);
  for (int i = 0; i < m; ++i) {
    invs[i] = static_cast<float>(1.0 / double(rows[i]));
    w[i] = static_cast<float>(double(rows[i]) / double(n));
  }

  c->dA_bytes = size_t(n) * size_t(c->ld) * eb * nplanes;
  if ((st = dalloc(c, &c->dA, c->dA_bytes)) ||
      (dtype == LP_FP8_E4M3 && (st = dalloc(c, &c->dScales, size_t(n) * 4))) ||
      (st = dalloc(c, &c->dSegs, (size_t(c->grid) + m) * sizeof(Segment))) ||
      (st = dalloc(c, &c->dSegPtr, (size_t(c->grid) + 1) * 4)) ||
      (st = dalloc(c, &c->dSlotBegin, (size_t(m) + 1) * 4)) || (st = dalloc(c, &c->dInvS, size_t(m) * 4)) ||
      (st = dalloc(c, &c->dW, size_t(m) * 4)) ||
      (c->tc_ready && ((st = dalloc(c, &c->dSegsTc, size_t(max_segments(c->tc.nclusters, m, n)) * sizeof(Segment))) ||
                       (st = dalloc(c, &c->dSegPtrTc, (size_t(c->tc.nclusters) + 1) * 4)) ||
                       (st = dalloc(c, &c->dSlotBeginTc, (size_t(m) + 1) * 4))))) {
    std::string msg = c->err;
    free_partitions(c);
    c->err = msg;
    return st;
  }
  if (c->tc_ready) {
    if (lp::tc_encode_map(c->dA, n, static_cast<int>(d), c->ld, &c->tc) != cudaSuccess) {
      c->tc_ready = false;  // no tensor map: BF16 solves use the SIMT step kernel
    } else {
      LP_CUDA(cudaMemcpyAsync(c->dSegsTc, segs_tc.data(), segs_tc.size() * sizeof(Segment), cudaMemcpyHostToDevice,
                              c->stream));
      LP_CUDA(cudaMemcpyAsync(c->dSegPtrTc, seg_ptr_tc.data(), seg_ptr_tc.size() * 4, cudaMemcpyHostToDevice,
                              c->stream));
      LP_CUDA(cudaMemcpyAsync(c->dSlotBeginTc, slot_begin_tc.data(), slot_begin_tc.size() * 4,
                              cudaMemcpyHostToDevice, c->stream));
    }
  }
  LP_CUDA(cudaMemcpyAsync(c->dSegs, segs.data(), segs.size() * sizeof(Segment), cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dSegPtr, seg_ptr.data(), seg_ptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dSlotBegin, slot_begin.data(), slot_begin.size() * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dInvS, invs.data(), m * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dW, w.data(), m * 4, cudaMemcpyHostToDevice, c->stream));
  // the host vectors above are pageable: the copies must finish before they go
  LP_CUDA(cudaStreamSynchronize(c->stream));
  }
  if (c->nprob == 1) {
    c->prob_begin = {0, m};
    c->prob_n = {n};
  }
  *reused = reuse;
  return LP_OK;
}

lp_status lp::load_pitched(lp_ctx* c, int m, const int64_t* rows, int64_t d, int64_t pitch, lp_dtype dtype,
                           const void* const* parts, const float* const* row_scales, lp_ptr_space space) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (pitch < d) return fail(c, LP_ERR_INVALID, "row pitch below d");
  if (m < 1 || !rows || !parts) return fail(c, LP_ERR_INVALID, "need m >= 1 and non-NULL rows/parts");
  if (d < 1 || d > (1 << 20)) return fail(c, LP_ERR_INVALID, "d out of range");
  if (dtype != LP_F32 && dtype != LP_BF16 && dtype != LP_FP8_E4M3 && dtype != LP_F32_BF16X2)
    return fail(c, LP_ERR_INVALID, "unknown dtype");
  if (space != LP_HOST && space != LP_DEVICE) return fail(c, LP_ERR_INVALID, "unknown pointer space");
  if (dtype == LP_FP8_E4M3 && !row_scales) return fail(c, LP_ERR_INVALID, "FP8 partitions need row_scales");
  int64_t n = 0;
  for (int i = 0; i < m; ++i) {
    if (rows[i] < 1) return fail(c, LP_ERR_INVALID, "partition " + std::to_string(i) + " has no rows");
    if (!parts[i]) return fail(c, LP_ERR_INVALID, "partition " + std::to_string(i) + " pointer is NULL");
    if (dtype == LP_FP8_E4M3 && !row_scales[i])
      return fail(c, LP_ERR_INVALID, "partition " + std::to_string(i) + " scales pointer is NULL");
    n += rows[i];
  }
  bool reuse = false;
  lp_status st = setup_partitions(c, m, rows, d, dtype, n, &reuse);
  if (st) return st;
  const bool split = dtype == LP_F32_BF16X2;
  const size_t eb = plane_bytes(dtype);
  const cudaMemcpyKind kind = space == LP_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  if (split) {
    // FP32 -> hi / lo planes on the device; host data go through a bounded FP32 staging buffer.
    uint16_t* hi = static_cast<uint16_t*>(c->dA);
    uint16_t* lo = hi + size_t(n) * c->ld;
    float* stage = nullptr;
    const int64_t chunk_rows = std::max<int64_t>(1, (int64_t(1) << 24) / d);  // 64 MB of FP32
    size_t stage_bytes = 0;
    if (space == LP_HOST) {
      stage_bytes = size_t(std::min(chunk_rows, *std::max_element(c->rows.begin(), c->rows.end()))) * d * 4;
      if ((st = dalloc(c, &stage, stage_bytes))) {
        std::string msg = c->err;
        free_partitions(c);
        c->err = msg;
        return st;
      }
    }
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < m && e == cudaSuccess; ++i) {
      const float* src = static_cast<const float*>(parts[i]);
      for (int64_t r0 = 0; r0 < rows[i] && e == cudaSuccess; r0 += chunk_rows) {
        const int64_t nr = std::min(chunk_rows, rows[i] - r0);
        const size_t off = size_t(c->row_off[i] + r0) * c->ld;
        const float* from = src + size_t(r0) * pitch;
        int64_t from_ld = pitch;
        if (space == LP_HOST) {
          e = cudaMemcpy2DAsync(stage, size_t(d) * 4, from, size_t(pitch) * 4, size_t(d) * 4, size_t(nr),
                                cudaMemcpyHostToDevice, c->stream);
          from = stage;
          from_ld = d;
        }
        if (e == cudaSuccess)
          e = lp::launch_split_planes(from, from_ld, nr, static_cast<int>(d), hi + off, lo + off, c->ld, c->stream);
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dfree(c, stage, stage_bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "split-plane load");
  } else if (c->ld != d && !reuse) {  // padding columns; a reload rewrites only columns [0, d)
    LP_CUDA(cudaMemsetAsync(c->dA, 0, c->dA_bytes, c->stream));
  }
  for (int i = 0; i < m && !split; ++i) {
    char* dst = static_cast<char*>(c->dA) + size_t(c->row_off[i]) * c->ld * eb;
    LP_CUDA(cudaMemcpy2DAsync(dst, size_t(c->ld) * eb, parts[i], size_t(pitch) * eb, size_t(d) * eb, size_t(rows[i]), kind,
                              c->stream));
    if (dtype == LP_FP8_E4M3)
      LP_CUDA(cudaMemcpyAsync(c->dScales + c->row_off[i], row_scales[i], size_t(rows[i]) * 4, kind, c->stream));
  }
  LP_CUDA(cudaStreamSynchronize(c->stream));
  if (dtype == LP_FP8_E4M3) {  // S = max_r s_r^2 for the tensor-core kernel's W scale
    std::vector<float> sc(static_cast<size_t>(n));
    LP_CUDA(cudaMemcpy(sc.data(), c->dScales, size_t(n) * 4, cudaMemcpyDeviceToHost));
    float mx = 0.f;
    for (float v : sc) mx = std::max(mx, std::fabs(v));
    c->smax2 = mx > 0.f && std::isfinite(mx * mx) ? mx * mx : 1.f;
  }
  return LP_OK;
}

lp_status lp::load_merged(lp_ctx* c, lp_ctx* const* src, int nsrc) {
  if (!c || !src || nsrc < 1) return LP_ERR_INVALID;
  c->err.clear();
  const lp_ctx* s0 = src[0];
  std::vector<int64_t> rows;
  int64_t n = 0;
  for (int j = 0; j < nsrc; ++j) {
    const lp_ctx* sj = src[j];
    if (!sj || sj->m == 0 || sj->d != s0->d || sj->dtype != s0->dtype || sj->ld != s0->ld || sj->nprob != 1 ||
        sj->device != c->device)
      return fail(c, LP_ERR_INVALID, "merged contexts must hold loaded partitions of one width, type and device");
    rows.insert(rows.end(), sj->rows.begin(), sj->rows.end());
    n += sj->n;
  }
  LP_CUDA(cudaSetDevice(c->device));
  for (int j = 0; j < nsrc; ++j) LP_CUDA(cudaStreamSynchronize(src[j]->stream));
  bool reuse = false;
  lp_status st = setup_partitions(c, static_cast<int>(rows.size()), rows.data(), s0->d, s0->dtype, n, &reuse);
  if (st) return st;
  // the stored rows (padding columns included) plane by plane: plane p of a
  // context with N rows starts N * ld elements after plane p - 1
  const size_t eb = plane_bytes(s0->dtype), row_bytes = size_t(c->ld) * eb;
  const int nplanes = s0->dtype == LP_F32_BF16X2 ? 2 : 1;
  int64_t off = 0;
  float smax2 = 0.f;
  for (int j = 0; j < nsrc; ++j) {
    const lp_ctx* sj = src[j];
    for (int pl = 0; pl < nplanes; ++pl)
      LP_CUDA(cudaMemcpyAsync(static_cast<char*>(c->dA) + (size_t(pl) * n + off) * row_bytes,
                              static_cast<const char*>(sj->dA) + size_t(pl) * sj->n * row_bytes,
                              size_t(sj->n) * row_bytes, cudaMemcpyDeviceToDevice, c->stream));
    if (s0->dtype == LP_FP8_E4M3) {
      LP_CUDA(cudaMemcpyAsync(c->dScales + off, sj->dScales, size_t(sj->n) * 4, cudaMemcpyDeviceToDevice, c->stream));
      smax2 = std::max(smax2, sj->smax2);
    }
    off += sj->n;
  }
  if (s0->dtype == LP_FP8_E4M3) c->smax2 = smax2 > 0.f ? smax2 : 1.f;
  LP_CUDA(cudaStreamSynchronize(c->stream));
  std::vector<int> begin(nsrc + 1, 0);
  for (int j = 0; j < nsrc; ++j) begin[j + 1] = begin[j] + src[j]->m;
  return lp::set_problems(c, nsrc, begin.data());
}

lp_status lp::set_problems(lp_ctx* c, int nprob, const int* part_begin) {
  if (!c) return LP_ERR_INVALID;
  if (c->m == 0) return fail(c, LP_ERR_STATE, "no partitions loaded");
  if (nprob < 1 || !part_begin || part_begin[0] != 0 || part_begin[nprob] != c->m)
    return fail(c, LP_ERR_INVALID, "problem ranges must cover the partitions");
  for (int q = 0; q < nprob; ++q)
    if (part_begin[q + 1] <= part_begin[q]) return fail(c, LP_ERR_INVALID, "every problem needs a partition");
  LP_CUDA(cudaSetDevice(c->device));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  // the solve buffers are sized by the problem count
  drop_graph(c);
  free_state(c);
  dfree(c, c->dPartProb, size_t(c->m) * 4);
  dfree(c, c->dPartBase, size_t(c->m) * 4);
  dfree(c, c->dProbBegin, (size_t(c->nprob) + 1) * 4);
  dfree(c, c->dProbN, size_t(c->nprob) * 8);
  c->nprob = nprob;
  c->prob_begin.assign(part_begin, part_begin + nprob + 1);
  c->prob_n.assign(nprob, 0);
  std::vector<int> part_prob(c->m), part_base(c->m);
  std::vector<float> w(c->m);
  for (int q = 0; q < nprob; ++q) {
    int b = part_begin[q];
    for (int i = part_begin[q]; i < part_begin[q + 1]; ++i) {
      c->prob_n[q] += c->rows[i];
      if (c->rows[i] > c->rows[b]) b = i;  // the first largest partition, as for one problem
    }
    for (int i = part_begin[q]; i < part_begin[q + 1]; ++i) {
      part_prob[i] = q;
      part_base[i] = b;
      w[i] = static_cast<float>(double(c->rows[i]) / double(c->prob_n[q]));
    }
  }
  c->base = part_base[0];
  lp_status st;
  if ((st = dalloc(c, &c->dPartProb, size_t(c->m) * 4)) || (st = dalloc(c, &c->dPartBase, size_t(c->m) * 4)) ||
      (st = dalloc(c, &c->dProbBegin, (size_t(nprob) + 1) * 4)) || (st = dalloc(c, &c->dProbN, size_t(nprob) * 8)))
    return st;
  std::vector<double> prob_nd(c->prob_n.begin(), c->prob_n.end());
  LP_CUDA(cudaMemcpyAsync(c->dPartProb, part_prob.data(), size_t(c->m) * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dPartBase, part_base.data(), size_t(c->m) * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dProbBegin, part_begin, (size_t(nprob) + 1) * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dProbN, prob_nd.data(), size_t(nprob) * 8, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaMemcpyAsync(c->dW, w.data(), size_t(c->m) * 4, cudaMemcpyHostToDevice, c->stream));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  c->solved = false;
  return LP_OK;
}

size_t lp::estimate_bytes(int sms, int m, const int64_t* rows, int64_t d, int64_t pitch_unused, lp_dtype dtype,
                          int k, lp_ptr_space space) {
  (void)pitch_unused;
  auto r256 = [](size_t b) -> size_t { return ((b ? b : 16) + 255) / 256 * 256; };
  int64_t n = 0, smax = 0;
  for (int i = 0; i < m; ++i) {
    n += rows[i];
    smax = std::max(smax, rows[i]);
  }
  const size_t eb = plane_bytes(dtype);
  const int planes = dtype == LP_F32_BF16X2 ? 2 : 1;
  const int64_t per16 = 16 / static_cast<int64_t>(eb);
  const size_t ld = size_t((d + per16 - 1) / per16 * per16);
  const size_t K = size_t(kcap_of(k)), D = size_t(d), M = size_t(m);
  size_t tot = r256(size_t(n) * ld * eb * planes);
  if (dtype == LP_FP8_E4M3) tot += r256(size_t(n) * 4);
  // segment tables of the three step kernels, weights
  const size_t segs_max = size_t(max_segments(sms, m, n));
  tot += 3 * (r256(segs_max * sizeof(Segment)) + r256((size_t(sms) + 1) * 4) + r256((M + 1) * 4)) + 2 * r256(M * 4);
  // solve state
  tot += r256(segs_max * D * K * 4) + 2 * r256(M * D * K * 4) + 3 * r256(D * K * 4) + r256(M * K * K * 4) +
         r256(D * LP_MAX_K * 8) + r256(LP_MAX_K * 8) + r256(M * D * K * 8) + r256(16);
  if (dtype == LP_F32_BF16X2 && space == LP_HOST) {
    const int64_t chunk_rows = std::max<int64_t>(1, (int64_t(1) << 24) / d);
    tot += r256(size_t(std::min(chunk_rows, smax)) * D * 4);  // load staging
  }
  return tot + (tot >> 6) + (1u << 20);  // slack for rounding
}

int lp::solve_state(lp_ctx* c) {
  if (!c || !c->solved) return -1;
  const cudaError_t e = cudaEventQuery(c->ev1);
  if (e == cudaSuccess) return 1;
  if (e == cudaErrorNotReady) return 0;
  (void)cudaGetLastError();
  return -1;
}

extern "C" {

// Widest d for which lp_eta forms the d x d matrices (its Lanczos vectors live in shared memory).
static constexpr int kEtaMaxD = 16384;

static lp_status validate_k(lp_ctx* c, int k) {
  if (c->m == 0) return fail(c, LP_ERR_STATE, "no partitions loaded");
  if (k < 1 || k > LP_MAX_K) return fail(c, LP_ERR_INVALID, "k must be in [1, 32]");
  if (k > c->d) return fail(c, LP_ERR_INVALID, "k exceeds d");
  const int64_t smin = *std::min_element(c->rows.begin(), c->rows.end());
  if (k > smin)
    return fail(c, LP_ERR_INVALID, "k exceeds the smallest partition's row count (its local Y_i would be rank deficient)");
  const int K = kcap_of(k);
  if (c->planes == 0 && c->dtype != LP_FP8_E4M3 && simt_launches(static_cast<int>(c->d), c->ld, c->dtype, K) == 0)
    return fail(c, LP_ERR_UNSUPPORTED, "no step kernel for d=" + std::to_string(c->d) + ", k=" + std::to_string(k));
  return LP_OK;
}

// Plans the streaming tensor-core step for k (once per padded k) and makes the
// device segment table match its cluster count.  LP_ERR_UNSUPPORTED when the
// shape has no streaming kernel.
static lp_status ensure_tcs(lp_ctx* c, int k) {
  const int K = kcap_of(k);
  const int idx = K == 8 ? 0 : (K == 16 ? 1 : 2);
  if (c->tcs_state[idx] == 0) {
    lp::TcsPlan& p = c->tcs[idx];
    c->tcs_state[idx] = -1;
    p = lp::TcsPlan{};
    bool planned = false;
    if (c->dtype == LP_FP8_E4M3) {  // one kernel reads FP8 codes on the tensor cores
      if (c->tuning.kernel == LP_KERNEL_PAIR)
        return fail(c, LP_ERR_UNSUPPORTED, "the pair kernel does not read FP8 codes");
      planned = lp::tcs8_plan(static_cast<int>(c->d), K, c->sms, c->tuning, &p);
      if (!planned)
        return fail(c, LP_ERR_UNSUPPORTED, "no FP8 tensor-core plan for d=" + std::to_string(c->d));
      LP_CUDA(lp::tcs8_encode_map(c->dA, c->n, static_cast<int>(c->d), c->ld, &p));
    } else {
      const int want = c->tuning.kernel == LP_KERNEL_DEFAULT ? kDefaultTcKernel : c->tuning.kernel;
      if (want == LP_KERNEL_PAIR)
        planned = lp::pair_plan(static_cast<int>(c->d), K, c->planes, c->sms, c->tuning, &p);
      if (!planned && c->tuning.kernel != LP_KERNEL_PAIR) {
        p = lp::TcsPlan{};
        planned = lp::tcs_plan(static_cast<int>(c->d), K, c->planes, c->sms, c->tuning, &p);
      }
      if (!planned)
        return fail(c, LP_ERR_UNSUPPORTED, "no streaming tensor-core plan for d=" + std::to_string(c->d));
      const uint16_t* hi = static_cast<const uint16_t*>(c->dA);
      const uint16_t* lo = c->planes == 2 ? hi + size_t(c->n) * c->ld : nullptr;
      LP_CUDA(lp::tcs_encode_maps(hi, lo, c->n, static_cast<int>(c->d), c->ld, &p, p.pair != 0));
    }
    c->tcs_state[idx] = 1;
  }
  if (c->tcs_state[idx] < 0)
    return fail(c, LP_ERR_UNSUPPORTED, "no streaming tensor-core plan for d=" + std::to_string(c->d));
  lp::TcsPlan& p = c->tcs[idx];
  // Whole 128-row tiles per cluster: no more clusters than tiles.
  const int G = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(p.nclusters, (c->n + 127) / 128)));
  p.nclusters = G;
  if (G != c->tcs_G) {
    std::vector<Segment> segs;
    std::vector<int> seg_ptr, slot_begin;
    build_segments(c, G, segs, seg_ptr, slot_begin, kTcChainRows);
    lp_status st;
    if (!c->dSegsTcs &&
        ((st = dalloc(c, &c->dSegsTcs, size_t(max_segments(c->sms, c->m, c->n)) * sizeof(Segment))) ||
         (st = dalloc(c, &c->dSegPtrTcs, (size_t(c->sms) + 1) * 4)) ||
         (st = dalloc(c, &c->dSlotBeginTcs, (size_t(c->m) + 1) * 4))))
      return st;
    LP_CUDA(cudaMemcpyAsync(c->dSegsTcs, segs.data(), segs.size() * sizeof(Segment), cudaMemcpyHostToDevice,
                            c->stream));
    LP_CUDA(cudaMemcpyAsync(c->dSegPtrTcs, seg_ptr.data(), seg_ptr.size() * 4, cudaMemcpyHostToDevice, c->stream));
    LP_CUDA(cudaMemcpyAsync(c->dSlotBeginTcs, slot_begin.data(), slot_begin.size() * 4, cudaMemcpyHostToDevice,
                            c->stream));
    // pageable sources: make sure the copies have read them before the vectors go
    LP_CUDA(cudaStreamSynchronize(c->stream));
    c->nslots_tcs = static_cast<int>(segs.size());
    c->max_slots[PATH_TCS] = max_slots_in(slot_begin);
    c->tcs_G = G;
  }
  c->tcs_cur = &p;
  return LP_OK;
}

// Picks the step kernel.  BF16 and split-plane data run on the tensor cores:
// the streaming kernel unless LP_FLAG_TC_RESIDENT asks for the resident one
// (BF16) or the shape has no streaming plan; LP_FLAG_SIMT (BF16 only) and the
// other dtypes use the SIMT FP32 kernel.
static lp_status select_path(lp_ctx* c, int k, unsigned flags) {
  c->path = PATH_SIMT;
  if (c->dtype == LP_FP8_E4M3 && !(flags & LP_FLAG_SIMT)) {
    const lp_status st = ensure_tcs(c, k);
    if (st == LP_OK) c->path = PATH_TCS;
    else if (st != LP_ERR_UNSUPPORTED || c->tuning.kernel != LP_KERNEL_DEFAULT) return st;
    c->err.clear();
  }
  if (c->planes > 0 && !(flags & LP_FLAG_SIMT)) {
    const bool resident = ((flags & LP_FLAG_TC_RESIDENT) || c->prefer_resident) && c->dtype == LP_BF16;
    if (!resident) {
      const lp_status st = ensure_tcs(c, k);
      if (st == LP_OK) c->path = PATH_TCS;
      else if (st != LP_ERR_UNSUPPORTED || c->tuning.kernel != LP_KERNEL_DEFAULT) return st;  // no silent substitute
      c->err.clear();
    }
    if (c->path == PATH_SIMT && c->dtype == LP_BF16 && c->tc_ready) {
      lp::TcPlan p;
      if (lp::tc_plan(static_cast<int>(c->d), k, c->sms, &p) && p.cluster == c->tc.cluster && p.nch == c->tc.nch) {
        c->tc.K = p.K;
        c->tc.smem = p.smem;
        c->path = PATH_TC;
      }
    }
  }
  if (c->path == PATH_SIMT) {
    if (c->dtype == LP_F32_BF16X2)
      return fail(c, LP_ERR_UNSUPPORTED,
                  "split-plane data run only on the streaming tensor-core kernel, which has no plan for d=" +
                      std::to_string(c->d) + ", k=" + std::to_string(k));
    if (simt_launches(static_cast<int>(c->d), c->ld, c->dtype, kcap_of(k)) == 0)
      return fail(c, LP_ERR_UNSUPPORTED,
                  "no step kernel for d=" + std::to_string(c->d) + ", k=" + std::to_string(k) + " on this path");
  }
  return LP_OK;
}

// The launch sequence of one solve (Alg. 1 in rounds, then Ritz or unpack), on
// the context's stream; lp_solve runs it eagerly or captures it into a graph.
static lp_status solve_body(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, int refine_rounds,
                            bool timing, const double* dy0, bool trace, bool kxk64) {
  const int d = static_cast<int>(c->d);
  const int m = c->m;
  const int K = kcap_of(k);
  // Several problems (a batch group): one start block, aggregate, orth and result
  // per problem; each partition multiplies its own problem's basis at the start
  // of a round and aligns with its own problem's base partition.
  const int NP = c->nprob;
  const bool multi = NP > 1;
  lp_status st;
  LP_CUDA(cudaMemsetAsync(c->dStatus, 0, 4, c->stream));
  if ((st = check_launch(c, lp::launch_pack(dy0, c->dY, NP, d, k, K, c->stream), "pack"))) return st;
  if ((st = check_launch(c, lp::launch_cholqr2(c->dY, c->dZ, NP, d, k, K, c->dStatus, c->stream, kxk64), "orth")))
    return st;

  const int rounds = T + refine_rounds;
  const int64_t zs = int64_t(d) * K;
  // the first step of a round: the shared basis, or each partition's copy of its problem's
  auto first_step = [&]() -> lp_status {
    if (!multi) return launch_step(c, K, c->dZ, 0, timing);
    lp_status s2 = check_launch(c, lp::launch_broadcast(c->dZ, c->dPartProb, m, d, K, c->dZl, c->stream), "broadcast");
    return s2 ? s2 : launch_step(c, K, c->dZl, zs, timing);
  };
  for (int t = 0; t < rounds; ++t) {
    const int p = t < T ? p_schedule[t] : 1;
    for (int j = 0; j < p; ++j) {
      if (j > 0 && (st = check_launch(c, lp::launch_cholqr2(c->dYl, c->dZl, m, d, k, K, c->dStatus, c->stream, kxk64),
                                      "local orth")))
        return st;
      if ((st = j == 0 ? first_step() : launch_step(c, K, c->dZl, zs, timing))) return st;
      if ((st = check_launch(c, lp::launch_reduce(c->dP, slot_begin_of(c), c->dInvS, m, d, K, c->dYl, c->stream,
                                                  c->max_slots[c->path]),
                             "reduce")))
        return st;
      c->stats.local_steps++;
    }
    const bool align = p > 1 && agg != LP_AGG_IDENTITY;
    if (align) {
      // The last basis each partition multiplied this round is Z_i (orth of its previous Y_i).
      if ((st = check_launch(c, lp::launch_align(c->dZl, zs, c->dZl + zs * c->base, m, d, k, K, c->base, agg, c->dG,
                                                 c->dStatus, c->stream, kxk64, multi ? c->dPartBase : nullptr),
                             "align")))
        return st;
    }
    if ((st = check_launch(c, lp::launch_aggregate(c->dYl, c->dW, align ? c->dG : nullptr, agg == LP_AGG_SIGN ? 1 : 0,
                                                   m, d, K, c->dY, c->stream, multi ? c->dProbBegin : nullptr, NP),
                           "aggregate")))
      return st;
    if ((st = check_launch(c, lp::launch_cholqr2(c->dY, c->dZ, NP, d, k, K, c->dStatus, c->stream, kxk64), "orth")))
      return st;
    if (trace) {
      LP_CUDA(cudaMemcpyAsync(c->dTraceZ + size_t(t) * d * K, c->dZ, size_t(d) * K * 4, cudaMemcpyDeviceToDevice,
                              c->stream));
      double* rho = c->dTraceRho + size_t(t) * m;
      if (p == 1) {
        LP_CUDA(cudaMemsetAsync(rho, 0, size_t(m) * 8, c->stream));
      } else if ((st = check_launch(c, lp::launch_rho(c->dZl, zs, c->dZl + zs * c->base, align ? c->dG : nullptr,
                                                      agg == LP_AGG_SIGN ? 1 : 0, c->base, m, d, k, K, rho,
                                                      c->dStatus, c->stream),
                                    "residual error"))) {
        return st;
      }
    }
    c->stats.rounds++;
  }
  if (c->ritz) {
    if ((st = first_step())) return st;
    if ((st = check_launch(c, lp::launch_reduce(c->dP, slot_begin_of(c), c->dInvS, m, d, K, c->dYl, c->stream, c->max_slots[c->path]), "reduce")))
      return st;
    if ((st = check_launch(c, lp::launch_aggregate(c->dYl, c->dW, nullptr, 0, m, d, K, c->dMZ, c->stream,
                                                   multi ? c->dProbBegin : nullptr, NP),
                           "aggregate")))
      return st;
    // the partials buffer is free again after the reduction: it holds the Ritz scratch,
    // for all problems at once when it is large enough, else for one after another
    const size_t P_bytes = state_sizes(c, K).P;
    if (lp::ritz_scratch_bytes(d, K) > P_bytes) return fail(c, LP_ERR_INVALID, "Ritz scratch too small");
    if (lp::ritz_scratch_bytes(d, K, NP) <= P_bytes) {
      if ((st = check_launch(c, lp::launch_ritz(c->dZ, c->dMZ, d, k, K, double(c->prob_n[0]), c->dZout, c->dSigma,
                                                reinterpret_cast<double*>(c->dP), c->dStatus, c->stream, kxk64, NP,
                                                multi ? c->dProbN : nullptr),
                             "ritz")))
        return st;
      c->stats.kernel_launches += 2;  // launch_ritz runs three kernels
    } else {
      for (int q = 0; q < NP; ++q) {
        if ((st = check_launch(c, lp::launch_ritz(c->dZ + q * zs, c->dMZ + q * zs, d, k, K, double(c->prob_n[q]),
                                                  c->dZout + size_t(q) * d * k, c->dSigma + size_t(q) * LP_MAX_K,
                                                  reinterpret_cast<double*>(c->dP), c->dStatus, c->stream, kxk64),
                               "ritz")))
          return st;
        c->stats.kernel_launches += 2;
      }
    }
  } else {
    if ((st = check_launch(c, lp::launch_unpack(c->dZ, c->dZout, NP, d, k, K, c->stream), "unpack"))) return st;
  }
  return LP_OK;
}

lp_status lp_set_tuning(lp_ctx* c, const lp_tuning* t) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  lp::TcsTuning nt;
  if (t) {
    if (t->ring_units < 0 || t->lag_units < 0 || t->prefetch_units < 0 || t->cache_hints < 0 || t->slice_cols < 0 ||
        (t->slice_cols != 0 && t->slice_cols % 128 != 0) || t->kernel < 0 || t->kernel > LP_KERNEL_PAIR ||
        t->test_stall_cycles < 0)
      return fail(c, LP_ERR_INVALID,
                  "tuning fields must be >= 0, slice_cols a multiple of 128, kernel one of LP_KERNEL_*");
    nt.ring_units = t->ring_units;
    nt.lag_units = t->lag_units;
    nt.prefetch_units = t->prefetch_units;
    nt.cache_hints = t->cache_hints;
    nt.slice_cols = t->slice_cols;
    nt.kernel = t->kernel;
    nt.test_stall_cycles = t->test_stall_cycles;
  }
  c->tuning = nt;
  c->prefer_resident = false;
  drop_graph(c);
  // plans are rebuilt on the next solve; the segment table is kept (same cluster count or rebuilt then)
  c->tcs_state[0] = c->tcs_state[1] = c->tcs_state[2] = 0;
  c->tcs_cur = nullptr;
  return LP_OK;
}

lp_status lp_autotune(lp_ctx* c, int k, lp_tuning* chosen, int* path_out, double* best_ms) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  lp_status st = validate_k(c, k);
  if (st) return st;
  LP_CUDA(cudaSetDevice(c->device));
  const int K = kcap_of(k);
  if ((st = ensure_state(c, K))) return st;
  struct Cand {
    lp::TcsTuning t;
    bool resident;
  };
  std::vector<Cand> cands;
  if (c->dtype == LP_FP8_E4M3) {
    for (int slice : {0, 256})
      for (int lag : {2, 4}) {
        Cand cd;
        cd.t.kernel = LP_KERNEL_STREAM;
        cd.t.lag_units = lag;
        cd.t.slice_cols = slice;
        cd.resident = false;
        cands.push_back(cd);
      }
  }
  if (c->planes > 0) {
    {
      Cand cd;
      cd.t.kernel = LP_KERNEL_PAIR;
      cd.resident = false;
      cands.push_back(cd);
    }
    for (int slice : {0, 512})
      for (int lag : {1, 2, 4})
        for (int hint : {0, 1}) {
          Cand cd;
          cd.t.kernel = LP_KERNEL_STREAM;
          cd.t.lag_units = lag;
          cd.t.cache_hints = hint;
          cd.t.slice_cols = slice;
          cd.resident = false;
          cands.push_back(cd);
        }
    if (c->dtype == LP_BF16 && c->tc_ready) cands.push_back(Cand{lp::TcsTuning{}, true});
  }
  const lp::TcsTuning saved = c->tuning;
  const bool saved_res = c->prefer_resident;
  double best = -1.0;
  Cand win{saved, saved_res};
  int win_path = PATH_SIMT;
  if (!cands.empty()) {
    LP_CUDA(cudaMemsetAsync(c->dZ, 0, size_t(c->d) * K * 4, c->stream));
    for (const Cand& cd : cands) {
      c->tuning = cd.t;
      c->prefer_resident = cd.resident;
      c->tcs_state[0] = c->tcs_state[1] = c->tcs_state[2] = 0;
      if ((st = select_path(c, k, 0))) {
        if (st == LP_ERR_UNSUPPORTED) continue;
        break;
      }
      if ((st = launch_step(c, K, c->dZ, 0, false))) break;
      LP_CUDA(cudaEventRecord(c->ev0, c->stream));
      for (int r = 0; r < 3 && !st; ++r) st = launch_step(c, K, c->dZ, 0, false);
      if (st) break;
      LP_CUDA(cudaEventRecord(c->ev1, c->stream));
      LP_CUDA(cudaEventSynchronize(c->ev1));
      float ms = 0.f;
      LP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
      const double per = ms / 3.0;
      if (best < 0 || per < best) {
        best = per;
        win = cd;
        win_path = reported_path(c);
      }
    }
  } else {
    if ((st = select_path(c, k, 0))) return st;
    win_path = reported_path(c);
  }
  c->tuning = win.t;
  c->prefer_resident = win.resident;
  drop_graph(c);
  c->tcs_state[0] = c->tcs_state[1] = c->tcs_state[2] = 0;
  c->solved = false;  // the timing launches overwrote the solve buffers
  if (st) return st;
  if (chosen) {
    chosen->ring_units = win.t.ring_units;
    chosen->lag_units = win.t.lag_units;
    chosen->prefetch_units = win.t.prefetch_units;
    chosen->cache_hints = win.t.cache_hints;
    chosen->slice_cols = win.t.slice_cols;
    chosen->kernel = win.t.kernel;
    chosen->test_stall_cycles = 0;
  }
  if (path_out) *path_out = win_path;
  if (best_ms) *best_ms = best;
  return LP_OK;
}

// Checks, kernel choice and device state of a solve; uploads y0 to the staging
// buffer (pageable host memory: never inside a captured graph).
static lp_status solve_prepare(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, const double* y0,
                               int refine_rounds, unsigned flags, bool record_start, const double** dy0) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  lp_status st = validate_k(c, k);
  if (st) return st;
  if (T < 0 || refine_rounds < 0 || T + refine_rounds < 1)
    return fail(c, LP_ERR_INVALID, "need T >= 0, refine_rounds >= 0 and at least one round");
  if (T > 0 && !p_schedule) return fail(c, LP_ERR_INVALID, "p_schedule is NULL");
  for (int t = 0; t < T; ++t)
    if (p_schedule[t] < 1) return fail(c, LP_ERR_INVALID, "p_schedule entries must be >= 1");
  if (agg != LP_AGG_IDENTITY && agg != LP_AGG_SIGN && agg != LP_AGG_OPT)
    return fail(c, LP_ERR_INVALID, "unknown aggregator");
  if (!y0) return fail(c, LP_ERR_INVALID, "y0 is NULL");
  LP_CUDA(cudaSetDevice(c->device));
  const int K = kcap_of(k);
  if ((st = select_path(c, k, flags))) return st;
  if ((st = ensure_state(c, K))) return st;
  c->traced_rounds = 0;
  if ((flags & LP_FLAG_TRACE) && c->nprob > 1)
    return fail(c, LP_ERR_INVALID, "LP_FLAG_TRACE records one problem per context");
  if (flags & LP_FLAG_TRACE) {
    const int rounds = T + refine_rounds;
    const size_t zb = size_t(rounds) * c->d * K * 4, rb = size_t(rounds) * c->m * 8;
    if (zb > c->trace_z_bytes || rb > c->trace_rho_bytes) {
      drop_graph(c);  // the captured sequence names the old buffers
      dfree(c, c->dTraceZ, c->trace_z_bytes);
      dfree(c, c->dTraceRho, c->trace_rho_bytes);
      c->trace_z_bytes = c->trace_rho_bytes = 0;
      if ((st = dalloc(c, &c->dTraceZ, zb)) || (st = dalloc(c, &c->dTraceRho, rb))) return st;
      c->trace_z_bytes = zb;
      c->trace_rho_bytes = rb;
    }
  }
  c->solved = false;
  c->k = k;
  c->ritz = (flags & LP_FLAG_RITZ) != 0;
  if (record_start) LP_CUDA(cudaEventRecord(c->ev0, c->stream));
  return stage_in(c, y0, size_t(c->nprob) * c->d * k, LP_HOST, dy0);  // one start block per problem
}

static void solve_mark(lp_ctx* c, int k, int rounds, unsigned flags) {
  c->traced_rounds = (flags & LP_FLAG_TRACE) ? rounds : 0;
  c->stats.k = k;
  c->stats.n = c->n;
  c->stats.d = c->d;
  c->stats.m = c->m;
  c->stats.path = reported_path(c);
  c->solved = true;
}

// Y_0 for lp_solve_seeded: N(0,1) entries from a counter-based generator,
// SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
// generators", OOPSLA 2014) on counters seed + (c + 1) * golden gamma, the top 53
// bits as a uniform in [0, 1), and the Box-Muller transform on consecutive pairs
// (counters 2q and 2q + 1 give entries 2q (cosine) and 2q + 1 (sine) of the
// row-major d x k block).
static uint64_t splitmix64_at(uint64_t seed, uint64_t counter) {
  uint64_t z = seed + (counter + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static void draw_start(uint64_t seed, size_t count, std::vector<double>& y) {
  y.resize(count);
  const double two_pi = 6.283185307179586476925286766559;
  for (size_t q = 0; 2 * q < count; ++q) {
    const double u1 = static_cast<double>(splitmix64_at(seed, 2 * q) >> 11) * 0x1.0p-53;
    const double u2 = static_cast<double>(splitmix64_at(seed, 2 * q + 1) >> 11) * 0x1.0p-53;
    const double r = std::sqrt(-2.0 * std::log1p(-u1));  // 1 - u1 lies in (0, 1]
    y[2 * q] = r * std::cos(two_pi * u2);
    if (2 * q + 1 < count) y[2 * q + 1] = r * std::sin(two_pi * u2);
  }
}

lp_status lp_solve_seeded(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, uint64_t seed,
                          int refine_rounds, unsigned flags) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (c->m == 0) return fail(c, LP_ERR_STATE, "no partitions loaded");
  if (k < 1 || k > LP_MAX_K) return fail(c, LP_ERR_INVALID, "k must be in [1, 32]");
  std::vector<double> y0;
  draw_start(seed, size_t(c->d) * size_t(k), y0);
  return lp_solve(c, k, p_schedule, T, agg, y0.data(), refine_rounds, flags);
}

lp_status lp_solve(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, const double* y0,
                   int refine_rounds, unsigned flags) {
  const double* dy0 = nullptr;
  lp_status st = solve_prepare(c, k, p_schedule, T, agg, y0, refine_rounds, flags, true, &dy0);
  if (st) return st;
  const bool timing = (flags & LP_FLAG_TIMING) != 0;
  // The launch sequence depends only on these; a matching key replays the captured graph.
  std::vector<int64_t> key = {int64_t(c->gen), k, T, int64_t(agg), refine_rounds, int64_t(flags), c->path};
  key.insert(key.end(), p_schedule, p_schedule + T);
  const bool use_graph = (flags & LP_FLAG_NO_GRAPH) == 0;
  if (use_graph && c->graph_exec && key == c->graph_key) {
    LP_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
    c->stats = c->graph_stats;
    c->step_ev_used = c->graph_step_ev_used;
  } else {
    if (use_graph) {
      drop_graph(c);
      key[0] = int64_t(c->gen);
      LP_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeRelaxed));
    }
    std::memset(&c->stats, 0, sizeof(c->stats));
    c->step_ev_used = 0;
    st = solve_body(c, k, p_schedule, T, agg, refine_rounds, timing, dy0, (flags & LP_FLAG_TRACE) != 0,
                    (flags & LP_FLAG_KXK_FP64) != 0);
    if (use_graph) {
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->stream, &g);
      if (st) {
        if (g) cudaGraphDestroy(g);
        return st;
      }
      if (e != cudaSuccess) return cuda_fail(c, e, "capturing the solve");
      const cudaError_t ei = cudaGraphInstantiate(&c->graph_exec, g, 0);
      cudaGraphDestroy(g);
      if (ei != cudaSuccess) {
        c->graph_exec = nullptr;
        return cuda_fail(c, ei, "instantiating the solve graph");
      }
      c->graph_key = key;
      c->graph_stats = c->stats;
      c->graph_step_ev_used = c->step_ev_used;
      LP_CUDA(cudaGraphLaunch(c->graph_exec, c->stream));
    } else if (st) {
      return st;
    }
  }
  LP_CUDA(cudaEventRecord(c->ev1, c->stream));
  solve_mark(c, k, T + refine_rounds, flags);
  return LP_OK;
}

lp_status lp_trace(lp_ctx* c, double* z_trace, double* rho) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (!c->solved || c->traced_rounds == 0) return fail(c, LP_ERR_STATE, "no traced solve (LP_FLAG_TRACE)");
  LP_CUDA(cudaSetDevice(c->device));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  const int R = c->traced_rounds, K = kcap_of(c->k), d = static_cast<int>(c->d), k = c->k;
  if (z_trace) {
    std::vector<float> h(size_t(R) * d * K);
    LP_CUDA(cudaMemcpy(h.data(), c->dTraceZ, h.size() * 4, cudaMemcpyDeviceToHost));
    for (int t = 0; t < R; ++t)
      for (int r = 0; r < d; ++r)
        for (int j = 0; j < k; ++j) z_trace[(size_t(t) * d + r) * k + j] = h[(size_t(t) * d + r) * K + j];
  }
  if (rho) {
    std::vector<double> h(size_t(R) * c->m);
    LP_CUDA(cudaMemcpy(h.data(), c->dTraceRho, h.size() * 8, cudaMemcpyDeviceToHost));
    for (int t = 0; t < R; ++t) rho[t] = *std::max_element(h.begin() + size_t(t) * c->m, h.begin() + size_t(t + 1) * c->m);
  }
  return LP_OK;
}

lp_status lp_result(lp_ctx* c, double* z_out, double* sigma_out, lp_stats* stats) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (!c->solved) return fail(c, LP_ERR_STATE, "no solve to report");
  LP_CUDA(cudaSetDevice(c->device));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  int status = 0;
  LP_CUDA(cudaMemcpy(&status, c->dStatus, 4, cudaMemcpyDeviceToHost));
  float ms = 0.f;
  LP_CUDA(cudaEventElapsedTime(&ms, c->ev0, c->ev1));
  c->stats.ms_solve = ms;
  double step_ms = 0.0;
  for (int e = 0; e + 1 < c->step_ev_used; e += 2) {
    float x = 0.f;
    LP_CUDA(cudaEventElapsedTime(&x, c->step_ev[e], c->step_ev[e + 1]));
    step_ms += x;
  }
  c->stats.ms_step_kernels = step_ms;
  if (z_out)
    LP_CUDA(cudaMemcpy(z_out, c->dZout, size_t(c->d) * c->k * 8, cudaMemcpyDeviceToHost));
  if (sigma_out) {
    if (c->ritz) LP_CUDA(cudaMemcpy(sigma_out, c->dSigma, size_t(c->k) * 8, cudaMemcpyDeviceToHost));
    else std::memset(sigma_out, 0, size_t(c->k) * 8);
  }
  if (stats) *stats = c->stats;
  if (status & lp::ST_TIMEOUT)  // first: a wait that gave up leaves the later steps garbage
    return fail(c, LP_ERR_TIMEOUT, "device wait timed out");
  if (status & lp::ST_CHOL) return fail(c, LP_ERR_NUMERIC, "Cholesky breakdown (non-positive or non-finite pivot)");
  if (status & lp::ST_NONFINITE) return fail(c, LP_ERR_NUMERIC, "non-finite iterate");
  if (status & lp::ST_JACOBI) return fail(c, LP_ERR_NUMERIC, "Jacobi iteration did not converge or singular block");
  return LP_OK;
}

lp_status lp_power_step(lp_ctx* c, int k, const double* z, int z_shared, double* y_out, lp_ptr_space space) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  lp_status st = validate_k(c, k);
  if (st) return st;
  if (!z || !y_out) return fail(c, LP_ERR_INVALID, "z and y_out must be non-NULL");
  LP_CUDA(cudaSetDevice(c->device));
  const int K = kcap_of(k);
  if ((st = select_path(c, k, 0))) return st;
  if ((st = ensure_state(c, K))) return st;
  LP_CUDA(cudaMemsetAsync(c->dStatus, 0, 4, c->stream));
  const int d = static_cast<int>(c->d);
  const int nb = z_shared ? 1 : c->m;
  const double* dz;
  if ((st = stage_in(c, z, size_t(nb) * d * k, space, &dz))) return st;
  float* Zt = z_shared ? c->dZ : c->dZl;
  if ((st = check_launch(c, lp::launch_pack(dz, Zt, nb, d, k, K, c->stream), "pack"))) return st;
  if ((st = launch_step(c, K, Zt, z_shared ? 0 : int64_t(d) * K, false))) return st;
  if ((st = check_launch(c, lp::launch_reduce(c->dP, slot_begin_of(c), c->dInvS, c->m, d, K, c->dYl, c->stream, c->max_slots[c->path]),
                         "reduce")))
    return st;
  double* dst = space == LP_DEVICE ? y_out : c->dStage;
  if ((st = check_launch(c, lp::launch_unpack(c->dYl, dst, c->m, d, k, K, c->stream), "unpack"))) return st;
  if (space == LP_HOST)
    LP_CUDA(cudaMemcpyAsync(y_out, dst, size_t(c->m) * d * k * 8, cudaMemcpyDeviceToHost, c->stream));
  int status = 0;
  LP_CUDA(cudaMemcpyAsync(&status, c->dStatus, 4, cudaMemcpyDeviceToHost, c->stream));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  if (status & lp::ST_TIMEOUT) return fail(c, LP_ERR_TIMEOUT, "device wait timed out in the power step");
  return LP_OK;
}

lp_status lp_eta(lp_ctx* c, double* eta, double* norms) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (c->m == 0) return fail(c, LP_ERR_STATE, "no partitions loaded");
  if (!eta) return fail(c, LP_ERR_INVALID, "eta must be non-NULL");
  const int d = static_cast<int>(c->d), m = c->m;
  if (d > kEtaMaxD) return fail(c, LP_ERR_UNSUPPORTED, "eta is computed for d <= " + std::to_string(kEtaMaxD));
  LP_CUDA(cudaSetDevice(c->device));
  // kb identity columns per step, in the padded width the context already has
  // (growing the state would free the last solve's result); no
  // orthonormalisation follows, so partitions with fewer rows than kb are fine.
  const int K = c->Kcap > 0 ? c->Kcap : kcap_of(std::min(16, d));
  const int kb = std::min(K, d);
  if (c->planes == 0 && c->dtype != LP_FP8_E4M3 && simt_launches(d, c->ld, c->dtype, K) == 0)
    return fail(c, LP_ERR_UNSUPPORTED, "no step kernel for d=" + std::to_string(d));
  lp_status st;
  if ((st = select_path(c, kb, 0))) return st;
  if ((st = ensure_state(c, K))) return st;
  // the last solve's statistics and status word stay as they were
  const lp_stats saved = c->stats;
  int saved_status = 0;
  LP_CUDA(cudaMemcpyAsync(&saved_status, c->dStatus, 4, cudaMemcpyDeviceToHost, c->stream));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  LP_CUDA(cudaMemsetAsync(c->dStatus, 0, 4, c->stream));
  const size_t dd = size_t(d) * d;
  const size_t mat_bytes = (size_t(m) + 1) * dd * 4;
  const size_t v_bytes = (size_t(m) + 1) * lp::lanczos_steps(d) * size_t(d) * 4;
  const size_t out_bytes = (size_t(m) + 1) * 8;
  float* dM = nullptr;
  float* dV = nullptr;
  double* dOut = nullptr;
  auto release = [&]() {
    dfree(c, dM, mat_bytes);
    dfree(c, dV, v_bytes);
    dfree(c, dOut, out_bytes);
    c->stats = saved;
  };
  if ((st = dalloc(c, &dM, mat_bytes)) || (st = dalloc(c, &dV, v_bytes)) || (st = dalloc(c, &dOut, out_bytes))) {
    release();
    return st;
  }
  std::vector<double> out(size_t(m) + 1, 0.0);
  int status = 0;
  auto run = [&]() -> lp_status {
    lp_status s2;
    for (int c0 = 0; c0 < d; c0 += kb) {
      if ((s2 = check_launch(c, lp::launch_identity_block(c->dZ, d, K, c0, c->stream), "identity block"))) return s2;
      if ((s2 = launch_step(c, K, c->dZ, 0, false))) return s2;
      if ((s2 = check_launch(c, lp::launch_reduce(c->dP, slot_begin_of(c), c->dInvS, m, d, K, c->dYl, c->stream, c->max_slots[c->path]),
                             "reduce")))
        return s2;
      if ((s2 = check_launch(
               c, lp::launch_scatter_columns(c->dYl, dM, m, d, K, c0, std::min(kb, d - c0), c->stream), "scatter")))
        return s2;
    }
    if ((s2 = check_launch(c, lp::launch_deviations(dM, c->dW, m, d, c->stream), "deviations"))) return s2;
    if ((s2 = check_launch(c, lp::launch_lanczos_norms(dM, m + 1, d, dV, dOut, c->stream), "lanczos"))) return s2;
    LP_CUDA(cudaMemcpyAsync(out.data(), dOut, out_bytes, cudaMemcpyDeviceToHost, c->stream));
    LP_CUDA(cudaMemcpyAsync(&status, c->dStatus, 4, cudaMemcpyDeviceToHost, c->stream));
    LP_CUDA(cudaStreamSynchronize(c->stream));
    LP_CUDA(cudaMemcpyAsync(c->dStatus, &saved_status, 4, cudaMemcpyHostToDevice, c->stream));
    LP_CUDA(cudaStreamSynchronize(c->stream));
    return LP_OK;
  };
  st = run();
  release();
  if (st) return st;
  if (status & lp::ST_TIMEOUT)  // first: a wait that gave up leaves the later steps garbage
    return fail(c, LP_ERR_TIMEOUT, "device wait timed out");
  double worst = 0.0;
  for (int i = 0; i <= m; ++i)
    if (!std::isfinite(out[i])) return fail(c, LP_ERR_NUMERIC, "non-finite matrix norm");
  for (int i = 0; i < m; ++i) worst = std::max(worst, out[i]);
  if (!(out[m] > 0.0)) return fail(c, LP_ERR_NUMERIC, "M is zero");
  *eta = worst / out[m];
  if (norms) std::memcpy(norms, out.data(), out_bytes);
  return LP_OK;
}

}  // extern "C"

// Scratch-owning helper for the standalone small-kernel entry points.
namespace {
struct Scratch {
  lp_ctx* c;
  std::vector<std::pair<void*, size_t>> bufs;
  ~Scratch() {
    for (auto& b : bufs) {
      void* p = b.first;
      dfree(c, p, b.second);
    }
  }
  template <typename T>
  lp_status get(T** p, size_t bytes) {
    lp_status st = dalloc(c, p, bytes);
    if (!st) bufs.push_back({static_cast<void*>(*p), bytes});
    return st;
  }
};

lp_status to_device(lp_ctx* c, Scratch& s, const double* src, size_t count, lp_ptr_space space, const double** dev) {
  if (space == LP_DEVICE) {
    *dev = src;
    return LP_OK;
  }
  double* p;
  lp_status st = s.get(&p, count * 8);
  if (st) return st;
  LP_CUDA(cudaMemcpyAsync(p, src, count * 8, cudaMemcpyHostToDevice, c->stream));
  *dev = p;
  return LP_OK;
}
}  // namespace

extern "C" {

lp_status lp_orth(lp_ctx* c, int batch, int64_t d, int k, const double* y, double* z, lp_ptr_space space,
                  unsigned flags) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (batch < 1 || d < 1 || k < 1 || k > LP_MAX_K || k > d || !y || !z)
    return fail(c, LP_ERR_INVALID, "need batch >= 1, 1 <= k <= min(32, d), non-NULL y and z");
  LP_CUDA(cudaSetDevice(c->device));
  const int K = kcap_of(k);
  Scratch s{c, {}};
  lp_status st;
  const double* dy;
  float *Y, *Z;
  double* dz;
  const size_t blk = size_t(batch) * d;
  if ((st = to_device(c, s, y, blk * k, space, &dy)) || (st = s.get(&Y, blk * K * 4)) ||
      (st = s.get(&Z, blk * K * 4)))
    return st;
  if (space == LP_DEVICE) dz = z;
  else if ((st = s.get(&dz, blk * k * 8))) return st;
  LP_CUDA(cudaMemsetAsync(c->dStatus, 0, 4, c->stream));
  if ((st = check_launch(c, lp::launch_pack(dy, Y, batch, static_cast<int>(d), k, K, c->stream), "pack"))) return st;
  if ((st = check_launch(c, lp::launch_cholqr2(Y, Z, batch, static_cast<int>(d), k, K, c->dStatus, c->stream,
                                               (flags & LP_FLAG_KXK_FP64) != 0),
                         "orth")))
    return st;
  if ((st = check_launch(c, lp::launch_unpack(Z, dz, batch, static_cast<int>(d), k, K, c->stream), "unpack")))
    return st;
  if (space == LP_HOST) LP_CUDA(cudaMemcpyAsync(z, dz, blk * k * 8, cudaMemcpyDeviceToHost, c->stream));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  int status = 0;
  LP_CUDA(cudaMemcpy(&status, c->dStatus, 4, cudaMemcpyDeviceToHost));
  if (status & lp::ST_CHOL) return fail(c, LP_ERR_NUMERIC, "Cholesky breakdown in orth");
  return LP_OK;
}

lp_status lp_align_aggregate(lp_ctx* c, int m, int64_t d, int k, lp_aggregator agg, int base, const double* w,
                             const double* ys, const double* zs, double* y_out, double* d_out, lp_ptr_space space,
                             unsigned flags) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (m < 1 || d < 1 || k < 1 || k > LP_MAX_K || k > d || base < 0 || base >= m || !w || !ys || !zs || !y_out)
    return fail(c, LP_ERR_INVALID, "bad arguments to lp_align_aggregate");
  if (agg != LP_AGG_IDENTITY && agg != LP_AGG_SIGN && agg != LP_AGG_OPT)
    return fail(c, LP_ERR_INVALID, "unknown aggregator");
  LP_CUDA(cudaSetDevice(c->device));
  const int K = kcap_of(k);
  const int di = static_cast<int>(d);
  Scratch s{c, {}};
  lp_status st;
  const double *dys, *dzs, *dw;
  float *Yl, *Zl, *G, *Y, *W;
  double *dy, *dG;
  const size_t blk = size_t(m) * d;
  if ((st = to_device(c, s, ys, blk * k, space, &dys)) || (st = to_device(c, s, zs, blk * k, space, &dzs)) ||
      (st = to_device(c, s, w, m, space, &dw)) || (st = s.get(&Yl, blk * K * 4)) || (st = s.get(&Zl, blk * K * 4)) ||
      (st = s.get(&G, size_t(m) * K * K * 4)) || (st = s.get(&Y, size_t(d) * K * 4)) || (st = s.get(&W, m * 4)) ||
      (st = s.get(&dG, size_t(m) * k * k * 8)))
    return st;
  if (space == LP_DEVICE) dy = y_out;
  else if ((st = s.get(&dy, size_t(d) * k * 8))) return st;
  LP_CUDA(cudaMemsetAsync(c->dStatus, 0, 4, c->stream));
  if ((st = check_launch(c, lp::launch_pack(dys, Yl, m, di, k, K, c->stream), "pack")) ||
      (st = check_launch(c, lp::launch_pack(dzs, Zl, m, di, k, K, c->stream), "pack")) ||
      (st = check_launch(c, lp::launch_pack(dw, W, 1, m, 1, 1, c->stream), "pack")))
    return st;
  const bool align = agg != LP_AGG_IDENTITY;
  if (align && (st = check_launch(c, lp::launch_align(Zl, int64_t(d) * K, Zl + int64_t(d) * K * base, m, di, k, K, base,
                                                      agg, G, c->dStatus, c->stream,
                                                      (flags & LP_FLAG_KXK_FP64) != 0, nullptr),
                                  "align")))
    return st;
  if ((st = check_launch(c, lp::launch_aggregate(Yl, W, align ? G : nullptr, agg == LP_AGG_SIGN ? 1 : 0, m, di, K, Y,
                                                 c->stream, nullptr, 1),
                         "aggregate")))
    return st;
  if ((st = check_launch(c, lp::launch_unpack(Y, dy, 1, di, k, K, c->stream), "unpack"))) return st;
  if (space == LP_HOST) LP_CUDA(cudaMemcpyAsync(y_out, dy, size_t(d) * k * 8, cudaMemcpyDeviceToHost, c->stream));
  if (d_out) {
    // G_i (K x K float) -> k x k FP64; identity blocks when agg is identity.
    std::vector<float> hG(size_t(m) * K * K, 0.f);
    if (align) LP_CUDA(cudaMemcpyAsync(hG.data(), G, hG.size() * 4, cudaMemcpyDeviceToHost, c->stream));
    LP_CUDA(cudaStreamSynchronize(c->stream));
    std::vector<double> out(size_t(m) * k * k);
    for (int i = 0; i < m; ++i)
      for (int a = 0; a < k; ++a)
        for (int b = 0; b < k; ++b)
          out[(size_t(i) * k + a) * k + b] = align ? hG[(size_t(i) * K + a) * K + b] : (a == b ? 1.0 : 0.0);
    if (space == LP_DEVICE) LP_CUDA(cudaMemcpy(d_out, out.data(), out.size() * 8, cudaMemcpyHostToDevice));
    else std::memcpy(d_out, out.data(), out.size() * 8);
  }
  LP_CUDA(cudaStreamSynchronize(c->stream));
  int status = 0;
  LP_CUDA(cudaMemcpy(&status, c->dStatus, 4, cudaMemcpyDeviceToHost));
  if (status & lp::ST_JACOBI) return fail(c, LP_ERR_NUMERIC, "Jacobi SVD did not converge or singular block");
  return LP_OK;
}

}  // extern "C"

// ---- hooks for the batch runner (one graph over many contexts) ----------------
lp_status lp::batch_prepare(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, const double* y0,
                            int refine_rounds, unsigned flags) {
  const double* dy0 = nullptr;
  return solve_prepare(c, k, p_schedule, T, agg, y0, refine_rounds, flags, false, &dy0);
}

lp_status lp::batch_enqueue(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, int refine_rounds,
                            unsigned flags, lp_stats* captured) {
  std::memset(&c->stats, 0, sizeof(c->stats));
  c->step_ev_used = 0;
  LP_CUDA(record_event(c->ev0, c->stream));
  const lp_status st = solve_body(c, k, p_schedule, T, agg, refine_rounds, (flags & LP_FLAG_TIMING) != 0, c->dStage,
                                  (flags & LP_FLAG_TRACE) != 0, (flags & LP_FLAG_KXK_FP64) != 0);
  if (st) return st;
  LP_CUDA(record_event(c->ev1, c->stream));
  *captured = c->stats;
  return LP_OK;
}

void lp::batch_mark(lp_ctx* c, int k, const lp_stats& captured, int rounds, unsigned flags) {
  c->stats = captured;
  solve_mark(c, k, rounds, flags);
}

cudaStream_t lp::ctx_stream(lp_ctx* c) { return c->stream; }

lp_status lp::problem_result(lp_ctx* c, int q, double* z_out, double* sigma_out, lp_stats* stats) {
  if (!c) return LP_ERR_INVALID;
  c->err.clear();
  if (q < 0 || q >= c->nprob) return fail(c, LP_ERR_INVALID, "problem index out of range");
  if (!c->solved) return fail(c, LP_ERR_STATE, "no solve to report");
  LP_CUDA(cudaSetDevice(c->device));
  LP_CUDA(cudaStreamSynchronize(c->stream));
  int status = 0;
  LP_CUDA(cudaMemcpy(&status, c->dStatus, 4, cudaMemcpyDeviceToHost));
  const size_t blk = size_t(c->d) * c->k;
  if (z_out) LP_CUDA(cudaMemcpy(z_out, c->dZout + q * blk, blk * 8, cudaMemcpyDeviceToHost));
  if (sigma_out) {
    if (c->ritz)
      LP_CUDA(cudaMemcpy(sigma_out, c->dSigma + size_t(q) * LP_MAX_K, size_t(c->k) * 8, cudaMemcpyDeviceToHost));
    else std::memset(sigma_out, 0, size_t(c->k) * 8);
  }
  if (stats) {
    // the group's counters, with the shape and the A bytes of this problem
    *stats = c->stats;
    stats->n = c->prob_n[q];
    stats->m = c->prob_begin[q + 1] - c->prob_begin[q];
    stats->a_bytes = c->stats.a_bytes * double(c->prob_n[q]) / double(c->n);
  }
  // the status word is shared by the group's problems
  if (status & lp::ST_TIMEOUT) return fail(c, LP_ERR_TIMEOUT, "device wait timed out");
  if (status & lp::ST_CHOL) return fail(c, LP_ERR_NUMERIC, "Cholesky breakdown (non-positive or non-finite pivot)");
  if (status & lp::ST_NONFINITE) return fail(c, LP_ERR_NUMERIC, "non-finite iterate");
  if (status & lp::ST_JACOBI) return fail(c, LP_ERR_NUMERIC, "Jacobi iteration did not converge or singular block");
  return LP_OK;
}
