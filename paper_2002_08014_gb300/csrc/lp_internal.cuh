// Internal declarations of the LocalPower CUDA library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>
#include <string>

#include "localpower.h"

namespace lp {

// Bits of the device status word (OR-ed by kernels, read by lp_result).
enum StatusBits : int {
  ST_CHOL = 1,        // non-positive or non-finite Cholesky pivot
  ST_NONFINITE = 2,   // non-finite value in an iterate
  ST_JACOBI = 4,      // Jacobi sweeps hit their limit
  ST_TIMEOUT = 8,     // a bounded wait gave up
};

// One contiguous run of rows of one partition processed by one CTA of the
// fused step kernel.  Global row indices into the packed A buffer.
struct Segment {
  int64_t row0, row1;  // [row0, row1)
  int part;            // partition index i
  int slot;            // output slot of the CTA's partial A_i^T A_i Z_i
};

// Lets every launch of `kern` request up to the device's opt-in shared memory per
// block, less the kernel's static shared memory (once per kernel).  The limit is
// a property of the function, not of a launch: set to each plan's own size, a
// smaller plan of another context (same kernel, another shape) would lower it
// under a larger launch already captured in a graph, and that launch would be
// rejected when the graph replays.
cudaError_t allow_max_dynamic_smem(const void* kern);

// ---- fused local power step (SIMT) ---------------------------------------
struct StepArgs {
  const void* A;          // packed partitions, row pitch `ld` elements
  int64_t ld;             // elements
  int d;                  // columns
  const float* scales;    // FP8 row scales (global row index) or nullptr
  const Segment* segs;    // all segments, CTA-major
  const int* seg_ptr;     // CTA g owns segs[seg_ptr[g] .. seg_ptr[g+1])
  const float* Z;         // d x K blocks (FP32, columns >= k are zero)
  int64_t z_stride;       // floats between partitions' Z blocks (0: shared)
  float* P;               // slots x d x K partial sums of A_i^T (A_i Z_i)
  int grid;               // CTAs
  int zld = 0, pld = 0;   // row strides of Z and P in floats (0: K); a launch on a column
                          // range of wider blocks passes the wider stride and offset pointers
  int* status = nullptr;  // device status word for ST_TIMEOUT (bounded waits), or nullptr
};

// Returns cudaErrorInvalidConfiguration when no SIMT instantiation fits.
cudaError_t launch_step_simt(const StepArgs& a, lp_dtype dtype, int K, cudaStream_t s);
// FP32 SIMT step with Z_i resident in tensor memory (K = 16, d <= 1024); the FP32
// dispatch of launch_step_simt prefers it where it is supported.
bool step_simt_tmem_supported(int d, int64_t ld, int K);
cudaError_t launch_step_simt_tmem(const StepArgs& a, cudaStream_t s);
// Shared memory the SIMT step needs (0 if unsupported); used to validate up front.
size_t step_simt_smem(int d, int64_t ld, lp_dtype dtype, int K, int* rows_per_tile);

// ---- fused local power step (tcgen05 tensor cores, BF16 A) ---------------
struct TcPlan {
  int K = 0;           // padded k (8, 16, 32); MMA N = 2K
  int nch = 0;         // 64-column chunks per CTA (2 or 4)
  int cluster = 0;     // CTAs per cluster splitting d
  int nclusters = 0;   // clusters in the grid (one CTA per SM)
  size_t smem = 0;     // dynamic shared memory per CTA
  alignas(64) unsigned char tmap[128];  // CUtensorMap of the packed BF16 A
};
// Fills the geometry for (d, k); false when the shape has no tensor-core kernel.
bool tc_plan(int d, int k, int sms, TcPlan* p);
// Encodes the 2-D tensor map of A (n rows, d columns, row pitch ld elements).
cudaError_t tc_encode_map(void* A, int64_t n, int d, int64_t ld, TcPlan* p);
cudaError_t launch_step_tc(const TcPlan& p, const Segment* segs, const int* seg_ptr, const float* Z, int64_t z_stride,
                           float* P, int d, int* status, cudaStream_t s);

// ---- fused local power step (tcgen05, streaming; BF16 plane or hi/lo planes) --
struct TcsPlan {
  int K = 0;           // padded k (8, 16, 32); MMA N = 2K
  int planes = 0;      // 1: BF16 A; 2: hi + lo BF16 planes of FP32 A
  int ncd = 0;         // 64-column chunks of each CTA's column slice (even)
  int cluster = 0;     // CTAs per cluster splitting d
  int nclusters = 0;   // clusters in the grid (one CTA per SM)
  int ring = 0;        // 32 KB ring units
  int lag = 0;         // first-pass units of tile t+1 issued before tile t's second pass
  int prefetch = 0;    // first-pass units prefetched into L2 ahead of their load
  int hints = 0;       // L2 eviction hints on the two passes
  uint32_t off_B1 = 0, off_B2 = 0, off_W = 0, off_Wrecv = 0, off_bar = 0, tmem_cols = 0;
  size_t smem = 0;     // dynamic shared memory per CTA
  // pass-split pair kernel (step_pair.cu): cluster = 2, `ring` is rank 0's ring,
  // off_B1 holds Z, off_B2 the W staging / W buffers
  int pair = 0;        // 1: this plan is for the pair kernel
  int ring1 = 0;       // rank 1 ring units
  int nd2 = 0;         // rank 1 Y-slice buffers in tensor memory
  uint32_t tmem_cols1 = 0;
  long long stall = 0;  // test hook (lp_tuning::test_stall_cycles)
  // FP8-E4M3 streaming kernel (step_tcs8.cu): codes staged by TMA, widened to FP16
  int fp8 = 0;         // 1: this plan is for step_tcs8_kernel
  int issuers = 1;     // streaming kernels: MMA-issuing threads (own partial D1 and ring slots each)
  int map3d = 0;       // pair kernel: the maps are (64 columns, row, chunk), one box per unit
  int stage = 0;       // staging ring units (16 KB of codes each)
  uint32_t off_stage = 0;
  alignas(64) unsigned char tmap[2][128];  // CUtensorMaps of the planes
};
// Tuning of the streaming kernel (lp_tuning without the C names); zeros are defaults.
struct TcsTuning {
  int ring_units = 0, lag_units = 0, prefetch_units = 0, cache_hints = 0, slice_cols = 0;
  int kernel = 0;  // LP_KERNEL_* of lp_tuning
  long long test_stall_cycles = 0;  // lp_tuning::test_stall_cycles
};
// Fills the geometry for (d, k, planes).  False when the shape has no streaming kernel.
bool tcs_plan(int d, int k, int planes, int sms, const TcsTuning& tune, TcsPlan* p);
// Encodes the tensor maps of the planes (plane1 may be NULL for one plane).
// unit_boxes: where d is a multiple of 64 and rows are unpadded, encode three-dimensional
// maps whose one box covers a whole 128-column unit (p->map3d = 1; the pair kernel's loads).
cudaError_t tcs_encode_maps(const void* plane0, const void* plane1, int64_t n, int d, int64_t ld, TcsPlan* p,
                            bool unit_boxes = false);
cudaError_t launch_step_tcs(const TcsPlan& p, const Segment* segs, const int* seg_ptr, const float* Z,
                            int64_t z_stride, float* P, int d, int* status, cudaStream_t s);
// Pass-split pair kernel: the same product with the HBM pass and the L2 pass on
// the two CTAs of a cluster.  False when the shape has no plan (d > 1024 at
// k > 16, d > 2048, or a ring under two units).
bool pair_plan(int d, int k, int planes, int sms, const TcsTuning& tune, TcsPlan* p);
// FP8-E4M3 codes with FP32 row scales on the tensor cores (streaming form; the
// codes are widened to FP16 in shared memory).  False when the shape has no plan.
bool tcs8_plan(int d, int k, int sms, const TcsTuning& tune, TcsPlan* p);
cudaError_t tcs8_encode_map(const void* codes, int64_t n, int d, int64_t ld, TcsPlan* p);
cudaError_t launch_step_tcs8(const TcsPlan& p, const Segment* segs, const int* seg_ptr, const float* Z,
                             int64_t z_stride, float* P, int d, const float* scales, float smax2, int* status,
                             cudaStream_t s);
cudaError_t launch_step_pair(const TcsPlan& p, const Segment* segs, const int* seg_ptr, const float* Z,
                             int64_t z_stride, float* P, int d, int* status, cudaStream_t s);
// FP32 rows (pitch src_ld) -> hi = RNE_bf16(a), lo = RNE_bf16(a - hi) planes (pitch ld,
// columns d..ld-1 zero).
cudaError_t launch_split_planes(const float* src, int64_t src_ld, int64_t rows, int d, uint16_t* hi, uint16_t* lo,
                                int64_t ld, cudaStream_t s);

// ---- context internals used by the request server ---------------------------
// lp_load_partitions with a row pitch (elements) for the partitions' source rows.
lp_status load_pitched(lp_ctx* c, int m, const int64_t* rows, int64_t d, int64_t pitch, lp_dtype dtype,
                       const void* const* parts, const float* const* row_scales, lp_ptr_space space);
// Device bytes a context needs to load these partitions and solve at rank k.
size_t estimate_bytes(int sms, int m, const int64_t* rows, int64_t d, int64_t pitch, lp_dtype dtype, int k,
                      lp_ptr_space space);
// 1: the last lp_solve finished on the device; 0: still running; -1: no solve or a CUDA error.
int solve_state(lp_ctx* c);
// A solve split for capture into one graph over many contexts: checks, kernel
// choice and y0 upload (outside the capture); the launch sequence on the
// context's stream (inside it; *captured receives its counters); and marking
// the context solved after the graph ran.
lp_status batch_prepare(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, const double* y0,
                        int refine_rounds, unsigned flags);
lp_status batch_enqueue(lp_ctx* c, int k, const int* p_schedule, int T, lp_aggregator agg, int refine_rounds,
                        unsigned flags, lp_stats* captured);
void batch_mark(lp_ctx* c, int k, const lp_stats& captured, int rounds, unsigned flags);
cudaStream_t ctx_stream(lp_ctx* c);
// Several independent problems in one context (the batch runner's groups): load the
// partitions of nsrc loaded single-problem contexts of one width and type back to
// back (device copies of the stored rows) and make each source one problem.
lp_status load_merged(lp_ctx* c, lp_ctx* const* src, int nsrc);
// Problem q owns partitions [part_begin[q], part_begin[q + 1]); weights s_i / n_q, the
// base is each problem's first largest partition.  lp_solve then takes nprob
// consecutive d x k start blocks.
lp_status set_problems(lp_ctx* c, int nprob, const int* part_begin);
// lp_result of problem q (the stats are the context's, with problem q's n, m and A bytes).
lp_status problem_result(lp_ctx* c, int q, double* z_out, double* sigma_out, lp_stats* stats);

// Message returned by lp_last_error(NULL) (failures of calls without a context).
void set_no_context_error(const char* msg);
inline void set_no_context_error(const std::string& msg) { set_no_context_error(msg.c_str()); }

// ---- small kernels --------------------------------------------------------
// Y_i = scale_i * sum_{slot in [slot_begin[i], slot_begin[i+1])} P[slot]; max_slots (the most
// slots any partition has) picks how many threads share one output.
cudaError_t launch_reduce(const float* P, const int* slot_begin, const float* scale, int m, int d, int K,
                          float* Y, cudaStream_t s, int max_slots);
// Z_b = orth(Y_b) (CholQR2 on FP32 data), batch blocks of d x K.  kxk_fp64: the k x k
// Gram and Cholesky in FP64; else FP32 with an FP64 Cholesky when a pivot is too small.
cudaError_t launch_cholqr2(const float* Y, float* Z, int batch, int d, int k, int K, int* status, cudaStream_t s,
                           bool kxk_fp64);
// G_i = aligning matrices (K x K, FP32) for agg in {SIGN, OPT}; base gets I.  kxk_fp64:
// the k x k Procrustes SVD in FP64, else FP32.
// part_base (device, may be nullptr): per-partition base partition (several problems in
// one context); then Zb and base are ignored and Z_b = Zl + z_stride * part_base[i].
cudaError_t launch_align(const float* Zl, int64_t z_stride, const float* Zb, int m, int d, int k, int K, int base,
                         lp_aggregator agg, float* G, int* status, cudaStream_t s, bool kxk_fp64,
                         const int* part_base);
// Y = sum_i w_i Y_i G_i  (G == nullptr: identity; diag_only: G_i diagonal).  With
// prob_begin (device, nprob + 1 offsets): Y_q = the sum over problem q's partitions,
// nprob consecutive d x K blocks.
cudaError_t launch_aggregate(const float* Yl, const float* w, const float* G, int diag_only, int m, int d, int K,
                             float* Y, cudaStream_t s, const int* prob_begin, int nprob);
// Zl[i] = Z[part_prob[i]] for the m partitions' d x K blocks.
cudaError_t launch_broadcast(const float* Z, const int* part_prob, int m, int d, int K, float* Zl, cudaStream_t s);
// Ritz: H = Z^T MZ (FP64 sums), eig by Jacobi (FP64 when kxk_fp64, else FP32), Zout = Z W
// (FP64), sigma = sqrt(n lambda).  Three launches; `scratch` holds ritz_scratch_bytes(d, K,
// nprob) bytes.  nprob problems at once: Z, MZ consecutive d x K blocks, Zout consecutive
// d x k blocks, sigma LP_MAX_K apart, n_of (device, may be nullptr for one problem) their
// row counts.
cudaError_t launch_ritz(const float* Z, const float* MZ, int d, int k, int K, double n, double* Zout, double* sigma,
                        double* scratch, int* status, cudaStream_t s, bool kxk_fp64, int nprob = 1,
                        const double* n_of = nullptr);
size_t ritz_scratch_bytes(int d, int K, int nprob = 1);
// out[i] = ||Z_i G_i - Z_b||_2 (Def. 3), G_i the aligner (nullptr: none; diag_only: sign-fixing); out[base] = 0.
cudaError_t launch_rho(const float* Zl, int64_t z_stride, const float* Zb, const float* G, int diag_only, int base,
                       int m, int d, int k, int K, double* out, int* status, cudaStream_t s);
// ---- eta of Def. 2 --------------------------------------------------------
// Z = columns [c0, c0 + K) of the d x d identity (d x K FP32 block).
cudaError_t launch_identity_block(float* Z, int d, int K, int c0, cudaStream_t s);
// Rows c0 .. c0 + ncols - 1 of slot i (d x d FP32, slot stride d^2) = columns of Y_i (d x K blocks).
cudaError_t launch_scatter_columns(const float* Y, float* Mall, int m, int d, int K, int c0, int ncols,
                                   cudaStream_t s);
// Slot m = M = sum_i w_i sym(slot i) (FP64 sums); slot i = sym(slot i) - M for i < m.
cudaError_t launch_deviations(float* Mall, const float* w, int m, int d, cudaStream_t s);
// out[j] = ||slot j||_2 for j < nmat (symmetric slots) by Lanczos with full
// reorthogonalisation; V holds nmat x lanczos_steps(d) x d floats.
cudaError_t launch_lanczos_norms(const float* Mall, int nmat, int d, float* V, double* out, cudaStream_t s);
int lanczos_steps(int d);
size_t lanczos_smem(int d);

// FP64 d x k (row-major) <-> FP32 d x K padded blocks
cudaError_t launch_pack(const double* src, float* dst, int batch, int d, int k, int K, cudaStream_t s);
cudaError_t launch_unpack(const float* src, double* dst, int batch, int d, int k, int K, cudaStream_t s);

}  // namespace lp
