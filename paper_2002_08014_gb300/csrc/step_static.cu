// lp_power_step_static: the local power step without any device allocation.
//
// Some callers cannot allocate device memory at all: code that runs inside a
// memory pool or allocator it must not re-enter, a host that has reserved the
// whole device up front, or a context where cudaMalloc would synchronise the
// device at the wrong moment.  For them this entry point runs the same
// kernels as lp_power_step (SIMT FP32 step, fixed-order reduce) but keeps all
// its scratch -- the per-CTA partial sums, the row-segment table, the padded
// copies of Z and Y -- in one file-scope __device__ array of kStaticScratchBytes.
//
// Notes for users:
//   * The array is part of the library image: every GPU that loads the library
//     holds it (32 MiB) until the process exits.
//   * The first call on a device, with that device current, looks up the
//     array's device address (cudaGetSymbolAddress) and caches it.
//   * All calls share the one array and it keeps the last call's contents.
//     Every byte a call reads is written earlier in the same call (the kernels
//     overwrite the tables, partials and padded blocks in full, and the status
//     word at the array's start is cleared on the stream first), but calls
//     whose work overlaps on the GPU race with each other: serialise them (one
//     stream, or events).
//   * The call returns before the GPU runs its work, so a bounded wait that
//     gives up inside the step kernel (a stall of seconds) cannot become a
//     status code: a last small kernel reads the status word and, if any bit
//     is set, overwrites every entry of y with NaN.
//   * Inputs and outputs stay the caller's: A (FP32, partitions back to back,
//     row pitch d), Z and Y (FP64) are device pointers.
#include <algorithm>
#include <mutex>
#include <string>
#include <vector>

#include "lp_internal.cuh"

namespace {

constexpr size_t kStaticScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Failures are reported like lp_create's: lp_last_error(NULL) returns the text.
lp_status fail(lp_status st, const std::string& msg) {
  lp::set_no_context_error(msg);
  return st;
}

size_t up256(size_t b) { return (b + 255) / 256 * 256; }

// y <- NaN everywhere when the step recorded a failure in the status word.
__global__ void poison_on_status_kernel(const int* status, double* y, int64_t count) {
  if (*status == 0) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < count; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = nan;
}

}  // namespace

extern "C" lp_status lp_power_step_static(const float* A, int m, const int64_t* rows, int64_t d, int k,
                                          const double* z, double* y, void* stream) {
  using lp::Segment;
  lp::set_no_context_error("");
  if (!A || !rows || !z || !y) return fail(LP_ERR_INVALID, "A, rows, z and y must be non-NULL");
  if (m < 1) return fail(LP_ERR_INVALID, "need m >= 1");
  if (d < 1 || d % 4 != 0) return fail(LP_ERR_INVALID, "d must be a positive multiple of 4 (16-byte rows)");
  if (reinterpret_cast<uintptr_t>(A) % 16 != 0) return fail(LP_ERR_INVALID, "A must be 16-byte aligned");
  if (k < 1 || k > LP_MAX_K || k > d) return fail(LP_ERR_INVALID, "k must be in [1, min(32, d)]");
  int64_t n = 0, smin = rows[0];
  for (int i = 0; i < m; ++i) {
    if (rows[i] < 1) return fail(LP_ERR_INVALID, "every partition needs at least one row");
    n += rows[i];
    smin = rows[i] < smin ? rows[i] : smin;
  }
  if (k > smin) return fail(LP_ERR_INVALID, "k exceeds the smallest partition's row count");
  const int K = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  if (lp::step_simt_smem(static_cast<int>(d), d, LP_F32, K, nullptr) == 0)
    return fail(LP_ERR_UNSUPPORTED, "no step kernel for this d and k");

  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return fail(LP_ERR_CUDA, std::string("device query failed: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(LP_ERR_UNSUPPORTED, "device ordinal beyond the address cache");
  void* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_static_scratch);
      if (e != cudaSuccess || !p)
        return fail(LP_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
      g_scratch_addr[dev] = p;
    }
    base = g_scratch_addr[dev];
  }

  // Row segments: CTA g owns rows [g n / G, (g+1) n / G), cut at partition ends.
  const int G = static_cast<int>(n / 32 < sms ? (n / 32 > 0 ? n / 32 : 1) : sms);
  std::vector<Segment> segs;
  std::vector<int> seg_ptr(G + 1, 0), slot_begin(m + 1, 0);
  std::vector<float> invs(m);
  {
    std::vector<int64_t> off(m);
    int64_t o = 0;
    for (int i = 0; i < m; ++i) {
      off[i] = o;
      o += rows[i];
      invs[i] = static_cast<float>(1.0 / static_cast<double>(rows[i]));
    }
    int part = 0;
    for (int g = 0; g < G; ++g) {
      seg_ptr[g] = static_cast<int>(segs.size());
      int64_t r0 = n * g / G, r1 = n * (g + 1) / G;
      while (r0 < r1) {
        while (off[part] + rows[part] <= r0) ++part;
        const int64_t pend = off[part] + rows[part];
        const int64_t end = r1 < pend ? r1 : pend;
        Segment s;
        s.row0 = r0;
        s.row1 = end;
        s.part = part;
        s.slot = static_cast<int>(segs.size());
        segs.push_back(s);
        r0 = end;
      }
    }
    seg_ptr[G] = static_cast<int>(segs.size());
    int s = 0;
    for (int i = 0; i < m; ++i) {
      while (s < static_cast<int>(segs.size()) && segs[s].part < i) ++s;
      slot_begin[i] = s;
    }
    slot_begin[m] = static_cast<int>(segs.size());
  }
  const int nslots = static_cast<int>(segs.size());
  int max_slots = 0;
  for (int i = 0; i < m; ++i) max_slots = std::max(max_slots, slot_begin[i + 1] - slot_begin[i]);

  // Carve the static array.
  unsigned char* cur = static_cast<unsigned char*>(base);
  auto take = [&](size_t bytes) {
    unsigned char* p = cur;
    cur += up256(bytes);
    return p;
  };
  const size_t need = up256(sizeof(int)) + up256(segs.size() * sizeof(Segment)) + up256((G + 1) * sizeof(int)) +
                      up256((m + 1) * sizeof(int)) + up256(m * sizeof(float)) + up256(size_t(d) * K * 4) +
                      up256(size_t(nslots) * d * K * 4) + up256(size_t(m) * d * K * 4);
  if (need > kStaticScratchBytes)
    return fail(LP_ERR_INVALID, "problem needs " + std::to_string(need) + " bytes of scratch; the static array holds " +
                                    std::to_string(kStaticScratchBytes));
  int* dStatus = reinterpret_cast<int*>(take(sizeof(int)));
  Segment* dSegs = reinterpret_cast<Segment*>(take(segs.size() * sizeof(Segment)));
  int* dSegPtr = reinterpret_cast<int*>(take((G + 1) * sizeof(int)));
  int* dSlotBegin = reinterpret_cast<int*>(take((m + 1) * sizeof(int)));
  float* dInvS = reinterpret_cast<float*>(take(m * sizeof(float)));
  float* dZ = reinterpret_cast<float*>(take(size_t(d) * K * 4));
  float* dP = reinterpret_cast<float*>(take(size_t(nslots) * d * K * 4));
  float* dY = reinterpret_cast<float*>(take(size_t(m) * d * K * 4));

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int di = static_cast<int>(d);
  if ((e = cudaMemsetAsync(dStatus, 0, sizeof(int), s)) ||
      (e = cudaMemcpyAsync(dSegs, segs.data(), segs.size() * sizeof(Segment), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dSegPtr, seg_ptr.data(), seg_ptr.size() * sizeof(int), cudaMemcpyHostToDevice, s)) ||
      (e = cudaMemcpyAsync(dSlotBegin, slot_begin.data(), slot_begin.size() * sizeof(int), cudaMemcpyHostToDevice,
                           s)) ||
      (e = cudaMemcpyAsync(dInvS, invs.data(), invs.size() * sizeof(float), cudaMemcpyHostToDevice, s)) ||
      (e = lp::launch_pack(z, dZ, 1, di, k, K, s)))
    return fail(LP_ERR_CUDA, std::string("staging failed: ") + cudaGetErrorString(e));
  lp::StepArgs a;
  a.A = A;
  a.ld = d;
  a.d = di;
  a.scales = nullptr;
  a.segs = dSegs;
  a.seg_ptr = dSegPtr;
  a.Z = dZ;
  a.z_stride = 0;
  a.P = dP;
  a.grid = G;
  a.status = dStatus;
  if ((e = lp::launch_step_simt(a, LP_F32, K, s)) || (e = lp::launch_reduce(dP, dSlotBegin, dInvS, m, di, K, dY, s, max_slots)) ||
      (e = lp::launch_unpack(dY, y, m, di, k, K, s)))
    return fail(LP_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  const int64_t count = int64_t(m) * d * k;
  poison_on_status_kernel<<<static_cast<unsigned>(std::min<int64_t>((count + 255) / 256, 1024)), 256, 0, s>>>(
      dStatus, y, count);
  if ((e = cudaGetLastError()) != cudaSuccess)
    return fail(LP_ERR_CUDA, std::string("launch failed: ") + cudaGetErrorString(e));
  // The host tables above are copied from pageable memory, so the copies have
  // completed (or been staged) by the time cudaMemcpyAsync returns.
  return LP_OK;
}
