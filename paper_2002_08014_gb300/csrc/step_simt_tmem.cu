// Fused local power step, SIMT FP32 with Z_i resident in tensor memory (k <= 16,
// d <= 1024):  P[slot] = A_seg^T (A_seg Z_i), the unscaled local product of
// eq. (2) (the reduce kernel applies 1/s_i).
//
// The FP32 products run on the FP32 pipe (the contraction is FP32 x FP32 and
// must stay FP32-exact), so the budget that matters is shared-memory
// bandwidth next to the FMAs.  Keeping Z_i (d x 16 FP32) in shared memory and
// reading it there for W = A_tile Z_i costs more shared-memory wavefronts than
// everything else in the step.  Here Z_i lives in TMEM instead: each of the
// four TMEM lane quarters holds a full copy, lane l holding rows c = l + 32 t
// of Z_i in columns 16 t .. 16 t + 15, and tcgen05.ld moves it to registers
// on a path of its own.
//
// One CTA of 512 threads per SM streams its rows once from HBM; 16-row tiles
// are double buffered in shared memory (cp.async).  Per tile:
//   phase 1  warp w computes row w of W = A_tile Z_i: lane l takes columns
//            c = l + 32 t (one shared-memory word per step, consecutive across
//            the warp) times row c of Z_i from TMEM; a shuffle reduce-scatter
//            sums the 32 lanes, so no cross-warp reduction is needed;
//   phase 2  Y += A_tile^T W with each thread's columns c = tid + 512 q of the
//            d x 16 partial Y in registers for the CTA's whole segment.
// For d = 1024 (the row length of the FP32 benchmark) a second kernel with
// compile-time geometry software-pipelines the tiles: phase 2 of tile t runs
// interleaved with phase 1 of tile t + 1 in every warp.
// Only one CTA fits an SM (512 threads x 128 registers), so the TMEM
// allocation never waits on another CTA.
#include "lp_internal.cuh"
#include "tc_ptx.cuh"

namespace lp {
namespace {

using tc::su32;

constexpr int kThr = 512;
constexpr int kK = 16;
constexpr int kR = 16;  // rows per tile: one per warp in phase 1

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(smem)), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// 32 lanes x 16 consecutive 32-bit columns, no wait (tcgen05.wait::ld waits for all).
__device__ __forceinline__ void tmem_ld16_async(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
// 32 lanes x 32 consecutive 32-bit columns, no wait.
__device__ __forceinline__ void tmem_ld32_async(uint32_t taddr, uint32_t (&r0)[16], uint32_t (&r1)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r0[0]), "=r"(r0[1]), "=r"(r0[2]), "=r"(r0[3]), "=r"(r0[4]), "=r"(r0[5]), "=r"(r0[6]), "=r"(r0[7]),
        "=r"(r0[8]), "=r"(r0[9]), "=r"(r0[10]), "=r"(r0[11]), "=r"(r0[12]), "=r"(r0[13]), "=r"(r0[14]), "=r"(r0[15]),
        "=r"(r1[0]), "=r"(r1[1]), "=r"(r1[2]), "=r"(r1[3]), "=r"(r1[4]), "=r"(r1[5]), "=r"(r1[6]), "=r"(r1[7]),
        "=r"(r1[8]), "=r"(r1[9]), "=r"(r1[10]), "=r"(r1[11]), "=r"(r1[12]), "=r"(r1[13]), "=r"(r1[14]), "=r"(r1[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float4 (&v)[4]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "f"(v[0].x), "f"(v[0].y), "f"(v[0].z), "f"(v[0].w), "f"(v[1].x), "f"(v[1].y), "f"(v[1].z), "f"(v[1].w),
      "f"(v[2].x), "f"(v[2].y), "f"(v[2].z), "f"(v[2].w), "f"(v[3].x), "f"(v[3].y), "f"(v[3].z), "f"(v[3].w)
      : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tc_sync() {
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
}

struct GeoT {
  int T;     // lane steps: ceil(d / 32)
  int lds;   // tile row stride in floats (>= 32 T and >= ld, multiple of 4)
  int cols;  // TMEM columns allocated (power of two >= 16 T)
};

__device__ __forceinline__ void fma_row(float2 (&acc)[kK / 2], float a, const uint32_t (&z)[16]) {
  const float2 a2 = make_float2(a, a);
#pragma unroll
  for (int j = 0; j < kK / 2; ++j)
    acc[j] = __ffma2_rn(a2, make_float2(__uint_as_float(z[2 * j]), __uint_as_float(z[2 * j + 1])), acc[j]);
}

// Sum a row's per-lane partials over the 32 lanes into Wrow[0..15]: a
// reduce-scatter whose halving steps leave lane l with the sum of column l >> 1,
// then the pair (l, l ^ 1) adds its halves.
__device__ __forceinline__ void store_row_sum(const float2 (&acc)[kK / 2], int lane, float* Wrow) {
  float v[kK];
#pragma unroll
  for (int j = 0; j < kK / 2; ++j) {
    v[2 * j] = acc[j].x;
    v[2 * j + 1] = acc[j].y;
  }
#pragma unroll
  for (int h = kK / 2, mask = 16; h >= 1; h >>= 1, mask >>= 1) {
    const bool up = (lane & mask) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const float send = up ? v[k] : v[k + h];
      const float keep = up ? v[k + h] : v[k];
      v[k] = keep + __shfl_xor_sync(0xffffffffu, send, mask);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  if ((lane & 1) == 0) Wrow[lane >> 1] = v[0];
}

template <int CPT>
__global__ void __launch_bounds__(kThr, 1) step_simt_tmem_kernel(StepArgs a, GeoT g) {
  extern __shared__ __align__(16) float smt[];
  __shared__ uint32_t tmem_holder;
  const int T = g.T;
  const int lds = g.lds;
  const int d = a.d;
  const int64_t ld = a.ld;
  float* buf0 = smt;
  float* buf1 = buf0 + kR * lds;
  float* Ws = buf1 + kR * lds;  // R x K

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int zld = a.zld > 0 ? a.zld : kK, pld = a.pld > 0 ? a.pld : kK;
  const float* A = static_cast<const float*>(a.A);
  const int cpr = static_cast<int>(ld / 4);  // 16-byte chunks per row
  // row-tile copy plan: rows per pass, this thread's first row and chunk (cpr <= threads)
  const int cp_rstep = kThr / cpr, cp_r0 = tid / cpr, cp_ch = tid % cpr;

  for (int r = 0; r < kR; ++r)
    for (int c = static_cast<int>(ld) + tid; c < lds; c += kThr) {
      buf0[r * lds + c] = 0.f;
      buf1[r * lds + c] = 0.f;
    }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                 "r"(g.cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t tq = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);  // this warp's lane quarter

  float2 y[CPT][kK / 2];
#pragma unroll
  for (int q = 0; q < CPT; ++q)
#pragma unroll
    for (int j = 0; j < kK / 2; ++j) y[q][j] = make_float2(0.f, 0.f);

  int cur_part = -1;
  const int sb = a.seg_ptr[blockIdx.x], se = a.seg_ptr[blockIdx.x + 1];
  for (int si = sb; si < se; ++si) {
    const Segment sg = a.segs[si];
    const int ntiles = static_cast<int>((sg.row1 - sg.row0 + kR - 1) / kR);
    // thread tid copies chunk cp_ch of rows cp_r0, cp_r0 + cp_rstep, ... (rows past
    // the segment are zero-filled)
    auto issue = [&](int t, float* buf) {
      const int64_t r0 = sg.row0 + int64_t(t) * kR;
      if (cp_r0 < cp_rstep)
        for (int r = cp_r0; r < kR; r += cp_rstep) {
          const int64_t grow = r0 + r;
          const bool ok = grow < sg.row1;
          cp_async16(buf + size_t(r) * lds + cp_ch * 4, A + (ok ? grow : sg.row0) * ld + int64_t(cp_ch) * 4,
                     ok ? 16 : 0);
        }
      cp_async_commit();
    };
    issue(0, buf0);  // the first tile loads while Z_i is staged
    if (sg.part != cur_part) {
      tc_sync();  // every warp's TMEM reads of the previous Z_i have completed
      cur_part = sg.part;
      const float* Zg = a.Z + a.z_stride * sg.part;
      // the four warps of a lane quarter split its T steps
      for (int t = warp >> 2; t < T; t += 4) {
        const int c = lane + 32 * t;
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j)
          v[j] = c < d ? *reinterpret_cast<const float4*>(Zg + size_t(c) * zld + 4 * j) : make_float4(0.f, 0.f, 0.f, 0.f);
        tmem_st16(tq + 16 * t, v);
      }
      tmem_wait_st();
      tc_sync();
    }
    for (int t = 0; t < ntiles; ++t) {
      const float* Tt = (t & 1) ? buf1 : buf0;
      if (t + 1 < ntiles) {
        issue(t + 1, (t & 1) ? buf0 : buf1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();

      // ---- phase 1: row `warp` of W, lanes over the columns, Z_i from TMEM
      const float* Arow = Tt + size_t(warp) * lds + lane;
      float2 acc[kK / 2];
#pragma unroll
      for (int j = 0; j < kK / 2; ++j) acc[j] = make_float2(0.f, 0.f);
      int s = 0;
#pragma unroll
      for (; s + 1 < T; s += 2) {
        uint32_t z0[16], z1[16];
        tmem_ld16_async(tq + 16 * s, z0);
        tmem_ld16_async(tq + 16 * (s + 1), z1);
        const float a0 = Arow[32 * s], a1 = Arow[32 * (s + 1)];
        tmem_wait_ld();
        fma_row(acc, a0, z0);
        fma_row(acc, a1, z1);
      }
      if (s < T) {
        uint32_t z0[16];
        tmem_ld16_async(tq + 16 * s, z0);
        const float a0 = Arow[32 * s];
        tmem_wait_ld();
        fma_row(acc, a0, z0);
      }
      store_row_sum(acc, lane, Ws + warp * kK);
      __syncthreads();

      // ---- phase 2: Y += T^T W (packed FP32 FMAs)
#pragma unroll 2
      for (int r = 0; r < kR; ++r) {
        float2 w[kK / 2];
#pragma unroll
        for (int j = 0; j < kK; j += 4) {
          const float4 q4 = *reinterpret_cast<const float4*>(Ws + r * kK + j);
          w[j / 2] = make_float2(q4.x, q4.y);
          w[j / 2 + 1] = make_float2(q4.z, q4.w);
        }
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const int c = tid + kThr * q;
          if (c < d) {
            const float av = Tt[size_t(r) * lds + c];
            const float2 a2 = make_float2(av, av);
#pragma unroll
            for (int j = 0; j < kK / 2; ++j) y[q][j] = __ffma2_rn(a2, w[j], y[q][j]);
          }
        }
      }
      __syncthreads();
    }
    float* Pd = a.P + size_t(sg.slot) * d * pld;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int c = tid + kThr * q;
      if (c < d) {
#pragma unroll
        for (int j = 0; j < kK / 2; j += 2)
          *reinterpret_cast<float4*>(Pd + size_t(c) * pld + 2 * j) =
              make_float4(y[q][j].x, y[q][j].y, y[q][j + 1].x, y[q][j + 1].y);
      }
#pragma unroll
      for (int j = 0; j < kK / 2; ++j) y[q][j] = make_float2(0.f, 0.f);
    }
  }
  tc_sync();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(g.cols) : "memory");
}

// d = ld = 1024, software-pipelined across tiles: each warp interleaves phase 2
// of tile t (row r of the tile against W(t)) with phase 1 of tile t + 1 (two
// lane steps of its own row), so the FMAs of one hide the TMEM and shared-memory
// latencies of the other and no phase leaves the FP32 pipe idle behind a
// barrier.  Three tile buffers (t, t + 1 in use, t + 2 loading) and two W
// buffers; one barrier per tile.  A tile's 16 rows are 64 KB contiguous in both
// global and shared memory, so one thread loads it with a single bulk copy
// completing on the buffer's mbarrier (rows past the segment are zeroed by
// plain stores); the waits on it are bounded.  Same arithmetic as the kernel
// above.
constexpr int kD = 1024, kT32 = 32, kTile = kR * kD;

// Bulk copy global -> this CTA's shared memory, completion counted in bytes on
// an mbarrier; addresses 16-byte aligned, size a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(mbar)
               : "memory");
}

template <bool NEXT>
__device__ __forceinline__ void fused_rows(const float* __restrict__ Acur, const float* __restrict__ Wcur,
                                           const float* Anext_row, uint32_t tq, int tid, float2 (&y)[2][kK / 2],
                                           float2 (&acc)[kK / 2]) {
#pragma unroll 2
  for (int r = 0; r < kR; ++r) {
    uint32_t z0[16], z1[16];
    float a0 = 0.f, a1 = 0.f;
    if (NEXT) {
      tmem_ld32_async(tq + 32 * r, z0, z1);
      a0 = Anext_row[64 * r];
      a1 = Anext_row[64 * r + 32];
    }
    float2 w[kK / 2];
#pragma unroll
    for (int j = 0; j < kK; j += 4) {
      const float4 q4 = *reinterpret_cast<const float4*>(Wcur + r * kK + j);
      w[j / 2] = make_float2(q4.x, q4.y);
      w[j / 2 + 1] = make_float2(q4.z, q4.w);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const float av = Acur[r * kD + tid + kThr * q];
      const float2 a2 = make_float2(av, av);
#pragma unroll
      for (int j = 0; j < kK / 2; ++j) y[q][j] = __ffma2_rn(a2, w[j], y[q][j]);
    }
    if (NEXT) {
      tmem_wait_ld();
      fma_row(acc, a0, z0);
      fma_row(acc, a1, z1);
    }
  }
}

__global__ void __launch_bounds__(kThr, 1) step_simt_tmem_d1024_kernel(StepArgs a) {
  extern __shared__ __align__(16) float smt[];
  __shared__ uint32_t tmem_holder;
  __shared__ __align__(8) uint64_t full[3];
  __shared__ int s_abort;  // set when a bounded wait gave up
  float* bufs = smt;                  // 3 tiles of R x 1024
  float* Wb = smt + 3 * kTile;        // 2 x (R x K)
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int zld = a.zld > 0 ? a.zld : kK, pld = a.pld > 0 ? a.pld : kK;
  const float* A = static_cast<const float*>(a.A);

  if (tid == 0) {
    for (int b = 0; b < 3; ++b) tc::mbar_init(&full[b], 1);
    s_abort = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(&tmem_holder)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_sync();
  const uint32_t tmem = tmem_holder;
  const uint32_t tq = tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16);

  float2 y[2][kK / 2];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int j = 0; j < kK / 2; ++j) y[q][j] = make_float2(0.f, 0.f);

  uint32_t g0 = 0;  // tiles of earlier segments: tile t of this one is the CTA's tile g0 + t
  // CTA tiles whose copy was issued / whose wait succeeded (both in tile order);
  // they differ at the end only after a wait gave up
  uint32_t issued = 0, waited = 0;
  bool aborted = false;
  int cur_part = -1;
  const int sb = a.seg_ptr[blockIdx.x], se = a.seg_ptr[blockIdx.x + 1];
  for (int si = sb; si < se && !aborted; ++si) {
    const Segment sg = a.segs[si];
    const int ntiles = static_cast<int>((sg.row1 - sg.row0 + kR - 1) / kR);
    // tile t -> buffer t % 3 (called by every thread: thread 0 issues the copy,
    // all zero the rows past the segment)
    auto issue = [&](int t) {
      issued = g0 + t + 1;
      const int b = (g0 + t) % 3;
      float* buf = bufs + b * kTile;
      const int64_t r0 = sg.row0 + int64_t(t) * kR;
      const int valid = static_cast<int>(sg.row1 - r0 < kR ? sg.row1 - r0 : kR);
      if (tid == 0) {
        tc::mbar_expect_tx(&full[b], static_cast<uint32_t>(valid) * kD * 4);
        bulk_g2s(su32(buf), A + r0 * kD, static_cast<uint32_t>(valid) * kD * 4, su32(&full[b]));
      }
      if (valid < kR) {
        for (int e = valid * kD + tid * 4; e < kTile; e += kThr * 4)
          *reinterpret_cast<float4*>(buf + e) = make_float4(0.f, 0.f, 0.f, 0.f);
        tc::fence_async_smem();  // before a later bulk copy rewrites these rows
      }
    };
    // wait for tile t (its buffer's latest fill); bounded
    auto landed = [&](int t) {
      const uint32_t g = g0 + t;
      const uint32_t addr = su32(&full[g % 3]);
      const uint32_t parity = (g / 3) & 1;
      const long long t0 = clock64();
      while (!tc::mbar_try(addr, parity)) {
        if (clock64() - t0 > tc::kTimeoutCycles) {
          // give up: record it; every thread leaves the tile loop at its next
          // check (after a barrier), no further copies are issued, and thread 0
          // waits for the copies still in flight before the CTA exits
          if (a.status && lane == 0) atomicOr(a.status, ST_TIMEOUT);
          s_abort = 1;
          return;
        }
      }
      waited = g + 1;
    };
    // every buffer is free here: the previous segment ended with a barrier
    issue(0);
    if (ntiles > 1) issue(1);
    if (sg.part != cur_part) {
      tc_sync();
      cur_part = sg.part;
      const float* Zg = a.Z + a.z_stride * sg.part;
      for (int t = warp >> 2; t < kT32; t += 4) {
        const int c = lane + 32 * t;
        float4 v[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) v[j] = *reinterpret_cast<const float4*>(Zg + size_t(c) * zld + 4 * j);
        tmem_st16(tq + 16 * t, v);
      }
      tmem_wait_st();
      tc_sync();
    }
    // prologue: phase 1 of tile 0 alone
    landed(0);
    __syncthreads();
    {
      const float* Arow = bufs + (g0 % 3) * kTile + warp * kD + lane;
      float2 acc[kK / 2];
#pragma unroll
      for (int j = 0; j < kK / 2; ++j) acc[j] = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int s = 0; s < kT32; s += 2) {
        uint32_t z0[16], z1[16];
        tmem_ld32_async(tq + 16 * s, z0, z1);
        const float a0 = Arow[32 * s], a1 = Arow[32 * (s + 1)];
        tmem_wait_ld();
        fma_row(acc, a0, z0);
        fma_row(acc, a1, z1);
      }
      store_row_sum(acc, lane, Wb + warp * kK);
    }
    __syncthreads();
    for (int t = 0; t < ntiles; ++t) {
      if (s_abort) {  // read after a barrier: the same decision in every thread
        aborted = true;
        break;
      }
      const bool next = t + 1 < ntiles;
      // tile t + 2 goes into the buffer tile t - 1 used (freed by the last barrier)
      if (t + 2 < ntiles) issue(t + 2);
      if (next) landed(t + 1);
      __syncthreads();  // tile t + 1 (and any zeroed rows) visible to every thread
      const float* Acur = bufs + ((g0 + t) % 3) * kTile;
      const float* Wcur = Wb + (t & 1) * kR * kK;
      float2 acc[kK / 2];
#pragma unroll
      for (int j = 0; j < kK / 2; ++j) acc[j] = make_float2(0.f, 0.f);
      if (next) {
        fused_rows<true>(Acur, Wcur, bufs + ((g0 + t + 1) % 3) * kTile + warp * kD + lane, tq, tid, y, acc);
        store_row_sum(acc, lane, Wb + ((t + 1) & 1) * kR * kK + warp * kK);
      } else {
        fused_rows<false>(Acur, Wcur, nullptr, tq, tid, y, acc);
      }
      __syncthreads();  // W(t + 1) complete; tile t's buffer and W(t) free
    }
    if (!aborted && s_abort) aborted = true;  // a wait in the segment's last tile gave up
    if (aborted) break;
    g0 += ntiles;
    float* Pd = a.P + size_t(sg.slot) * kD * pld;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int c = tid + kThr * q;
#pragma unroll
      for (int j = 0; j < kK / 2; j += 2)
        *reinterpret_cast<float4*>(Pd + size_t(c) * pld + 2 * j) =
            make_float4(y[q][j].x, y[q][j].y, y[q][j + 1].x, y[q][j + 1].y);
#pragma unroll
      for (int j = 0; j < kK / 2; ++j) y[q][j] = make_float2(0.f, 0.f);
    }
  }
  // After a wait gave up: the copies issued but not seen to land must land
  // before the CTA's shared memory is released (bounded again).
  if (tid == 0) {
    for (uint32_t g = waited; g < issued; ++g) {
      const uint32_t addr = su32(&full[g % 3]);
      const long long t0 = clock64();
      while (!tc::mbar_try(addr, (g / 3) & 1) && clock64() - t0 < tc::kTimeoutCycles) {
      }
    }
  }
  tc_sync();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
}

constexpr size_t kSmemLimitT = 227 * 1024;

bool geo_tmem(int d, int64_t ld, GeoT* g, size_t* bytes) {
  if (d < 1 || d > 2 * kThr || ld % 4 != 0 || ld / 4 > kThr) return false;
  g->T = (d + 31) / 32;
  int l = static_cast<int>(ld) > 32 * g->T ? static_cast<int>(ld) : 32 * g->T;
  g->lds = (l + 3) / 4 * 4;
  int cols = 32;
  while (cols < 16 * g->T) cols <<= 1;
  g->cols = cols;
  *bytes = size_t(4) * (2 * kR * size_t(g->lds) + kR * kK);
  return cols <= 512 && *bytes <= kSmemLimitT;
}

}  // namespace

bool step_simt_tmem_supported(int d, int64_t ld, int K) {
  GeoT g;
  size_t b;
  return K == kK && geo_tmem(d, ld, &g, &b);
}

cudaError_t launch_step_simt_tmem(const StepArgs& a, cudaStream_t s) {
  GeoT g;
  size_t bytes;
  if (!geo_tmem(a.d, a.ld, &g, &bytes)) return cudaErrorInvalidConfiguration;
  if (a.d == kD && a.ld == kD) {
    const size_t b3 = size_t(4) * (3 * kTile + 2 * kR * kK);
    cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(step_simt_tmem_d1024_kernel));
    if (e != cudaSuccess) return e;
    step_simt_tmem_d1024_kernel<<<a.grid, kThr, b3, s>>>(a);
    return cudaGetLastError();
  }
  auto kern = a.d > kThr ? step_simt_tmem_kernel<2> : step_simt_tmem_kernel<1>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<a.grid, kThr, bytes, s>>>(a, g);
  return cudaGetLastError();
}

}  // namespace lp
