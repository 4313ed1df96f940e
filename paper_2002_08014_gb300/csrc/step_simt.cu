// Fused local power step, SIMT FP32 path:  P[slot] = A_seg^T (A_seg Z_i)  for
// every row segment, i.e. the unscaled local product of eq. (2), Y_i = M_i Z_i
// with M_i = (1/s_i) A_i^T A_i (the 1/s_i is applied by the reduce kernel).
//
// Each CTA streams its contiguous rows of A exactly once from HBM.  A row tile
// (R rows x d) is staged in shared memory with cp.async (double buffered) and
// used twice from there:
//   phase 1  W = A_tile Z      split-K over d: each thread owns a 4x4 (row, col)
//                              micro-tile over one d-slice; slices are summed
//                              through shared memory into W (R x K);
//   phase 2  Y += A_tile^T W   each thread owns columns c = tid + 256 q of the
//                              d x K partial Y, held in registers for the CTA's
//                              whole segment.
// Z (d x K, FP32) sits in shared memory in a swizzled 4x4-block layout so that
// the phase-1 reads are bank-conflict free.  BF16 and FP8 tiles are widened to
// FP32 in shared memory (FP8 rows times their scale) before the two phases;
// all arithmetic is FP32.
// This file holds the 256-thread kernel (FP8, forced-SIMT BF16, remaining
// shapes) and a 512-thread FP32 kernel; FP32 at 8 < k <= 16 and d <= 1024 goes
// to the kernels with Z_i in tensor memory (step_simt_tmem.cu) instead.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_fp8.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

template <typename T> struct Elem;
template <> struct Elem<float> { static constexpr int kPer16 = 4; };
template <> struct Elem<uint16_t> { static constexpr int kPer16 = 8; };
template <> struct Elem<uint8_t> { static constexpr int kPer16 = 16; };

// Widen one 16-byte chunk of raw elements to FP32 (times `scale`, FP8 only).
__device__ __forceinline__ void widen16(const uint16_t* src, float* dst, float) {
  uint4 v = *reinterpret_cast<const uint4*>(src);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    dst[2 * e] = __uint_as_float(w[e] << 16);
    dst[2 * e + 1] = __uint_as_float(w[e] & 0xFFFF0000u);
  }
}
__device__ __forceinline__ void widen16(const uint8_t* src, float* dst, float scale) {
  uint4 v = *reinterpret_cast<const uint4*>(src);
  const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    __half2_raw lo = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w[e] & 0xFFFFu), __NV_E4M3);
    __half2_raw hi = __nv_cvt_fp8x2_to_halfraw2(static_cast<__nv_fp8x2_storage_t>(w[e] >> 16), __NV_E4M3);
    float2 a = __half22float2(*reinterpret_cast<__half2*>(&lo));
    float2 b = __half22float2(*reinterpret_cast<__half2*>(&hi));
    dst[4 * e + 0] = a.x * scale;
    dst[4 * e + 1] = a.y * scale;
    dst[4 * e + 2] = b.x * scale;
    dst[4 * e + 3] = b.y * scale;
  }
}

// Geometry shared by host and device.
struct Geo {
  int S;      // phase-1 d-slices
  int Qp;     // 4-column quads, padded to a multiple of S
  int lds;    // FP32 smem row stride (floats) of the tile read by the phases
  int ldr;    // raw smem row stride (elements) of the cp.async buffers
};

__host__ __device__ inline Geo make_geo(int d, int64_t ld, int R, int K, int elem) {
  Geo g;
  g.S = 4096 / (R * K);
  int q = (d + 3) / 4;
  g.Qp = g.S * ((q + g.S - 1) / g.S);
  int need = 4 * g.Qp;
  if (elem == 4) {
    int l = static_cast<int>(ld) > need ? static_cast<int>(ld) : need;
    g.lds = (l + 3) / 4 * 4;
    g.ldr = g.lds;
  } else {
    g.lds = need;
    g.ldr = static_cast<int>(ld);
  }
  return g;
}

template <typename Tin, int K, int CPT, int R>
struct Smem {
  // floats
  __host__ __device__ static size_t zs(const Geo& g) { return size_t(4) * g.Qp * K; }
  __host__ __device__ static size_t red(const Geo& g) { return size_t(g.S) * (R * K + 4); }
  __host__ __device__ static size_t ws() { return size_t(R) * K; }
  __host__ __device__ static size_t af(const Geo& g) { return sizeof(Tin) == 4 ? 0 : size_t(R) * g.lds; }
  __host__ __device__ static size_t raw_bytes(const Geo& g) { return size_t(2) * R * g.ldr * sizeof(Tin); }
  __host__ __device__ static size_t bytes(const Geo& g) {
    return raw_bytes(g) + 4 * (zs(g) + red(g) + ws() + af(g)) + 16;
  }
};

template <typename Tin, int K, int CPT, int R>
__global__ void __launch_bounds__(kThreads, 1) step_simt_kernel(StepArgs a, Geo g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  using S_ = Smem<Tin, K, CPT, R>;
  Tin* raw0 = reinterpret_cast<Tin*>(smem_raw);
  Tin* raw1 = raw0 + size_t(R) * g.ldr;
  float* Zs = reinterpret_cast<float*>(smem_raw + S_::raw_bytes(g));
  float* red = Zs + S_::zs(g);
  float* Ws = red + S_::red(g);
  float* Af = Ws + S_::ws();
  constexpr bool kF32 = sizeof(Tin) == 4;
  constexpr int kPer16 = Elem<Tin>::kPer16;

  const int tid = threadIdx.x;
  const int d = a.d;
  const int zld = a.zld > 0 ? a.zld : K, pld = a.pld > 0 ? a.pld : K;
  const Tin* A = static_cast<const Tin*>(a.A);
  const int chunks_per_row = static_cast<int>(a.ld / kPer16);
  const int redst = R * K + 4;

  // phase-1 thread role
  const int S = g.S;
  const int s_id = tid % S;
  const int mt = tid / S;
  const int rg = mt / (K / 4);
  const int jg = mt % (K / 4);
  const int nq = g.Qp / S;

  // Zero the smem columns that cp.async never writes (FP32 tiles read up to 4*Qp).
  if (kF32) {
    for (int r = 0; r < R; ++r)
      for (int c = static_cast<int>(a.ld) + tid; c < g.lds; c += kThreads) {
        reinterpret_cast<float*>(raw0)[r * g.lds + c] = 0.f;
        reinterpret_cast<float*>(raw1)[r * g.lds + c] = 0.f;
      }
  } else {
    for (int r = 0; r < R; ++r)
      for (int c = static_cast<int>(a.ld) + tid; c < g.lds; c += kThreads) Af[r * g.lds + c] = 0.f;
  }

  float y[CPT][K];
#pragma unroll
  for (int q = 0; q < CPT; ++q)
#pragma unroll
    for (int j = 0; j < K; ++j) y[q][j] = 0.f;

  int cur_part = -1;
  const int sb = a.seg_ptr[blockIdx.x], se = a.seg_ptr[blockIdx.x + 1];
  for (int si = sb; si < se; ++si) {
    const Segment sg = a.segs[si];
    const int64_t nrows = sg.row1 - sg.row0;
    const int ntiles = static_cast<int>((nrows + R - 1) / R);

    if (sg.part != cur_part) {
      __syncthreads();  // previous readers of Zs are done
      cur_part = sg.part;
      const float* Zg = a.Z + a.z_stride * sg.part;
      const int n4 = g.Qp * 4 * (K / 4);
      for (int e = tid; e < n4; e += kThreads) {
        const int c = e / (K / 4), jgz = e % (K / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < d) v = *reinterpret_cast<const float4*>(Zg + size_t(c) * zld + 4 * jgz);
        const int q = c >> 2, i = c & 3;
        float* dst = Zs + (size_t(jgz) * g.Qp + q) * 16 + 4 * (i ^ ((q >> 1) & 3));
        *reinterpret_cast<float4*>(dst) = v;
      }
    }

    auto issue = [&](int t, Tin* buf) {
      const int64_t r0 = sg.row0 + int64_t(t) * R;
      const int total = R * chunks_per_row;
      for (int e = tid; e < total; e += kThreads) {
        const int r = e / chunks_per_row, ch = e % chunks_per_row;
        const int64_t grow = r0 + r;
        const bool ok = grow < sg.row1;
        const Tin* src = A + (ok ? grow : sg.row0) * a.ld + int64_t(ch) * kPer16;
        cp_async16(buf + size_t(r) * g.ldr + ch * kPer16, src, ok ? 16 : 0);
      }
      cp_async_commit();
    };

    issue(0, raw0);
    for (int t = 0; t < ntiles; ++t) {
      Tin* cur = (t & 1) ? raw1 : raw0;
      if (t + 1 < ntiles) {
        issue(t + 1, (t & 1) ? raw0 : raw1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();

      const float* T;
      if constexpr (kF32) {
        T = reinterpret_cast<const float*>(cur);
      } else {
        const int64_t r0 = sg.row0 + int64_t(t) * R;
        const int total = R * chunks_per_row;
        for (int e = tid; e < total; e += kThreads) {
          const int r = e / chunks_per_row, ch = e % chunks_per_row;
          float sc = 1.f;
          if (a.scales != nullptr) {
            const int64_t grow = r0 + r;
            sc = grow < sg.row1 ? a.scales[grow] : 0.f;
          }
          float tmp[kPer16];
          widen16(cur + size_t(r) * g.ldr + ch * kPer16, tmp, sc);
#pragma unroll
          for (int v = 0; v < kPer16; v += 4)
            *reinterpret_cast<float4*>(Af + size_t(r) * g.lds + ch * kPer16 + v) =
                make_float4(tmp[v], tmp[v + 1], tmp[v + 2], tmp[v + 3]);
        }
        __syncthreads();
        T = Af;
      }

      // ---- phase 1: W = T Z (split over d-slices) ----
      float acc[4][4];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[r][b] = 0.f;
      const float* Trow = T + size_t(4 * rg) * g.lds;
      const float* Zblk = Zs + size_t(jg) * g.Qp * 16;
#pragma unroll 2
      for (int u = 0; u < nq; ++u) {
        const int q = s_id + S * u;
        float4 av[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) av[r] = *reinterpret_cast<const float4*>(Trow + size_t(r) * g.lds + 4 * q);
        const float* zb = Zblk + size_t(q) * 16;
        const int f = (q >> 1) & 3;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 z = *reinterpret_cast<const float4*>(zb + 4 * (i ^ f));
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            const float ai = i == 0 ? av[r].x : i == 1 ? av[r].y : i == 2 ? av[r].z : av[r].w;
            acc[r][0] = fmaf(ai, z.x, acc[r][0]);
            acc[r][1] = fmaf(ai, z.y, acc[r][1]);
            acc[r][2] = fmaf(ai, z.z, acc[r][2]);
            acc[r][3] = fmaf(ai, z.w, acc[r][3]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        *reinterpret_cast<float4*>(red + size_t(s_id) * redst + (4 * rg + r) * K + 4 * jg) =
            make_float4(acc[r][0], acc[r][1], acc[r][2], acc[r][3]);
      __syncthreads();
      for (int e = tid; e < R * K; e += kThreads) {
        float sum = 0.f;
        for (int s2 = 0; s2 < S; ++s2) sum += red[size_t(s2) * redst + e];
        Ws[e] = sum;
      }
      __syncthreads();

      // ---- phase 2: Y += T^T W ----
#pragma unroll 2
      for (int r = 0; r < R; ++r) {
        float w[K];
#pragma unroll
        for (int j = 0; j < K; j += 4) {
          const float4 v = *reinterpret_cast<const float4*>(Ws + r * K + j);
          w[j] = v.x; w[j + 1] = v.y; w[j + 2] = v.z; w[j + 3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const int c = tid + kThreads * q;
          if (c < d) {
            const float av = T[size_t(r) * g.lds + c];
#pragma unroll
            for (int j = 0; j < K; ++j) y[q][j] = fmaf(av, w[j], y[q][j]);
          }
        }
      }
      __syncthreads();
    }

    // flush this segment's partial
    float* Pd = a.P + size_t(sg.slot) * d * pld;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int c = tid + kThreads * q;
      if (c < d) {
#pragma unroll
        for (int j = 0; j < K; j += 4)
          *reinterpret_cast<float4*>(Pd + size_t(c) * pld + j) = make_float4(y[q][j], y[q][j + 1], y[q][j + 2], y[q][j + 3]);
      }
#pragma unroll
      for (int j = 0; j < K; ++j) y[q][j] = 0.f;
    }
  }
}

// ---------------------------------------------------------------------------
// FP32 kernel, second design (512 threads).  Phase 1 maps a warp onto all
// (R/4) x (K/4) micro-tiles of W for 32/MT d-slices, so lanes that share rows
// (or output columns) read the same shared-memory words and the reads
// broadcast: about 8 wavefronts per 64 FMAs instead of 24.  The slices of a
// warp are combined with shuffles, the warps through shared memory.  A's
// shared row stride is 8 floats past a multiple of 32 and Z's 4-row blocks
// swap row pairs on odd quads, which keeps both read patterns conflict free.
// Phase 2 is the design above with two columns per thread.
constexpr int kThreads2 = 512;

struct Geo2 {
  int S;    // d-slices (16 warps x slices per warp)
  int Qp;   // quads, padded to a multiple of S
  int lds;  // A tile row stride (floats)
};

template <int K, int R>
struct Simt2 {
  static constexpr int MT = (R / 4) * (K / 4);  // micro-tiles
  static constexpr int SPW = 32 / MT;           // slices per warp
  static_assert(MT <= 32 && 32 % MT == 0, "micro-tiles must tile a warp");
  static Geo2 geo(int d, int64_t ld) {
    Geo2 g;
    g.S = 16 * SPW;
    const int q = (d + 3) / 4;
    g.Qp = g.S * ((q + g.S - 1) / g.S);
    int l = static_cast<int>(ld) > 4 * g.Qp ? static_cast<int>(ld) : 4 * g.Qp;
    g.lds = (l + 31) / 32 * 32 + 8;
    return g;
  }
  static size_t bytes(const Geo2& g) {
    return size_t(4) * (2 * R * g.lds + 4 * g.Qp * K + 16 * MT * 16 + R * K) + 16;
  }
};

template <int K, int CPT, int R>
__global__ void __launch_bounds__(kThreads2, 1) step_simt2_kernel(StepArgs a, Geo2 g) {
  using G2 = Simt2<K, R>;
  constexpr int MT = G2::MT, SPW = G2::SPW, RG = R / 4;
  extern __shared__ __align__(16) float sm2[];
  float* buf0 = sm2;
  float* buf1 = buf0 + R * g.lds;
  float* Zs = buf1 + R * g.lds;
  float* red = Zs + 4 * g.Qp * K;
  float* Ws = red + 16 * MT * 16;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int d = a.d;
  const int zld = a.zld > 0 ? a.zld : K, pld = a.pld > 0 ? a.pld : K;
  const float* A = static_cast<const float*>(a.A);
  const int cpr = static_cast<int>(a.ld / 4);  // 16-byte chunks per row
  // row-tile copy plan: rows per pass, this thread's first row and chunk (cpr <= threads)
  const int cp_rstep = kThreads2 / cpr, cp_r0 = tid / cpr, cp_ch = tid % cpr;
  const int sp = lane / MT, mt = lane % MT;
  const int rg = mt / (K / 4), jg = mt % (K / 4);
  const int s_id = warp * SPW + sp;
  const int nq = g.Qp / g.S;

  for (int r = 0; r < R; ++r)
    for (int c = static_cast<int>(a.ld) + tid; c < g.lds; c += kThreads2) {
      buf0[r * g.lds + c] = 0.f;
      buf1[r * g.lds + c] = 0.f;
    }

  float2 y[CPT][K / 2];
#pragma unroll
  for (int q = 0; q < CPT; ++q)
#pragma unroll
    for (int j = 0; j < K / 2; ++j) y[q][j] = make_float2(0.f, 0.f);

  int cur_part = -1;
  const int sb = a.seg_ptr[blockIdx.x], se = a.seg_ptr[blockIdx.x + 1];
  for (int si = sb; si < se; ++si) {
    const Segment sg = a.segs[si];
    const int ntiles = static_cast<int>((sg.row1 - sg.row0 + R - 1) / R);
    // thread tid copies chunk cp_ch of rows cp_r0, cp_r0 + cp_rstep, ... (rows past
    // the segment are zero-filled)
    auto issue = [&](int t, float* buf) {
      const int64_t r0 = sg.row0 + int64_t(t) * R;
      if (cp_r0 < cp_rstep)
        for (int r = cp_r0; r < R; r += cp_rstep) {
          const int64_t grow = r0 + r;
          const bool ok = grow < sg.row1;
          cp_async16(buf + size_t(r) * g.lds + cp_ch * 4, A + (ok ? grow : sg.row0) * a.ld + int64_t(cp_ch) * 4,
                     ok ? 16 : 0);
        }
      cp_async_commit();
    };
    issue(0, buf0);  // the first tile loads while Z_i is staged
    if (sg.part != cur_part) {
      __syncthreads();
      cur_part = sg.part;
      const float* Zg = a.Z + a.z_stride * sg.part;
      for (int e = tid; e < g.Qp * 4 * (K / 4); e += kThreads2) {
        const int c = e / (K / 4), jz = e % (K / 4);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (c < d) v = *reinterpret_cast<const float4*>(Zg + size_t(c) * zld + 4 * jz);
        const int q = c >> 2, i = c & 3;
        *reinterpret_cast<float4*>(Zs + (size_t(q) * 4 + (i ^ (q & 1))) * K + 4 * jz) = v;
      }
    }
    for (int t = 0; t < ntiles; ++t) {
      const float* T = (t & 1) ? buf1 : buf0;
      if (t + 1 < ntiles) {
        issue(t + 1, (t & 1) ? buf0 : buf1);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncthreads();

      // ---- phase 1: rows {rg + RG*aa}, columns {4jg .. 4jg+3}, quads q = s_id + S*u
      // (packed FP32 FMAs: two output columns per instruction)
      float2 acc[4][2];
#pragma unroll
      for (int aa = 0; aa < 4; ++aa) {
        acc[aa][0] = make_float2(0.f, 0.f);
        acc[aa][1] = make_float2(0.f, 0.f);
      }
#pragma unroll 2
      for (int u = 0; u < nq; ++u) {
        const int q = s_id + g.S * u;
        float4 av[4];
#pragma unroll
        for (int aa = 0; aa < 4; ++aa)
          av[aa] = *reinterpret_cast<const float4*>(T + size_t(rg + RG * aa) * g.lds + 4 * q);
        const float* zq = Zs + size_t(q) * 4 * K + 4 * jg;
        const int sw = q & 1;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float4 z = *reinterpret_cast<const float4*>(zq + (i ^ sw) * K);
          const float2 z01 = make_float2(z.x, z.y), z23 = make_float2(z.z, z.w);
#pragma unroll
          for (int aa = 0; aa < 4; ++aa) {
            const float ai = i == 0 ? av[aa].x : i == 1 ? av[aa].y : i == 2 ? av[aa].z : av[aa].w;
            const float2 a2 = make_float2(ai, ai);
            acc[aa][0] = __ffma2_rn(a2, z01, acc[aa][0]);
            acc[aa][1] = __ffma2_rn(a2, z23, acc[aa][1]);
          }
        }
      }
      // slices of this warp -> lane group sp == 0
#pragma unroll
      for (int off = MT; off < 32; off <<= 1)
#pragma unroll
        for (int aa = 0; aa < 4; ++aa)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            acc[aa][h].x += __shfl_xor_sync(0xffffffffu, acc[aa][h].x, off);
            acc[aa][h].y += __shfl_xor_sync(0xffffffffu, acc[aa][h].y, off);
          }
      // per-warp partial W in row-major R x K blocks: a micro-tile row is 16
      // contiguous bytes and the lanes' rows are contiguous, so both the writes
      // and the column-wise reads below are conflict free
      if (sp == 0) {
#pragma unroll
        for (int aa = 0; aa < 4; ++aa)
          *reinterpret_cast<float4*>(red + (size_t(warp) * R + rg + RG * aa) * K + 4 * jg) =
              make_float4(acc[aa][0].x, acc[aa][0].y, acc[aa][1].x, acc[aa][1].y);
      }
      __syncthreads();
      for (int e = tid; e < R * K; e += kThreads2) {
        float sum = 0.f;
#pragma unroll 4
        for (int w = 0; w < 16; ++w) sum += red[size_t(w) * R * K + e];
        Ws[e] = sum;
      }
      __syncthreads();

      // ---- phase 2: Y += T^T W (packed FP32 FMAs)
#pragma unroll 2
      for (int r = 0; r < R; ++r) {
        float2 w[K / 2];
#pragma unroll
        for (int j = 0; j < K; j += 4) {
          const float4 v = *reinterpret_cast<const float4*>(Ws + r * K + j);
          w[j / 2] = make_float2(v.x, v.y);
          w[j / 2 + 1] = make_float2(v.z, v.w);
        }
#pragma unroll
        for (int q = 0; q < CPT; ++q) {
          const int c = tid + kThreads2 * q;
          if (c < d) {
            const float av = T[size_t(r) * g.lds + c];
            const float2 a2 = make_float2(av, av);
#pragma unroll
            for (int j = 0; j < K / 2; ++j) y[q][j] = __ffma2_rn(a2, w[j], y[q][j]);
          }
        }
      }
      __syncthreads();
    }
    float* Pd = a.P + size_t(sg.slot) * d * pld;
#pragma unroll
    for (int q = 0; q < CPT; ++q) {
      const int c = tid + kThreads2 * q;
      if (c < d) {
#pragma unroll
        for (int j = 0; j < K / 2; j += 2)
          *reinterpret_cast<float4*>(Pd + size_t(c) * pld + 2 * j) = make_float4(y[q][j].x, y[q][j].y, y[q][j + 1].x,
                                                                              y[q][j + 1].y);
      }
#pragma unroll
      for (int j = 0; j < K / 2; ++j) y[q][j] = make_float2(0.f, 0.f);
    }
  }
}

constexpr size_t kSmemLimit2 = 227 * 1024;

template <int K, int CPT, int R>
cudaError_t launch_two(const StepArgs& a, const Geo2& g, size_t bytes, cudaStream_t s) {
  auto kern = step_simt2_kernel<K, CPT, R>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<a.grid, kThreads2, bytes, s>>>(a, g);
  return cudaGetLastError();
}

// Chooses the row tile (16, else 8) whose shared memory fits; returns false if none.
template <int K>
bool simt2_pick(int d, int64_t ld, int* R, Geo2* g, size_t* bytes) {
  if (d > 2 * kThreads2 || ld / 4 > kThreads2 || (d + kThreads2 - 1) / kThreads2 * K > 64) return false;
  const Geo2 g16 = Simt2<K, 16>::geo(d, ld);
  if (32 % Simt2<K, 16>::MT == 0 && Simt2<K, 16>::bytes(g16) <= kSmemLimit2) {
    *R = 16; *g = g16; *bytes = Simt2<K, 16>::bytes(g16);
    return true;
  }
  const Geo2 g8 = Simt2<K, 8>::geo(d, ld);
  if (Simt2<K, 8>::bytes(g8) <= kSmemLimit2) {
    *R = 8; *g = g8; *bytes = Simt2<K, 8>::bytes(g8);
    return true;
  }
  return false;
}

template <int K>
cudaError_t launch_v2(const StepArgs& a, cudaStream_t s) {
  int R;
  Geo2 g;
  size_t bytes;
  if (!simt2_pick<K>(a.d, a.ld, &R, &g, &bytes)) return cudaErrorInvalidConfiguration;
  const bool two = a.d > kThreads2;
  if (R == 16) return two ? launch_two<K, 2, 16>(a, g, bytes, s) : launch_two<K, 1, 16>(a, g, bytes, s);
  return two ? launch_two<K, 2, 8>(a, g, bytes, s) : launch_two<K, 1, 8>(a, g, bytes, s);
}

bool v2_supported(int d, int64_t ld, int K) {
  int R;
  Geo2 g;
  size_t b;
  switch (K) {
    case 8: return simt2_pick<8>(d, ld, &R, &g, &b);
    case 16: return simt2_pick<16>(d, ld, &R, &g, &b);
    case 32: return simt2_pick<32>(d, ld, &R, &g, &b);
  }
  return false;
}

cudaError_t launch_f32(const StepArgs& a, int K, cudaStream_t s) {
  if (v2_supported(a.d, a.ld, K)) {
    switch (K) {
      case 8: return launch_v2<8>(a, s);
      case 16: return launch_v2<16>(a, s);
      case 32: return launch_v2<32>(a, s);
    }
  }
  return cudaErrorInvalidConfiguration;
}

template <typename Tin, int K, int CPT, int R>
cudaError_t launch_one(const StepArgs& a, cudaStream_t s) {
  const Geo g = make_geo(a.d, a.ld, R, K, sizeof(Tin));
  const size_t bytes = Smem<Tin, K, CPT, R>::bytes(g);
  auto kern = step_simt_kernel<Tin, K, CPT, R>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  kern<<<a.grid, kThreads, bytes, s>>>(a, g);
  return cudaGetLastError();
}

constexpr size_t kSmemLimit = 227 * 1024;

template <typename Tin, int K, int CPT>
cudaError_t launch_r(const StepArgs& a, cudaStream_t s) {
  const Geo g16 = make_geo(a.d, a.ld, 16, K, sizeof(Tin));
  if (Smem<Tin, K, CPT, 16>::bytes(g16) <= kSmemLimit) return launch_one<Tin, K, CPT, 16>(a, s);
  const Geo g8 = make_geo(a.d, a.ld, 8, K, sizeof(Tin));
  if (Smem<Tin, K, CPT, 8>::bytes(g8) <= kSmemLimit) return launch_one<Tin, K, CPT, 8>(a, s);
  return cudaErrorInvalidConfiguration;
}

template <typename Tin, int K>
cudaError_t launch_cpt(const StepArgs& a, cudaStream_t s) {
  const int cpt = (a.d + kThreads - 1) / kThreads;
  if (cpt <= 1) return launch_r<Tin, K, 1>(a, s);
  if (cpt <= 2) return launch_r<Tin, K, 2>(a, s);
  if (cpt <= 4) return launch_r<Tin, K, 4>(a, s);
  return cudaErrorInvalidConfiguration;
}

template <typename Tin>
cudaError_t launch_k(const StepArgs& a, int K, cudaStream_t s) {
  switch (K) {
    case 8: return launch_cpt<Tin, 8>(a, s);
    case 16: return launch_cpt<Tin, 16>(a, s);
    case 32: return launch_cpt<Tin, 32>(a, s);
    default: return cudaErrorInvalidConfiguration;
  }
}

template <typename Tin>
size_t smem_for(int d, int64_t ld, int K, int* rows) {
  const int cpt = (d + kThreads - 1) / kThreads;
  if (cpt > 4 || (K != 8 && K != 16 && K != 32)) return 0;
  for (int R : {16, 8}) {
    const Geo g = make_geo(d, ld, R, K, sizeof(Tin));
    // Smem::bytes does not depend on CPT.
    size_t b;
    if (K == 8) b = R == 16 ? Smem<Tin, 8, 1, 16>::bytes(g) : Smem<Tin, 8, 1, 8>::bytes(g);
    else if (K == 16) b = R == 16 ? Smem<Tin, 16, 1, 16>::bytes(g) : Smem<Tin, 16, 1, 8>::bytes(g);
    else b = R == 16 ? Smem<Tin, 32, 1, 16>::bytes(g) : Smem<Tin, 32, 1, 8>::bytes(g);
    if (b <= kSmemLimit) {
      if (rows) *rows = R;
      return b;
    }
  }
  return 0;
}

}  // namespace

cudaError_t launch_step_simt(const StepArgs& a, lp_dtype dtype, int K, cudaStream_t s) {
  switch (dtype) {
    case LP_F32:
      if (step_simt_tmem_supported(a.d, a.ld, K)) return launch_step_simt_tmem(a, s);
      return v2_supported(a.d, a.ld, K) ? launch_f32(a, K, s) : launch_k<float>(a, K, s);
    case LP_BF16: return launch_k<uint16_t>(a, K, s);
    case LP_FP8_E4M3: return launch_k<uint8_t>(a, K, s);
  }
  return cudaErrorInvalidConfiguration;
}

size_t step_simt_smem(int d, int64_t ld, lp_dtype dtype, int K, int* rows_per_tile) {
  switch (dtype) {
    case LP_F32: return smem_for<float>(d, ld, K, rows_per_tile);
    case LP_BF16: return smem_for<uint16_t>(d, ld, K, rows_per_tile);
    case LP_FP8_E4M3: return smem_for<uint8_t>(d, ld, K, rows_per_tile);
  }
  return 0;
}

}  // namespace lp
