// Fused local power step on the 5th-generation tensor cores for A stored as
// FP8-E4M3 codes with one FP32 scale per row (a_r = s_r q_r):
//   P[slot] = A_seg^T (A_seg Z_i) = Q^T diag(s^2) Q Z_i      (eq. (2), unscaled),
// streaming form (the geometry, ring, interleave and cluster exchange of the
// streaming BF16 kernel in step_tcs.cu).
//
// The scales factor out of both contractions, so the tensor cores only ever see
// the codes.  Every E4M3 value is exactly an FP16 value (3 significand bits,
// exponents 2^-9 .. 2^8), and one cvt.rn.f16x2.e4m3x2 turns two codes into two
// FP16, so:
//   * TMA lands each 128-row x 128-column box of codes (16 KB) in a staging ring;
//   * four converter warps widen it into the FP16 operand layout the MMAs read
//     (SWIZZLE_128B, K-major, 32 KB per unit) in the operand ring;
//   * first pass  D1 += Q_u [Z_hi | Z_lo]  (kind::f16 with FP16 operands; Z
//     split into FP16 hi + lo, 22 significand bits between them);
//   * epilogue    W = D1[:, :K] + D1[:, K:] (cluster-summed), then row r scaled
//     by s_r^2 / S with S = max_r s_r^2 (so |W| never exceeds the FP16 range:
//     |q_r . z| <= 448 sqrt(d)), split into FP16 hi + lo;
//   * second pass D2[b] += Q_u^T [W_hi | W_lo], re-read from L2 and widened
//     again; P = S (D2[:, :K] + D2[:, K:]).
// A row whose s_r^2 / S is below the FP16 range contributes nothing: its
// contribution is below 2^-24 of the largest row's, under FP32 rounding of P.
//
// Roles (384 threads): warp 0 lane 0 issues TMA; warp 1 lane 0 issues MMAs;
// warps 4-7 run the epilogue; warps 8-11 convert; all warps stage Z at segment
// starts.  Every wait is bounded: on expiry the kernel records ST_TIMEOUT, stops
// issuing, waits (bounded) for its own copies in flight, retires its MMAs,
// frees tensor memory and returns.
#include <cuda_fp16.h>

#include "lp_internal.cuh"
#include "tc_ptx.cuh"

namespace lp {
namespace {

using namespace tc;

constexpr int kThreads8 = 384;
constexpr int kConvWarp0 = 8;                // warps 8-11
constexpr int kConvThreads = 128;
constexpr int kUnitBytes = 2 * kChunkBytes;  // 128 rows x 128 columns of FP16 (two 64-column chunks)
constexpr int kStageBytes = kBM * 128;       // 128 rows x 128 E4M3 codes
constexpr int kMaxRing = 8;
constexpr int kSmemLimit = 232448;

enum Tcs8Bar { S_D1FULL0 = 0, S_D1EMPTY0 = 2, S_B2FULL0 = 4, S_B2FREE0 = 6, S_D2FULL = 8, S_REDFULL = 9,
               S_WFULL = 10, S_DONE = 11, S_EPI = 12, S_RING0 = 13 };
// operand ring: FULL[s] = S_RING0 + s, EMPTY[s] = S_RING0 + kMaxRing + s;
// staging ring: FULL[q] = S_RING0 + 2 kMaxRing + q, EMPTY[q] = S_RING0 + 3 kMaxRing + q
constexpr int S_STG0 = S_RING0 + 2 * kMaxRing;
constexpr int kNumBars8 = S_RING0 + 4 * kMaxRing;

struct Tcs8Args {
  const Segment* segs;
  const int* seg_ptr;  // per cluster
  const float* Z;
  int64_t z_stride;
  float* P;
  int d;
  int* status;
  const float* scales;  // per global row
  float smax2;          // S = max_r s_r^2
  int ncd;              // 64-column chunks in this CTA's slice (even)
  int ring;             // operand ring units
  int stage;            // staging ring units
  int lag;
  int hints;
  uint32_t off_stage, off_B1, off_B2, off_W, off_Wrecv, off_bar, tmem_cols;
};

template <typename F>
__device__ __forceinline__ bool for_each_unit8(int ntiles, int U, int lag, F&& fn) {
  for (int t = 0; t <= ntiles; ++t)
    for (int u = 0; u < U + lag; ++u) {
      if (t < ntiles && u < U && !fn(false, t, u)) return false;
      if (t >= 1 && u >= lag && u - lag < U && !fn(true, t - 1, u - lag)) return false;
    }
  return true;
}

// Instruction descriptor: kind::f16 with FP16 A and B, FP32 accumulate, dense.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N, bool a_mn_major, bool b_mn_major) {
  return (1u << 4) | ((a_mn_major ? 1u : 0u) << 15) | ((b_mn_major ? 1u : 0u) << 16) |
         (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t e4m3x2_to_f16x2(uint32_t two_codes) {
  uint32_t r;
  asm("{ .reg .b16 t; cvt.u16.u32 t, %1; cvt.rn.f16x2.e4m3x2 %0, t; }" : "=r"(r) : "r"(two_codes));
  return r;
}

__device__ __forceinline__ uint16_t f16_bits(float x) { return __half_as_ushort(__float2half_rn(x)); }
__device__ __forceinline__ float f16_val(uint16_t b) { return __half2float(__ushort_as_half(b)); }

template <int K>
__global__ void __launch_bounds__(kThreads8, 1)
    step_tcs8_kernel(const __grid_constant__ CUtensorMap map, Tcs8Args a) {
  constexpr int N = 2 * K;
  constexpr uint32_t B2BUF = 2 * N * 128;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sRing = base;
  unsigned char* sStage = base + a.off_stage;
  unsigned char* sB1 = base + a.off_B1;
  unsigned char* sB2 = base + a.off_B2;
  float* sW = reinterpret_cast<float*>(base + a.off_W);
  float* sWrecv = reinterpret_cast<float*>(base + a.off_Wrecv);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + a.off_bar);
  const int R = a.ring, R8 = a.stage;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + kNumBars8);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t crank = cluster_rank();
  const uint32_t CL = cluster_size();
  const int RPC = kBM / static_cast<int>(CL);
  const int cluster_id = blockIdx.x / CL;
  const int DC = 64 * a.ncd;
  const int c0 = static_cast<int>(crank) * DC;
  const int U = a.ncd / 2;  // one unit per 128-column block
  const int LAG = a.lag;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar[S_D1FULL0 + s], 1);
      mbar_init(&bar[S_D1EMPTY0 + s], 4);
      mbar_init(&bar[S_B2FULL0 + s], kBM);
      mbar_init(&bar[S_B2FREE0 + s], 1);
    }
    mbar_init(&bar[S_D2FULL], 1);
    mbar_init(&bar[S_REDFULL], 1);
    mbar_init(&bar[S_WFULL], 1);
    mbar_init(&bar[S_DONE], 1);
    mbar_init(&bar[S_EPI], 128);
    for (int s = 0; s < kMaxRing; ++s) {
      mbar_init(&bar[S_RING0 + s], kConvThreads / 32);  // one arrival per converter warp
      mbar_init(&bar[S_RING0 + kMaxRing + s], 1);        // MMA commit
      mbar_init(&bar[S_STG0 + s], 1);                    // TMA bytes
      mbar_init(&bar[S_STG0 + kMaxRing + s], kConvThreads / 32);
    }
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  auto give_up = [&]() {
    *abort_flag = 1;
    atomicOr(a.status, ST_TIMEOUT);
  };
  auto wait = [&](int id, uint32_t parity, bool cluster_scope) -> bool {
    const uint32_t addr = su32(&bar[id]);
    const long long t0 = clock64();
    while (true) {
      if (cluster_scope ? mbar_try_cluster(addr, parity) : mbar_try(addr, parity)) return true;
      if (*abort_flag) return false;
      if (clock64() - t0 > kTimeoutCycles) {
        give_up();
        return false;
      }
    }
  };

  constexpr uint32_t idesc1 = idesc_f16(128, N, false, false);
  constexpr uint32_t idesc2 = idesc_f16(128, N, true, false);

  const int sb = a.seg_ptr[cluster_id], se = a.seg_ptr[cluster_id + 1];
  uint32_t T = 0;          // tiles before this segment (same in every CTA of the cluster)
  uint32_t epi_phase = 0;  // uses of the epilogue barrier so far
  uint32_t G = 0;          // units before this segment
  uint32_t g_prod_end = 0;
  for (int si = sb; si < se; ++si) {
    const Segment sg = a.segs[si];
    const int ntiles = static_cast<int>((sg.row1 - sg.row0 + kBM - 1) / kBM);

    // ---- stage this slice of Z as [Z_hi | Z_lo]^T in FP16 (N rows x DC, K-major, SWIZZLE_128B)
    __syncthreads();
    if (si == sb || sg.part != a.segs[si - 1].part) {
      const float* Zg = a.Z + a.z_stride * sg.part;
      for (int e = tid; e < DC * K; e += kThreads8) {
        const int c = e / K, j = e % K;
        const float z = (c0 + c < a.d) ? Zg[static_cast<int64_t>(c0 + c) * K + j] : 0.f;
        const uint16_t hi = f16_bits(z);
        const uint16_t lo = f16_bits(z - f16_val(hi));
        *reinterpret_cast<uint16_t*>(sB1 + sw128_off(j, c, N)) = hi;
        *reinterpret_cast<uint16_t*>(sB1 + sw128_off(K + j, c, N)) = lo;
      }
    }
    fence_async_smem();
    __syncthreads();

    if (warp == 0 && lane == 0) {
      // ------------------------------------------------------------ TMA producer (codes into staging)
      uint64_t pol_keep = 0, pol_drop = 0;
      if (a.hints) {
        pol_keep = l2_policy_evict_last();
        pol_drop = l2_policy_evict_first();
      }
      uint32_t g = G;
      for_each_unit8(ntiles, U, LAG, [&](bool second, int t, int u) -> bool {
        const uint32_t q = g % R8;
        if (!wait(S_STG0 + kMaxRing + q, ((g / R8) + 1) & 1, false)) return false;
        mbar_expect_tx(&bar[S_STG0 + q], kStageBytes);
        const int row = static_cast<int>(sg.row0) + t * kBM;
        const uint32_t dst = su32(sStage + q * kStageBytes);
        if (a.hints) tma_load_2d_hint(dst, &map, c0 + 128 * u, row, &bar[S_STG0 + q], second ? pol_drop : pol_keep);
        else tma_load_2d(dst, &map, c0 + 128 * u, row, &bar[S_STG0 + q]);
        ++g;
        return true;
      });
      g_prod_end = g;
    } else if (warp >= kConvWarp0 && warp < kConvWarp0 + kConvThreads / 32) {
      // ------------------------------------------------------------ converters: codes -> FP16 operand
      const int ct = tid - kConvWarp0 * 32;
      uint32_t g = G;
      for_each_unit8(ntiles, U, LAG, [&](bool, int, int) -> bool {
        const uint32_t q = g % R8, s = g % R;
        if (!wait(S_STG0 + q, (g / R8) & 1, false)) return false;
        if (!wait(S_RING0 + kMaxRing + s, ((g / R) + 1) & 1, false)) return false;
        const unsigned char* stg = sStage + q * kStageBytes;
        unsigned char* dst = sRing + s * kUnitBytes;
#pragma unroll 4
        for (int gi = ct; gi < kBM * 16; gi += kConvThreads) {
          const int r = gi >> 4, c8 = gi & 15;  // row, group of 8 columns
          const uint2 codes = *reinterpret_cast<const uint2*>(stg + r * 128 + c8 * 8);
          uint4 out;
          out.x = e4m3x2_to_f16x2(codes.x & 0xFFFFu);
          out.y = e4m3x2_to_f16x2(codes.x >> 16);
          out.z = e4m3x2_to_f16x2(codes.y & 0xFFFFu);
          out.w = e4m3x2_to_f16x2(codes.y >> 16);
          *reinterpret_cast<uint4*>(dst + (c8 >> 3) * kChunkBytes + r * 128 + ((((c8 & 7) ^ (r & 7))) << 4)) = out;
        }
        fence_async_smem();  // the MMAs read these tiles through the async proxy
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&bar[S_RING0 + s]);
          mbar_arrive(&bar[S_STG0 + kMaxRing + q]);
        }
        ++g;
        return true;
      });
    } else if (warp == 1 && lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      uint32_t g = G;
      for_each_unit8(ntiles, U, LAG, [&](bool second, int t, int u) -> bool {
        const uint32_t s = g % R, Tg = T + t, buf = Tg & 1;
        if (!wait(S_RING0 + s, (g / R) & 1, false)) return false;
        if (u == 0) {
          if (!second && !wait(S_D1EMPTY0 + buf, ((Tg >> 1) + 1) & 1, false)) return false;
          if (second && !wait(S_B2FULL0 + buf, (Tg >> 1) & 1, false)) return false;
        }
        tc_fence_after();
        const uint32_t aS = su32(sRing + s * kUnitBytes);
        if (!second) {
          const uint32_t bS = su32(sB1);
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sdesc(aS + j * kChunkBytes + kk * 32, 16, 1024);
              const uint64_t bd = sdesc(bS + (2 * u + j) * N * 128 + kk * 32, 16, 1024);
              mma_bf16(tmem + buf * N, ad, bd, idesc1, (u | j | kk) != 0);
            }
          mma_commit(&bar[S_RING0 + kMaxRing + s]);
          if (u == U - 1) mma_commit(&bar[S_D1FULL0 + buf]);
        } else {
          const uint32_t bS = su32(sB2 + buf * B2BUF);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            const uint64_t ad = sdesc(aS + kk * 2048, kChunkBytes, 1024);
            const uint64_t bd = sdesc(bS + (kk >> 2) * N * 128 + (kk & 3) * 32, 16, 1024);
            mma_bf16(tmem + 2 * N + u * N, ad, bd, idesc2, (t == 0 && kk == 0) ? 0u : 1u);
          }
          mma_commit(&bar[S_RING0 + kMaxRing + s]);
          if (u == U - 1) mma_commit(&bar[S_B2FREE0 + buf]);
        }
        ++g;
        return true;
      });
      mma_commit(&bar[S_D2FULL]);
    } else if (warp >= 4 && warp < 8) {
      // ------------------------------------------------------------ epilogue
      const int r = (warp - 4) * 32 + lane;
      const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
      bool ok = true;
      auto epi_sync = [&]() -> bool {
        mbar_arrive(&bar[S_EPI]);
        return wait(S_EPI, (epi_phase++) & 1, false);
      };
      for (int t = 0; ok && t < ntiles; ++t) {
        const uint32_t Tg = T + t, buf = Tg & 1;
        if (!(ok = wait(S_D1FULL0 + buf, (Tg >> 1) & 1, false))) break;
        tc_fence_after();
        float w[K];
#pragma unroll
        for (int q = 0; q < N / 16; ++q) {
          float v[16];
          tmem_ld16(tmem + lane_base + buf * N + q * 16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = q * 16 + i;
            if (col < K) w[col] = v[i];
            else w[col - K] += v[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[S_D1EMPTY0 + buf]);
        const int64_t grow = sg.row0 + static_cast<int64_t>(t) * kBM + r;
        const bool valid = grow < sg.row1;
        if (!valid) {
#pragma unroll
          for (int j = 0; j < K; ++j) w[j] = 0.f;
        }
        if (CL > 1) {
          const uint32_t rows_bytes = static_cast<uint32_t>(RPC * K * 4);
          if (!(ok = epi_sync())) break;
#pragma unroll
          for (int j = 0; j < K; j += 4)
            *reinterpret_cast<float4*>(sW + wpos<K>(r, j)) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
          fence_async_smem();
          if (!(ok = epi_sync())) break;
          if (r == 0) {
            mbar_expect_tx(&bar[S_REDFULL], (CL - 1) * rows_bytes);
            for (uint32_t o = 0; o < CL; ++o)
              if (o != crank)
                bulk_s2s_cluster(mapa(su32(sWrecv + crank * RPC * K), o), su32(sW + o * RPC * K), rows_bytes,
                                 mapa(su32(&bar[S_REDFULL]), o));
            bulk_commit();
            bulk_wait_read0();
          }
          if (!(ok = wait(S_REDFULL, Tg & 1, true))) break;
          const int per = RPC * K / kBM;
          for (int e = 0; e < per; ++e) {
            const int idx = r * per + e, rl = idx / K, col = idx % K;
            const int own = wpos<K>(static_cast<int>(crank) * RPC + rl, col);
            const int rel = own - static_cast<int>(crank) * RPC * K;
            float sum = 0.f;
            for (uint32_t src = 0; src < CL; ++src) sum += src == crank ? sW[own] : sWrecv[src * RPC * K + rel];
            sW[own] = sum;
          }
          fence_async_smem();
          if (!(ok = epi_sync())) break;
          if (r == 0) {
            mbar_expect_tx(&bar[S_WFULL], (CL - 1) * rows_bytes);
            for (uint32_t dst = 0; dst < CL; ++dst)
              if (dst != crank)
                bulk_s2s_cluster(mapa(su32(sW + crank * RPC * K), dst), su32(sW + crank * RPC * K), rows_bytes,
                                 mapa(su32(&bar[S_WFULL]), dst));
            bulk_commit();
            bulk_wait_read0();
          }
          if (!(ok = wait(S_WFULL, Tg & 1, true))) break;
#pragma unroll
          for (int j = 0; j < K; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(sW + wpos<K>(r, j));
            w[j] = v.x;
            w[j + 1] = v.y;
            w[j + 2] = v.z;
            w[j + 3] = v.w;
          }
        }
        // row scale: W_r <- W_r s_r^2 / S (so the FP16 operand cannot overflow)
        const float sc = valid ? a.scales[grow] : 0.f;
        const float f = sc * sc / a.smax2;
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] *= f;
        if (!(ok = wait(S_B2FREE0 + buf, ((Tg >> 1) + 1) & 1, false))) break;
        unsigned char* B2 = sB2 + buf * B2BUF;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const uint16_t hi = f16_bits(w[j]);
          const uint16_t lo = f16_bits(w[j] - f16_val(hi));
          *reinterpret_cast<uint16_t*>(B2 + sw128_off(j, r, N)) = hi;
          *reinterpret_cast<uint16_t*>(B2 + sw128_off(K + j, r, N)) = lo;
        }
        fence_async_smem();
        mbar_arrive(&bar[S_B2FULL0 + buf]);
      }
      // segment end: Y slice = S (D2[:, :K] + D2[:, K:]) -> P[slot]
      if (ok && wait(S_D2FULL, (si - sb) & 1, false)) {
        tc_fence_after();
        float* Pd = a.P + static_cast<int64_t>(sg.slot) * a.d * K;
        for (int b = 0; b < U; ++b) {
          float y[K];
#pragma unroll
          for (int q = 0; q < N / 16; ++q) {
            float v[16];
            tmem_ld16(tmem + lane_base + 2 * N + b * N + q * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int col = q * 16 + i;
              if (col < K) y[col] = v[i];
              else y[col - K] += v[i];
            }
          }
          const int dcol = c0 + b * 128 + (warp & 3) * 32 + lane;
          if (dcol < a.d) {
            float4* dst = reinterpret_cast<float4*>(Pd + static_cast<int64_t>(dcol) * K);
#pragma unroll
            for (int j = 0; j < K; j += 4)
              dst[j / 4] = make_float4(a.smax2 * y[j], a.smax2 * y[j + 1], a.smax2 * y[j + 2], a.smax2 * y[j + 3]);
          }
        }
        tc_fence_before();
      }
    }
    T += ntiles;
    G += 2u * static_cast<uint32_t>(ntiles) * static_cast<uint32_t>(U);
  }

  // ---- teardown: copies landed (after an abort), MMAs retired, no remote traffic, then free TMEM
  if (warp == 0 && lane == 0) {
    for (uint32_t q = g_prod_end > static_cast<uint32_t>(R8) ? g_prod_end - R8 : 0; q < g_prod_end; ++q) {
      const uint32_t addr = su32(&bar[S_STG0 + q % R8]);
      const long long t0 = clock64();
      while (!mbar_try(addr, (q / R8) & 1) && clock64() - t0 < kTimeoutCycles) {
      }
    }
  }
  if (warp == 1 && lane == 0) mma_commit(&bar[S_DONE]);
  __syncthreads();
  if (warp == 0) {
    const uint32_t addr = su32(&bar[S_DONE]);
    const long long t0 = clock64();
    while (!mbar_try(addr, 0) && clock64() - t0 < kTimeoutCycles) {
    }
  }
  __syncthreads();
  cluster_sync_all();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

template <int K>
cudaLaunchConfig_t tcs8_config(unsigned grid, int cl, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads8, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(cl);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int K>
int tcs8_active_clusters(int cl, size_t smem) {
  if (allow_max_dynamic_smem(reinterpret_cast<const void*>(step_tcs8_kernel<K>)) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tcs8_config<K>(static_cast<unsigned>(cl), cl, smem, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, step_tcs8_kernel<K>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

template <int K>
cudaError_t launch_tcs8_t(const TcsPlan& p, const Tcs8Args& a, cudaStream_t s) {
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(step_tcs8_kernel<K>));
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tcs8_config<K>(static_cast<unsigned>(p.nclusters * p.cluster), p.cluster, p.smem, s, attr);
  const CUtensorMap* m0 = reinterpret_cast<const CUtensorMap*>(p.tmap[0]);
  return cudaLaunchKernelEx(&cfg, step_tcs8_kernel<K>, *m0, a);
}

}  // namespace

namespace {
bool tcs8_plan_slice(int d, int k, int sms, const TcsTuning& tune, int ncd_max, TcsPlan* p);
}  // namespace

// Without a slice width from the tuning, the widest slice that has a plan (fewest
// CTAs per cluster, least W exchange; measured at d = 2,048, k = 32: 512-column
// slices with two staging units beat 256-column slices with four).
bool tcs8_plan(int d, int k, int sms, const TcsTuning& tune, TcsPlan* p) {
  const int K = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  if (tune.slice_cols >= 128) return tcs8_plan_slice(d, k, sms, tune, (tune.slice_cols / 128) * 2, p);
  for (int ncd_max = K == 32 ? 8 : 16; ncd_max >= 4; ncd_max /= 2)
    if (tcs8_plan_slice(d, k, sms, tune, ncd_max, p)) return true;
  return false;
}

namespace {
bool tcs8_plan_slice(int d, int k, int sms, const TcsTuning& tune, int ncd_max, TcsPlan* p) {
  const int K = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  const int N = 2 * K;
  int nc = (d + 63) / 64;
  nc += nc & 1;
  int cl = 1;
  while (cl * ncd_max < nc) cl *= 2;
  if (cl > 8) return false;
  int ncd = (nc + cl - 1) / cl;
  ncd += ncd & 1;
  const uint32_t B1 = static_cast<uint32_t>(ncd) * N * 128;
  const uint32_t B2 = 2u * (2u * N * 128);
  const uint32_t W = cl > 1 ? 128u * K * 4 : 0u;
  const uint32_t bars = kNumBars8 * 8 + 16;
  const int avail = kSmemLimit - 1024 - static_cast<int>(B1 + B2 + 2 * W + bars);
  // operand ring of 32 KB units (two suffice: the converters fill it as fast as the
  // MMAs drain it), the rest to the staging ring that covers load latency
  int ring = 2;
  if (tune.ring_units > 0 && tune.ring_units < ring) ring = tune.ring_units;
  int stage = (avail - ring * kUnitBytes) / kStageBytes;
  if (stage > kMaxRing) stage = kMaxRing;
  if (stage < 2 || ring < 2) return false;
  p->K = K;
  p->planes = 1;
  p->ncd = ncd;
  p->cluster = cl;
  p->ring = ring;
  p->stage = stage;
  int lag = tune.lag_units > 0 ? tune.lag_units : (cl > 1 ? 4 : 2);
  const int U = ncd / 2;
  p->lag = lag < U ? lag : U;
  p->prefetch = 0;
  p->hints = 1;  // first pass evict_last, second pass evict_first
  p->off_stage = static_cast<uint32_t>(ring) * kUnitBytes;
  p->off_B1 = p->off_stage + static_cast<uint32_t>(stage) * kStageBytes;
  p->off_B2 = p->off_B1 + B1;
  p->off_W = p->off_B2 + B2;
  p->off_Wrecv = p->off_W + W;
  p->off_bar = p->off_Wrecv + W;
  p->smem = p->off_bar + bars + 1024;
  const uint32_t used = static_cast<uint32_t>(2 * N + U * N);
  uint32_t cols = 32;
  while (cols < used) cols *= 2;
  if (cols > 512) return false;
  p->tmem_cols = cols;
  if (p->smem > static_cast<size_t>(kSmemLimit)) return false;
  const int active = K == 8 ? tcs8_active_clusters<8>(cl, p->smem)
                            : K == 16 ? tcs8_active_clusters<16>(cl, p->smem) : tcs8_active_clusters<32>(cl, p->smem);
  p->nclusters = sms / cl;
  if (active > 0 && active < p->nclusters) p->nclusters = active;
  p->fp8 = 1;
  return p->nclusters >= 1;
}
}  // namespace

cudaError_t tcs8_encode_map(const void* codes, int64_t n, int d, int64_t ld, TcsPlan* p) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(d), static_cast<cuuint64_t>(n)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld)};
  cuuint32_t box[2] = {128, static_cast<cuuint32_t>(kBM)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(p->tmap[0]), CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                      const_cast<void*>(codes), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step_tcs8(const TcsPlan& p, const Segment* segs, const int* seg_ptr, const float* Z,
                             int64_t z_stride, float* P, int d, const float* scales, float smax2, int* status,
                             cudaStream_t s) {
  Tcs8Args a;
  a.segs = segs;
  a.seg_ptr = seg_ptr;
  a.Z = Z;
  a.z_stride = z_stride;
  a.P = P;
  a.d = d;
  a.status = status;
  a.scales = scales;
  a.smax2 = smax2;
  a.ncd = p.ncd;
  a.ring = p.ring;
  a.stage = p.stage;
  a.lag = p.lag;
  a.hints = p.hints;
  a.off_stage = p.off_stage;
  a.off_B1 = p.off_B1;
  a.off_B2 = p.off_B2;
  a.off_W = p.off_W;
  a.off_Wrecv = p.off_Wrecv;
  a.off_bar = p.off_bar;
  a.tmem_cols = p.tmem_cols;
  if (p.K == 8) return launch_tcs8_t<8>(p, a, s);
  if (p.K == 16) return launch_tcs8_t<16>(p, a, s);
  return launch_tcs8_t<32>(p, a, s);
}

}  // namespace lp
