// Fused local power step on the 5th-generation tensor cores (tcgen05), for A
// stored in BF16:  P[slot] = A_seg^T (A_seg Z_i)  (the unscaled local product of
// eq. (2)), FP32 accumulation in tensor memory.
//
// Geometry.  Rows are processed in tiles of 128 (the MMA's M).  The d columns
// are split over a thread-block cluster of CL CTAs (CL in {1, 2, 4, 8}); CTA c
// owns columns [c*DC, (c+1)*DC) with DC = 64*NCH, so one row tile of its slice
// (128 x DC BF16 = 16*NCH KB) stays resident in shared memory for both
// contractions and A is read from HBM exactly once.
//
// Per tile (all CTAs of a cluster walk the same row tiles):
//   TMA    A tile slice -> smem (SWIZZLE_128B boxes of 64 columns x 128 rows)
//   C1     D1 = A_slice [Z_hi | Z_lo]          M=128, N=2K, K-major A and B
//   epi    W_partial = D1[:, :K] + D1[:, K:]; summed over the cluster through
//          distributed shared memory (owner CTAs reduce 128/CL rows each);
//          rows outside the segment are zeroed; W -> [W_hi | W_lo] in BF16
//   C2     D2[b] += A_slice^T [W_hi | W_lo]    M=128 d-columns, N=2K, MN-major A
// After a segment's last tile, Y = D2[:, :K] + D2[:, K:] is written to P.
// The hi/lo splits keep Z and W at about 16 significant bits, so the products
// carry FP32-level accuracy although the tensor cores take BF16 operands.
//
// Roles (256 threads): warp 0 lane 0 issues TMA; warp 1 lane 0 issues MMAs;
// warps 4-7 (one per TMEM lane quadrant) run the epilogue; every warp helps
// stage Z at segment starts.  Every mbarrier wait is bounded: on expiry the
// kernel records ST_TIMEOUT, stops issuing work and unwinds.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "lp_internal.cuh"
#include "tc_ptx.cuh"

namespace lp {
namespace {

using namespace tc;


struct TcArgs {
  const Segment* segs;
  const int* seg_ptr;  // per cluster
  const float* Z;
  int64_t z_stride;
  float* P;
  int d;
  int* status;
};

template <int K, int NCH>
struct TcLayout {
  static constexpr int N = 2 * K;
  static constexpr int DC = 64 * NCH;
  static constexpr int STAGE = NCH * kChunkBytes;
  static constexpr int B1 = NCH * N * 128;
  static constexpr int B2 = 2 * N * 128;
  static constexpr int NB2BUF = K == 32 ? 1 : 2;  // W operand buffers (one at K = 32 to fit shared memory)
  static constexpr int NB2 = NCH / 2;
  // Cluster sum of the row products: all-gather (one shared-memory trip) for
  // K <= 16 and clusters of up to 4 CTAs, else reduce-scatter + broadcast.
  static constexpr bool AG = K <= 16;
  static constexpr int WBYTES = kBM * K * 4;                    // one 128 x K FP32 block (wpos layout)
  static constexpr int RECV = AG ? 2 * 3 * WBYTES : WBYTES;      // AG: 2 parities x 3 peers
  static constexpr int off_A = 0;
  static constexpr int off_B1 = off_A + 2 * STAGE;
  static constexpr int off_B2 = off_B1 + B1;
  static constexpr int off_W = off_B2 + NB2BUF * B2;   // this CTA's partial rows (RS: then the owned sums)
  static constexpr int off_Wrecv = off_W + WBYTES;      // peers' partials
  static constexpr int off_bar = off_Wrecv + RECV;
  static constexpr int kBars = 18;
  static constexpr int bytes = off_bar + kBars * 8 + 16;
  static constexpr int alloc_bytes = bytes + 1024;  // room to align the base to 1024
  static constexpr uint32_t tmem_used = 2 * N + NB2 * N;
  static constexpr uint32_t tmem_cols = tmem_used <= 32 ? 32 : tmem_used <= 64 ? 64 : tmem_used <= 128 ? 128
                                        : tmem_used <= 256 ? 256 : 512;
};

enum BarId { B_FULL0 = 0, B_EMPTY0 = 2, B_D1FULL0 = 4, B_D1EMPTY0 = 6, B_B2FULL0 = 8, B_B2FREE0 = 10, B_D2FULL = 12,
             B_REDFULL = 13, B_WFULL = 14, B_DONE = 15, B_RED1 = 16, B_EPI = 17 };

template <int K, int NCH>
__global__ void __launch_bounds__(kThreads, 1) step_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  using L = TcLayout<K, NCH>;
  constexpr int N = L::N;
  constexpr int DC = L::DC;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sA = base + L::off_A;
  unsigned char* sB1 = base + L::off_B1;
  unsigned char* sB2 = base + L::off_B2;
  float* sW = reinterpret_cast<float*>(base + L::off_W);
  float* sWrecv = reinterpret_cast<float*>(base + L::off_Wrecv);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + L::off_bar);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + L::kBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t crank = cluster_rank();
  const uint32_t CL = cluster_size();
  const int RPC = kBM / static_cast<int>(CL);
  const int cluster_id = blockIdx.x / CL;
  const int c0 = static_cast<int>(crank) * DC;

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar[B_FULL0 + s], 1);
      mbar_init(&bar[B_EMPTY0 + s], 1);
      mbar_init(&bar[B_D1FULL0 + s], 1);
      mbar_init(&bar[B_D1EMPTY0 + s], 4);
      mbar_init(&bar[B_B2FULL0 + s], kBM);
      mbar_init(&bar[B_B2FREE0 + s], 1);
    }
    mbar_init(&bar[B_D2FULL], 1);
    mbar_init(&bar[B_REDFULL], 1);  // local expect_tx + bytes of the peers' partial rows
    mbar_init(&bar[B_RED1], 1);     // all-gather, odd tiles
    mbar_init(&bar[B_EPI], 128);    // barrier of the four epilogue warps (bounded waits)
    mbar_init(&bar[B_WFULL], 1);    // local expect_tx + bytes of the owners' summed rows
    mbar_init(&bar[B_DONE], 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"(L::tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // every CTA's barriers exist before any remote arrive
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  auto wait = [&](int id, uint32_t parity, bool cluster_scope) -> bool {
    const uint32_t addr = su32(&bar[id]);
    const long long t0 = clock64();
    while (true) {
      if (cluster_scope ? mbar_try_cluster(addr, parity) : mbar_try(addr, parity)) return true;
      if (*abort_flag) return false;
      if (clock64() - t0 > kTimeoutCycles) {
        *abort_flag = 1;
        atomicOr(a.status, ST_TIMEOUT);
        return false;
      }
    }
  };

  constexpr uint32_t idesc1 = idesc_bf16(128, N, false, false);
  constexpr uint32_t idesc2 = idesc_bf16(128, N, true, false);

  const int sb = a.seg_ptr[cluster_id], se = a.seg_ptr[cluster_id + 1];
  uint32_t T = 0;  // tiles processed so far (identical in every CTA of the cluster)
  uint32_t epi_phase = 0;  // uses of the epilogue barrier so far (epilogue threads)
  for (int si = sb; si < se; ++si) {
    const Segment sg = a.segs[si];
    const int ntiles = static_cast<int>((sg.row1 - sg.row0 + kBM - 1) / kBM);

    // ---- stage Z slice as [Z_hi | Z_lo]^T (N rows x DC, K-major, SWIZZLE_128B)
    __syncthreads();
    if (si == sb || sg.part != a.segs[si - 1].part) {  // consecutive pieces of a partition share Z_i
      const float* Zg = a.Z + a.z_stride * sg.part;
      for (int e = tid; e < DC * K; e += kThreads) {
        const int c = e / K, j = e % K;
        const float z = (c0 + c < a.d) ? Zg[static_cast<int64_t>(c0 + c) * K + j] : 0.f;
        const uint16_t hi = bf16_bits(z);
        const uint16_t lo = bf16_bits(z - bf16_val(hi));
        *reinterpret_cast<uint16_t*>(sB1 + sw128_off(j, c, N)) = hi;
        *reinterpret_cast<uint16_t*>(sB1 + sw128_off(K + j, c, N)) = lo;
      }
    }
    fence_async_smem();
    __syncthreads();

    if (warp == 0 && lane == 0) {
      // ------------------------------------------------------------ TMA producer
      for (int t = 0; t < ntiles; ++t) {
        const uint32_t Tg = T + t, s = Tg & 1;
        if (!wait(B_EMPTY0 + s, ((Tg >> 1) + 1) & 1, false)) break;
        mbar_expect_tx(&bar[B_FULL0 + s], L::STAGE);
        const int row = static_cast<int>(sg.row0) + t * kBM;
        for (int ch = 0; ch < NCH; ++ch)
          tma_load_2d(su32(sA + s * L::STAGE + ch * kChunkBytes), &tmap, c0 + ch * 64, row, &bar[B_FULL0 + s]);
      }
    } else if (warp == 1 && lane == 0) {
      // ------------------------------------------------------------ MMA issuer
      // C1 of tile t+1 and C2 of tile t wait on different events (A landing vs W
      // ready); the issuer polls both and issues whichever is ready first.
      auto c1 = [&](uint32_t Tg) {
        const uint32_t s = Tg & 1, b = Tg & 1;
        const uint32_t aS = su32(sA + s * L::STAGE), bS = su32(sB1);
#pragma unroll
        for (int ch = 0; ch < NCH; ++ch)
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {
            const uint64_t ad = sdesc(aS + ch * kChunkBytes + kk * 32, 16, 1024);
            const uint64_t bd = sdesc(bS + ch * N * 128 + kk * 32, 16, 1024);
            mma_bf16(tmem + b * N, ad, bd, idesc1, (ch | kk) != 0);
          }
        mma_commit(&bar[B_D1FULL0 + b]);
      };
      auto c2 = [&](uint32_t Tg, bool first) {
        const uint32_t s = Tg & 1, bb = Tg % L::NB2BUF;
        const uint32_t aS = su32(sA + s * L::STAGE), bS = su32(sB2 + bb * L::B2);
#pragma unroll
        for (int mb = 0; mb < L::NB2; ++mb)
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            // A^T: M = 128 d-columns (two 64-column chunks, LBO apart), K = 16 rows (two 8-row groups, SBO apart)
            const uint64_t ad = sdesc(aS + (2 * mb) * kChunkBytes + kk * 2048, kChunkBytes, 1024);
            const uint64_t bd = sdesc(bS + (kk >> 2) * N * 128 + (kk & 3) * 32, 16, 1024);
            mma_bf16(tmem + 2 * N + mb * N, ad, bd, idesc2, (first && kk == 0) ? 0u : 1u);
          }
        mma_commit(&bar[B_EMPTY0 + s]);
        mma_commit(&bar[B_B2FREE0 + bb]);
      };
      auto ready = [&](int id, uint32_t parity) { return mbar_test(su32(&bar[id]), parity); };
      int n1 = 0, n2 = 0;  // tiles of this segment whose C1 / C2 have been issued
      long long last = clock64();
      while (n2 < ntiles) {
        bool progressed = false;
        if (n1 < ntiles && n1 <= n2 + 1) {
          const uint32_t Tg = T + n1;
          if (ready(B_FULL0 + (Tg & 1), (Tg >> 1) & 1) && ready(B_D1EMPTY0 + (Tg & 1), ((Tg >> 1) + 1) & 1)) {
            tc_fence_after();
            c1(Tg);
            ++n1;
            progressed = true;
          }
        }
        if (n2 < n1) {
          const uint32_t Tg = T + n2;
          if (ready(B_B2FULL0 + Tg % L::NB2BUF, (Tg / L::NB2BUF) & 1)) {
            tc_fence_after();
            c2(Tg, n2 == 0);
            ++n2;
            progressed = true;
          }
        }
        if (progressed) {
          last = clock64();
        } else if (*abort_flag) {
          break;
        } else if (clock64() - last > kTimeoutCycles) {
          *abort_flag = 1;
          atomicOr(a.status, ST_TIMEOUT);
          break;
        }
      }
      mma_commit(&bar[B_D2FULL]);
    } else if (warp >= 4) {
      // ------------------------------------------------------------ epilogue
      const int r = (warp - 4) * 32 + lane;
      const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
      bool ok = true;
      // Barrier of the 128 epilogue threads on an mbarrier with a bounded wait
      // (a named barrier could hang if some threads left the loop on an abort).
      auto epi_sync = [&]() -> bool {
        mbar_arrive(&bar[B_EPI]);
        return wait(B_EPI, (epi_phase++) & 1, false);
      };
      for (int t = 0; ok && t < ntiles; ++t) {
        const uint32_t Tg = T + t, b = Tg & 1;
        if (!(ok = wait(B_D1FULL0 + b, (Tg >> 1) & 1, false))) break;
        tc_fence_after();
        float w[K];
#pragma unroll
        for (int q = 0; q < N / 16; ++q) {
          float v[16];
          tmem_ld16(tmem + lane_base + b * N + q * 16, v);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int col = q * 16 + i;
            if (col < K) w[col] = v[i];
            else w[col - K] += v[i];
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[B_D1EMPTY0 + b]);
        const bool valid = sg.row0 + static_cast<int64_t>(t) * kBM + r < sg.row1;
        if (!valid) {
#pragma unroll
          for (int j = 0; j < K; ++j) w[j] = 0.f;
        }
        if (CL > 1 && L::AG && CL <= 4) {
          // All-gather: every CTA ships its 128 partial rows to each peer (bulk
          // copies counted in bytes on the peer's barrier for this tile's
          // parity) and then sums all CL partials of its own rows in source-rank
          // order.  A peer can refill a parity's slots only after this CTA has
          // sent its next tile, i.e. after it finished reading them.
          const uint32_t par = Tg & 1;
          const int rb = par ? B_RED1 : B_REDFULL;
          const uint32_t blk = static_cast<uint32_t>(L::WBYTES);
          if (!(ok = epi_sync())) break;  // the previous tile's bulk copies have read sW (r == 0 waited)
#pragma unroll
          for (int j = 0; j < K; j += 4)
            *reinterpret_cast<float4*>(sW + wpos<K>(r, j)) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
          fence_async_smem();
          if (!(ok = epi_sync())) break;
          if (r == 0) {
            mbar_expect_tx(&bar[rb], (CL - 1) * blk);
            for (uint32_t o = 0; o < CL; ++o)
              if (o != crank) {
                const uint32_t slot = par * 3 + (crank < o ? crank : crank - 1);  // this CTA's slot at peer o
                bulk_s2s_cluster(mapa(su32(sWrecv + slot * kBM * K), o), su32(sW), blk, mapa(su32(&bar[rb]), o));
              }
            bulk_commit();
            bulk_wait_read0();
          }
          if (!(ok = wait(rb, (Tg >> 1) & 1, true))) break;
          float acc[K];
#pragma unroll
          for (int j = 0; j < K; ++j) acc[j] = 0.f;
          for (uint32_t src = 0; src < CL; ++src) {
            const float* pb = src == crank ? sW : sWrecv + (par * 3 + (src < crank ? src : src - 1)) * kBM * K;
#pragma unroll
            for (int j = 0; j < K; j += 4) {
              const float4 v = *reinterpret_cast<const float4*>(pb + wpos<K>(r, j));
              acc[j] += v.x;
              acc[j + 1] += v.y;
              acc[j + 2] += v.z;
              acc[j + 3] += v.w;
            }
          }
#pragma unroll
          for (int j = 0; j < K; ++j) w[j] = acc[j];
        } else if (CL > 1) {
          // Reduce-scatter + broadcast.  Owner o holds rows [o*RPC, (o+1)*RPC).
          // Every CTA writes its partial rows to sW and one thread ships each
          // owner its rows (bulk copies counted in bytes on the owner's
          // barrier); owners add the partials in source-rank order, in place,
          // and ship the sums back the same way.  Peers' data land only in rows
          // whose earlier contents were already consumed (see the waits).
          const uint32_t rows_bytes = static_cast<uint32_t>(RPC * K * 4);
          if (!(ok = epi_sync())) break;  // the previous tile's bulk copies have read sW (r == 0 waited)
#pragma unroll
          for (int j = 0; j < K; j += 4)
            *reinterpret_cast<float4*>(sW + wpos<K>(r, j)) = make_float4(w[j], w[j + 1], w[j + 2], w[j + 3]);
          fence_async_smem();
          if (!(ok = epi_sync())) break;
          if (r == 0) {
            mbar_expect_tx(&bar[B_REDFULL], (CL - 1) * rows_bytes);
            for (uint32_t o = 0; o < CL; ++o)
              if (o != crank)
                bulk_s2s_cluster(mapa(su32(sWrecv + crank * RPC * K), o), su32(sW + o * RPC * K), rows_bytes,
                                 mapa(su32(&bar[B_REDFULL]), o));
            bulk_commit();
            bulk_wait_read0();
          }
          if (!(ok = wait(B_REDFULL, Tg & 1, true))) break;
          const int per = RPC * K / kBM;  // values per epilogue thread (K / CL)
          for (int e = 0; e < per; ++e) {
            const int idx = r * per + e, rl = idx / K, col = idx % K;
            const int own = wpos<K>(static_cast<int>(crank) * RPC + rl, col);
            const int rel = own - static_cast<int>(crank) * RPC * K;  // offset inside one owner's row block
            float sum = 0.f;
            for (uint32_t src = 0; src < CL; ++src) sum += src == crank ? sW[own] : sWrecv[src * RPC * K + rel];
            sW[own] = sum;
          }
          fence_async_smem();
          if (!(ok = epi_sync())) break;
          if (r == 0) {
            mbar_expect_tx(&bar[B_WFULL], (CL - 1) * rows_bytes);
            for (uint32_t dsti = 0; dsti < CL; ++dsti)
              if (dsti != crank)
                bulk_s2s_cluster(mapa(su32(sW + crank * RPC * K), dsti), su32(sW + crank * RPC * K), rows_bytes,
                                 mapa(su32(&bar[B_WFULL]), dsti));
            bulk_commit();
            bulk_wait_read0();
          }
          if (!(ok = wait(B_WFULL, Tg & 1, true))) break;
#pragma unroll
          for (int j = 0; j < K; j += 4) {
            const float4 v = *reinterpret_cast<const float4*>(sW + wpos<K>(r, j));
            w[j] = v.x;
            w[j + 1] = v.y;
            w[j + 2] = v.z;
            w[j + 3] = v.w;
          }
        }
        // [W_hi | W_lo]^T into B2: row n = output column, k-index = tile row r
        const uint32_t bb = Tg % L::NB2BUF;
        if (!(ok = wait(B_B2FREE0 + bb, ((Tg / L::NB2BUF) + 1) & 1, false))) break;
        unsigned char* B2 = sB2 + bb * L::B2;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const uint16_t hi = bf16_bits(w[j]);
          const uint16_t lo = bf16_bits(w[j] - bf16_val(hi));
          *reinterpret_cast<uint16_t*>(B2 + sw128_off(j, r, N)) = hi;
          *reinterpret_cast<uint16_t*>(B2 + sw128_off(K + j, r, N)) = lo;
        }
        fence_async_smem();
        mbar_arrive(&bar[B_B2FULL0 + bb]);
      }
      // segment end: Y slice = D2[:, :K] + D2[:, K:] -> P[slot]
      if (ok && wait(B_D2FULL, (si - sb) & 1, false)) {
        tc_fence_after();
        float* Pd = a.P + static_cast<int64_t>(sg.slot) * a.d * K;
        for (int mb = 0; mb < L::NB2; ++mb) {
          float y[K];
#pragma unroll
          for (int q = 0; q < N / 16; ++q) {
            float v[16];
            tmem_ld16(tmem + lane_base + 2 * N + mb * N + q * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int col = q * 16 + i;
              if (col < K) y[col] = v[i];
              else y[col - K] += v[i];
            }
          }
          const int dcol = c0 + mb * 128 + (warp & 3) * 32 + lane;
          if (dcol < a.d) {
            float4* dst = reinterpret_cast<float4*>(Pd + static_cast<int64_t>(dcol) * K);
#pragma unroll
            for (int j = 0; j < K; j += 4) dst[j / 4] = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
          }
        }
        tc_fence_before();
      }
    }
    T += ntiles;
  }

  // ---- teardown: all MMAs retired, no remote traffic in flight, then free TMEM
  if (warp == 1 && lane == 0) mma_commit(&bar[B_DONE]);
  __syncthreads();
  if (warp == 0) {
    const uint32_t addr = su32(&bar[B_DONE]);
    const long long t0 = clock64();
    while (!mbar_try(addr, 0) && clock64() - t0 < kTimeoutCycles) {
    }
  }
  __syncthreads();
  cluster_sync_all();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(L::tmem_cols) : "memory");
  }
}

template <int K, int NCH>
cudaError_t launch_tc_t(const TcPlan& p, const TcArgs& a, cudaStream_t s) {
  using L = TcLayout<K, NCH>;
  auto kern = step_tc_kernel<K, NCH>;
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(kern));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(p.nclusters * p.cluster), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = L::alloc_bytes;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(p.cluster);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(p.tmap);
  return cudaLaunchKernelEx(&cfg, kern, *map, a);
}

}  // namespace

// Clusters of `cl` CTAs that the device can hold at once for this kernel (0 if unknown).
// Clusters must fit inside one GPC, so this can be below sms / cl; launching more
// would run a second, mostly empty wave.
template <int K, int NCH>
int active_clusters(int cl) {
  using L = TcLayout<K, NCH>;
  auto kern = step_tc_kernel<K, NCH>;
  if (allow_max_dynamic_smem(reinterpret_cast<const void*>(kern)) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(static_cast<unsigned>(cl), 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
  cfg.dynamicSmemBytes = L::alloc_bytes;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = static_cast<unsigned>(cl);
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

bool tc_plan(int d, int k, int sms, TcPlan* p) {
  const int K = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  const int nch = d <= 128 ? 2 : 4;
  const int dc = 64 * nch;
  int cl = (d + dc - 1) / dc;
  int c2 = 1;
  while (c2 < cl) c2 *= 2;
  if (c2 > 8) return false;
  p->K = K;
  p->nch = nch;
  p->cluster = c2;
  size_t bytes;
  int active;
  if (nch == 2) {
    bytes = K == 8 ? TcLayout<8, 2>::alloc_bytes : K == 16 ? TcLayout<16, 2>::alloc_bytes : TcLayout<32, 2>::alloc_bytes;
    active = K == 8 ? active_clusters<8, 2>(c2) : K == 16 ? active_clusters<16, 2>(c2) : active_clusters<32, 2>(c2);
  } else {
    bytes = K == 8 ? TcLayout<8, 4>::alloc_bytes : K == 16 ? TcLayout<16, 4>::alloc_bytes : TcLayout<32, 4>::alloc_bytes;
    active = K == 8 ? active_clusters<8, 4>(c2) : K == 16 ? active_clusters<16, 4>(c2) : active_clusters<32, 4>(c2);
  }
  p->nclusters = sms / c2;
  if (active > 0 && active < p->nclusters) p->nclusters = active;
  if (p->nclusters < 1) return false;
  p->smem = bytes;
  return bytes <= 232448;
}

cudaError_t tc_encode_map(void* A, int64_t n, int d, int64_t ld, TcPlan* p) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  static_assert(sizeof(CUtensorMap) <= sizeof(p->tmap), "tensor map storage");
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(d), static_cast<cuuint64_t>(n)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
  cuuint32_t box[2] = {64, static_cast<cuuint32_t>(kBM)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(p->tmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, A, dims, strides,
                      box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_step_tc(const TcPlan& p, const Segment* segs, const int* seg_ptr, const float* Z, int64_t z_stride,
                           float* P, int d, int* status, cudaStream_t s) {
  TcArgs a;
  a.segs = segs;
  a.seg_ptr = seg_ptr;
  a.Z = Z;
  a.z_stride = z_stride;
  a.P = P;
  a.d = d;
  a.status = status;
  if (p.nch == 2) {
    if (p.K == 8) return launch_tc_t<8, 2>(p, a, s);
    if (p.K == 16) return launch_tc_t<16, 2>(p, a, s);
    return launch_tc_t<32, 2>(p, a, s);
  }
  if (p.K == 8) return launch_tc_t<8, 4>(p, a, s);
  if (p.K == 16) return launch_tc_t<16, 4>(p, a, s);
  return launch_tc_t<32, 4>(p, a, s);
}

}  // namespace lp
