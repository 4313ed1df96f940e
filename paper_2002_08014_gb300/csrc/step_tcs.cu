// Fused local power step on the 5th-generation tensor cores, streaming form:
//   P[slot] = A_seg^T (A_seg Z_i)   (the unscaled local product of eq. (2)),
// FP32 accumulation in tensor memory, A stored as one BF16 plane or as two
// (hi = RNE_bf16(a), lo = RNE_bf16(a - hi), the FP32 data of the partition).
//
// Geometry.  Rows go in tiles of 128 (the MMA's M).  A CTA owns a column slice
// of DC = 64 * ncd columns (the whole row for d <= 1024 at k <= 16; otherwise a
// cluster of CL CTAs splits d and sums the row products through distributed
// shared memory).  The tile slice streams through a ring of 32 KB units (128
// rows x 128 columns of one plane) twice:
//   first  C1: D1 += A_u [Z_hi | Z_lo]                (M = 128 rows, N = 2K)
//   epi       W = D1[:, :K] + D1[:, K:] (cluster-summed), rows outside the
//             segment zeroed, written as [W_hi | W_lo] BF16 operand
//   second C2: D2[b] += A_u^T [W_hi | W_lo]           (M = 128 columns, N = 2K)
// The first pass reads A from HBM; the second re-reads the same unit shortly
// after, from L2.  The producer interleaves the first pass of tile t+1 with the
// second pass of tile t, `lag` units behind, so the tensor pipe has work while
// the epilogue forms W(t) and HBM always has loads in flight; no unit has to
// stay in shared memory while W is formed.  With Z resident per segment (its
// hi/lo split keeps ~16 significant bits) and W split the same way, the
// products carry FP32-level accuracy on BF16 tensor-core operands.
//
// Roles (256 threads): warp 0 lane 0 issues TMA; lane 0 of warps 1 and 2 issue
// MMAs (two issuers: one thread issues a small-N MMA only every ~55 cycles, and
// every ~100 when it polls barriers between MMAs), each owning alternate
// 128-column blocks (both planes of a block) with its own partial D1 (the
// epilogue sums the two in issuer order) and its own part of the ring, so that
// it consumes its slots strictly in order; warps 4-7 (one per TMEM lane
// quadrant) run the epilogue; all warps stage Z at segment starts.  Every wait is bounded: on expiry the kernel records
// ST_TIMEOUT, stops issuing, waits (bounded) for its own copies in flight,
// frees tensor memory and returns.
#include "lp_internal.cuh"
#include "tc_ptx.cuh"

namespace lp {
namespace {

using namespace tc;

constexpr int kUnitBytes = 2 * kChunkBytes;  // 128 rows x 128 columns BF16
constexpr int kMaxRing = 8;
constexpr int kSmemLimit = 232448;

enum TcsBar { S_D1FULL0 = 0, S_D1EMPTY0 = 2, S_B2FULL0 = 4, S_B2FREE0 = 6, S_D2FULL = 8, S_REDFULL = 9,
              S_WFULL = 10, S_DONE = 11, S_EPI = 12, S_RING0 = 13 };  // ring: FULL[s] = S_RING0 + s, EMPTY[s] = S_RING0 + ring + s

struct TcsArgs {
  const Segment* segs;
  const int* seg_ptr;  // per cluster
  const float* Z;
  int64_t z_stride;
  float* P;
  int d;
  int* status;
  int ncd;   // 64-column chunks in this CTA's slice (even)
  int ring;  // ring units
  int lag;   // first-pass units of tile t+1 issued before the second pass of tile t starts
  int issuers;  // MMA-issuing threads (1 or 2), each with its own partial D1
  int prefetch;  // first-pass units brought into L2 ahead of their load (0: none)
  int hints;     // 1: first-pass loads evict_last, second-pass loads evict_first
  uint32_t off_B1, off_B2, off_W, off_Wrecv, off_bar, tmem_cols;
};


// Walks the load/consume order of one segment: first pass of tile t (units
// 0..U-1) interleaved with the second pass of tile t-1, `lag` units behind.
// fn(second, t, u) returns false to stop.
template <typename F>
__device__ __forceinline__ bool for_each_unit(int ntiles, int U, int lag, F&& fn) {
  for (int t = 0; t <= ntiles; ++t)
    for (int u = 0; u < U + lag; ++u) {
      if (t < ntiles && u < U && !fn(false, t, u)) return false;
      if (t >= 1 && u >= lag && u - lag < U && !fn(true, t - 1, u - lag)) return false;
    }
  return true;
}

template <int K, int PL>
__global__ void __launch_bounds__(kThreads, 1)
    step_tcs_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1, TcsArgs a) {
  constexpr int N = 2 * K;
  constexpr uint32_t B2BUF = 2 * N * 128;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sRing = base;
  unsigned char* sB1 = base + a.off_B1;
  unsigned char* sB2 = base + a.off_B2;
  float* sW = reinterpret_cast<float*>(base + a.off_W);
  float* sWrecv = reinterpret_cast<float*>(base + a.off_Wrecv);
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + a.off_bar);
  const int R = a.ring;
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + S_RING0 + 2 * R);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t crank = cluster_rank();
  const uint32_t CL = cluster_size();
  const int RPC = kBM / static_cast<int>(CL);
  const int cluster_id = blockIdx.x / CL;
  const int DC = 64 * a.ncd;
  const int c0 = static_cast<int>(crank) * DC;
  const int NB = a.ncd / 2;
  const int U = NB * PL;
  const int LAG = a.lag;
  // Issuer h owns blocks b = h, h + HE, ... and ring slots [ring_base(h),
  // ring_base(h) + ring_len(h)) (R dealt as evenly as it goes: 3 = 2 + 1).
  const int HE = a.issuers < NB ? a.issuers : NB;
  auto ring_len = [&](int hh) { return R / HE + (hh < R % HE ? 1 : 0); };
  auto ring_base = [&](int hh) { return hh * (R / HE) + (hh < R % HE ? hh : R % HE); };
  const int h = warp - 1;
  const bool issuer = lane == 0 && (warp == 1 || warp == 2);

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar[S_D1FULL0 + s], HE);
      mbar_init(&bar[S_D1EMPTY0 + s], 4);
      mbar_init(&bar[S_B2FULL0 + s], kBM);
      mbar_init(&bar[S_B2FREE0 + s], HE);
    }
    mbar_init(&bar[S_D2FULL], HE);
    mbar_init(&bar[S_REDFULL], 1);
    mbar_init(&bar[S_WFULL], 1);
    mbar_init(&bar[S_DONE], 2);  // both issuer threads commit (an idle one at once)
    mbar_init(&bar[S_EPI], 128);  // barrier of the four epilogue warps (bounded waits)
    for (int s = 0; s < R; ++s) {
      mbar_init(&bar[S_RING0 + s], 1);
      mbar_init(&bar[S_RING0 + R + s], 1);
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

  constexpr uint32_t idesc1 = idesc_bf16(128, N, false, false);
  constexpr uint32_t idesc2 = idesc_bf16(128, N, true, false);

  const int sb = a.seg_ptr[cluster_id], se = a.seg_ptr[cluster_id + 1];
  uint32_t T = 0;  // tiles before this segment (same in every CTA of the cluster)
  uint32_t epi_phase = 0;  // uses of the epilogue barrier so far (epilogue threads)
  uint32_t pcnt[2] = {0u, 0u};  // producer: units dealt to each issuer so far
  uint32_t fills[kMaxRing] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};  // producer: fills of each slot
  uint32_t c_own = 0;           // issuer: own units consumed so far
  for (int si = sb; si < se; ++si) {
    const Segment sg = a.segs[si];
    const int ntiles = static_cast<int>((sg.row1 - sg.row0 + kBM - 1) / kBM);

    // ---- stage this slice of Z as [Z_hi | Z_lo]^T (N rows x DC, K-major, SWIZZLE_128B)
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
      uint64_t pol_keep = 0, pol_drop = 0;
      if (a.hints) {
        pol_keep = l2_policy_evict_last();
        pol_drop = l2_policy_evict_first();
      }
      const int PF = a.prefetch;
      // first-pass units [0, PF) of the segment go to L2 up front; later ones PF units ahead of their load
      for (int q = 0; q < PF && q < ntiles * U; ++q) {
        const int t2 = q / U, u2 = q % U, b2 = u2 / PL, pl2 = u2 % PL;
        for (int j = 0; j < 2; ++j)
          tma_prefetch_2d(pl2 ? &map1 : &map0, c0 + 64 * (2 * b2 + j), static_cast<int>(sg.row0) + t2 * kBM);
      }
      for_each_unit(ntiles, U, LAG, [&](bool second, int t, int u) -> bool {
        // the next slot of the issuer that consumes this unit
        const int hh = (u / PL) % HE;
        const uint32_t k = pcnt[hh], RH = static_cast<uint32_t>(ring_len(hh));
        const uint32_t s = static_cast<uint32_t>(ring_base(hh)) + k % RH;
        if (!wait(S_RING0 + R + s, ((k / RH) + 1) & 1, false)) return false;
        pcnt[hh] = k + 1;
        ++fills[s];
        mbar_expect_tx(&bar[S_RING0 + s], kUnitBytes);
        const int b = u / PL, pl = u % PL;
        const int row = static_cast<int>(sg.row0) + t * kBM;
        const CUtensorMap* map = pl ? &map1 : &map0;
        for (int j = 0; j < 2; ++j) {
          const uint32_t dst = su32(sRing + s * kUnitBytes + j * kChunkBytes);
          if (a.hints)
            tma_load_2d_hint(dst, map, c0 + 64 * (2 * b + j), row, &bar[S_RING0 + s], second ? pol_drop : pol_keep);
          else
            tma_load_2d(dst, map, c0 + 64 * (2 * b + j), row, &bar[S_RING0 + s]);
        }
        if (!second && PF > 0) {
          const int q = t * U + u + PF;
          if (q < ntiles * U) {
            const int t2 = q / U, u2 = q % U, b2 = u2 / PL, pl2 = u2 % PL;
            for (int j = 0; j < 2; ++j)
              tma_prefetch_2d(pl2 ? &map1 : &map0, c0 + 64 * (2 * b2 + j), static_cast<int>(sg.row0) + t2 * kBM);
          }
        }
        return true;
      });
      // Copies still in flight (only after an abort) land before the CTA exits:
      // the last fill of every slot (earlier fills were waited for by then).
      for (int q = 0; q < R; ++q) {
        if (fills[q] == 0) continue;
        const uint32_t addr = su32(&bar[S_RING0 + q]);
        const long long t0 = clock64();
        while (!mbar_try(addr, (fills[q] - 1) & 1) && clock64() - t0 < kTimeoutCycles) {
        }
      }
    } else if (issuer && h < HE) {
      // ------------------------------------------------------------ MMA issuers
      // issuer h: units of blocks b = h, h + HE, ... in the shared unit order
      const int b_last = h + ((NB - 1 - h) / HE) * HE;
      const int u_first = h * PL, u_last = b_last * PL + PL - 1;
      const uint32_t RH = static_cast<uint32_t>(ring_len(h)), rb = static_cast<uint32_t>(ring_base(h));
      for_each_unit(ntiles, U, LAG, [&](bool second, int t, int u) -> bool {
        if ((u / PL) % HE != h) return true;
        const uint32_t s = rb + c_own % RH, Tg = T + t, buf = Tg & 1;
        if (!wait(S_RING0 + s, (c_own / RH) & 1, false)) return false;
        ++c_own;
        if (u == u_first) {
          if (!second && !wait(S_D1EMPTY0 + buf, ((Tg >> 1) + 1) & 1, false)) return false;
          if (second && !wait(S_B2FULL0 + buf, (Tg >> 1) & 1, false)) return false;
        }
        tc_fence_after();
        const int b = u / PL, pl = u % PL;
        const uint32_t aS = su32(sRing + s * kUnitBytes);
        if (!second) {
          const uint32_t bS = su32(sB1);
#pragma unroll
          for (int j = 0; j < 2; ++j)
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
              const uint64_t ad = sdesc(aS + j * kChunkBytes + kk * 32, 16, 1024);
              const uint64_t bd = sdesc(bS + (2 * b + j) * N * 128 + kk * 32, 16, 1024);
              mma_bf16(tmem + (buf * HE + h) * N, ad, bd, idesc1, (u != u_first || j != 0 || kk != 0) ? 1u : 0u);
            }
          mma_commit(&bar[S_RING0 + R + s]);
          if (u == u_last) mma_commit(&bar[S_D1FULL0 + buf]);
        } else {
          const uint32_t bS = su32(sB2 + buf * B2BUF);
#pragma unroll
          for (int kk = 0; kk < 8; ++kk) {
            // A^T: M = 128 columns (two 64-column chunks, LBO apart), K = 16 rows (two 8-row groups, SBO apart)
            const uint64_t ad = sdesc(aS + kk * 2048, kChunkBytes, 1024);
            const uint64_t bd = sdesc(bS + (kk >> 2) * N * 128 + (kk & 3) * 32, 16, 1024);
            mma_bf16(tmem + 2 * HE * N + b * N, ad, bd, idesc2, (t == 0 && pl == 0 && kk == 0) ? 0u : 1u);
          }
          mma_commit(&bar[S_RING0 + R + s]);
          if (u == u_last) mma_commit(&bar[S_B2FREE0 + buf]);
        }
        return true;
      });
      mma_commit(&bar[S_D2FULL]);
    } else if (warp >= 4) {
      // ------------------------------------------------------------ epilogue
      const int r = (warp - 4) * 32 + lane;
      const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
      bool ok = true;
      // Barrier of the 128 epilogue threads on an mbarrier with a bounded wait
      // (a named barrier could hang if some threads left the loop on an abort).
      auto epi_sync = [&]() -> bool {
        mbar_arrive(&bar[S_EPI]);
        return wait(S_EPI, (epi_phase++) & 1, false);
      };
      for (int t = 0; ok && t < ntiles; ++t) {
        const uint32_t Tg = T + t, buf = Tg & 1;
        if (!(ok = wait(S_D1FULL0 + buf, (Tg >> 1) & 1, false))) break;
        tc_fence_after();
        // W = the issuers' partials, each [hi part | lo part], summed in a fixed order
        float w[K];
#pragma unroll
        for (int j = 0; j < K; ++j) w[j] = 0.f;
        for (int hh = 0; hh < HE; ++hh) {
#pragma unroll
          for (int q = 0; q < N / 16; ++q) {
            float v[16];
            tmem_ld16(tmem + lane_base + (buf * HE + hh) * N + q * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int col = q * 16 + i;
              w[col < K ? col : col - K] += v[i];
            }
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[S_D1EMPTY0 + buf]);
        const bool valid = sg.row0 + static_cast<int64_t>(t) * kBM + r < sg.row1;
        if (!valid) {
#pragma unroll
          for (int j = 0; j < K; ++j) w[j] = 0.f;
        }
        if (CL > 1) {
          // Cluster sum of W.  Owner o holds rows [o*RPC, (o+1)*RPC).  Every CTA
          // writes its partial rows to sW and one thread ships each owner its
          // rows (bulk copies counted in bytes on the owner's barrier); owners
          // add the partials in source-rank order, in place, and ship the sums
          // back the same way.  A buffer is rewritten only after the waits show
          // its previous contents were consumed.
          const uint32_t rows_bytes = static_cast<uint32_t>(RPC * K * 4);
          if (!(ok = epi_sync())) break;  // the previous tile's bulk copies have read sW (r == 0 waited)
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
          const int per = RPC * K / kBM;  // values per epilogue thread (K / CL)
          for (int e = 0; e < per; ++e) {
            const int idx = r * per + e, rl = idx / K, col = idx % K;
            const int own = wpos<K>(static_cast<int>(crank) * RPC + rl, col);
            const int rel = own - static_cast<int>(crank) * RPC * K;  // offset inside one owner's row block
            float sum = 0.f;
            for (uint32_t src = 0; src < CL; ++src)
              sum += src == crank ? sW[own] : sWrecv[src * RPC * K + rel];
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
        // [W_hi | W_lo]^T into B2[buf]: row n = output column, k-index = tile row r
        if (!(ok = wait(S_B2FREE0 + buf, ((Tg >> 1) + 1) & 1, false))) break;
        unsigned char* B2 = sB2 + buf * B2BUF;
#pragma unroll
        for (int j = 0; j < K; ++j) {
          const uint16_t hi = bf16_bits(w[j]);
          const uint16_t lo = bf16_bits(w[j] - bf16_val(hi));
          *reinterpret_cast<uint16_t*>(B2 + sw128_off(j, r, N)) = hi;
          *reinterpret_cast<uint16_t*>(B2 + sw128_off(K + j, r, N)) = lo;
        }
        fence_async_smem();
        mbar_arrive(&bar[S_B2FULL0 + buf]);
      }
      // segment end: Y slice = D2[:, :K] + D2[:, K:] -> P[slot]
      if (ok && wait(S_D2FULL, (si - sb) & 1, false)) {
        tc_fence_after();
        float* Pd = a.P + static_cast<int64_t>(sg.slot) * a.d * K;
        for (int b = 0; b < NB; ++b) {
          float y[K];
#pragma unroll
          for (int q = 0; q < N / 16; ++q) {
            float v[16];
            tmem_ld16(tmem + lane_base + 2 * HE * N + b * N + q * 16, v);
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
            for (int j = 0; j < K; j += 4) dst[j / 4] = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
          }
        }
        tc_fence_before();
      }
    }
    T += ntiles;
  }

  // ---- teardown: all MMAs retired, no remote traffic in flight, then free TMEM
  if (issuer) mma_commit(&bar[S_DONE]);
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

template <int K, int PL>
cudaError_t set_smem_attr(size_t) {
  return allow_max_dynamic_smem(reinterpret_cast<const void*>(step_tcs_kernel<K, PL>));
}

template <int K, int PL>
cudaLaunchConfig_t tcs_config(unsigned grid, int cl, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kThreads, 1, 1);
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

template <int K, int PL>
int tcs_active_clusters(int cl, size_t smem) {
  if (set_smem_attr<K, PL>(smem) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = tcs_config<K, PL>(static_cast<unsigned>(cl), cl, smem, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, step_tcs_kernel<K, PL>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

template <int K, int PL>
cudaError_t launch_tcs_t(const TcsPlan& p, const TcsArgs& a, cudaStream_t s) {
  cudaError_t e = set_smem_attr<K, PL>(p.smem);
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg =
      tcs_config<K, PL>(static_cast<unsigned>(p.nclusters * p.cluster), p.cluster, p.smem, s, attr);
  const CUtensorMap* m0 = reinterpret_cast<const CUtensorMap*>(p.tmap[0]);
  const CUtensorMap* m1 = reinterpret_cast<const CUtensorMap*>(p.tmap[PL > 1 ? 1 : 0]);
  return cudaLaunchKernelEx(&cfg, step_tcs_kernel<K, PL>, *m0, *m1, a);
}

int active_for(int K, int planes, int cl, size_t smem) {
  if (planes == 1)
    return K == 8 ? tcs_active_clusters<8, 1>(cl, smem) : K == 16 ? tcs_active_clusters<16, 1>(cl, smem)
                                                                  : tcs_active_clusters<32, 1>(cl, smem);
  return K == 8 ? tcs_active_clusters<8, 2>(cl, smem) : K == 16 ? tcs_active_clusters<16, 2>(cl, smem)
                                                                : tcs_active_clusters<32, 2>(cl, smem);
}

}  // namespace

bool tcs_plan(int d, int k, int planes, int sms, const TcsTuning& tune, TcsPlan* p) {
  const int ring_cap = tune.ring_units;
  int lag = tune.lag_units;
  if (planes != 1 && planes != 2) return false;
  const int K = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  const int N = 2 * K;
  // <= 64 KB of resident Z slice; with two planes at most 512 columns, so a
  // tile's units (and with them the distance from a unit's first read to its L2
  // re-read) stay at 256 KB per CTA
  int ncd_max = K == 32 ? 8 : 16;
  if (planes == 2 && ncd_max > 8) ncd_max = 8;
  if (tune.slice_cols >= 128 && tune.slice_cols / 64 < ncd_max) ncd_max = (tune.slice_cols / 128) * 2;
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
  const int fixed_no_bars = static_cast<int>(B1 + B2 + 2 * W);
  int ring = (kSmemLimit - 1024 - fixed_no_bars - (S_RING0 + 2 * kMaxRing) * 8 - 16) / kUnitBytes;
  if (ring > kMaxRing) ring = kMaxRing;
  if (ring_cap > 0 && ring > ring_cap) ring = ring_cap;
  if (ring < 2) return false;
  p->K = K;
  p->planes = planes;
  p->ncd = ncd;
  p->cluster = cl;
  p->ring = ring;
  const int U = (ncd / 2) * planes;
  if (lag <= 0) lag = cl > 1 ? 4 : 2;
  p->lag = lag < U ? lag : U;
  p->prefetch = tune.prefetch_units > 0 ? tune.prefetch_units : 0;
  p->hints = tune.cache_hints ? 1 : 0;
  p->off_B1 = static_cast<uint32_t>(ring) * kUnitBytes;
  p->off_B2 = p->off_B1 + B1;
  p->off_W = p->off_B2 + B2;
  p->off_Wrecv = p->off_W + W;
  p->off_bar = p->off_Wrecv + W;
  p->smem = p->off_bar + (S_RING0 + 2 * ring) * 8 + 16 + 1024;
  // two issuers (two partial D1 per buffer) when tensor memory holds them
  const int NBp = ncd / 2;
  // (independent of the ring depth, which must only reorder loads: any ring of two
  // or more units deals each issuer at least one slot)
  p->issuers = (4 * N + NBp * N <= 512 && NBp >= 2) ? 2 : 1;
  const uint32_t used = static_cast<uint32_t>(2 * p->issuers * N + NBp * N);
  uint32_t cols = 32;
  while (cols < used) cols *= 2;
  if (cols > 512) return false;
  p->tmem_cols = cols;
  if (p->smem > static_cast<size_t>(kSmemLimit)) return false;
  const int active = active_for(K, planes, cl, p->smem);
  p->nclusters = sms / cl;
  if (active > 0 && active < p->nclusters) p->nclusters = active;
  return p->nclusters >= 1;
}

cudaError_t tcs_encode_maps(const void* plane0, const void* plane1, int64_t n, int d, int64_t ld, TcsPlan* p,
                            bool unit_boxes) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  static_assert(sizeof(CUtensorMap) <= sizeof(p->tmap[0]), "tensor map storage");
  const void* planes[2] = {plane0, plane1};
  p->map3d = 0;
  // One box per 128-column unit (both 64-column chunks): the matrix viewed as
  // (column within a chunk, row, chunk), which stays inside every row only when
  // d is a whole number of chunks and rows are not padded (ld == d).
  if (unit_boxes && d % 64 == 0 && ld == d) {
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) {
      if (!planes[i]) continue;
      cuuint64_t dims[3] = {64, static_cast<cuuint64_t>(n), static_cast<cuuint64_t>(d / 64)};
      cuuint64_t strides[2] = {static_cast<cuuint64_t>(ld) * 2, 128};
      cuuint32_t box[3] = {64, static_cast<cuuint32_t>(kBM), 2};
      cuuint32_t estr[3] = {1, 1, 1};
      ok = encode(reinterpret_cast<CUtensorMap*>(p->tmap[i]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                  const_cast<void*>(planes[i]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (ok) {
      p->map3d = 1;
      return cudaSuccess;
    }
  }
  for (int i = 0; i < 2; ++i) {
    if (!planes[i]) continue;
    cuuint64_t dims[2] = {static_cast<cuuint64_t>(d), static_cast<cuuint64_t>(n)};
    cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * 2};
    cuuint32_t box[2] = {64, static_cast<cuuint32_t>(kBM)};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = encode(reinterpret_cast<CUtensorMap*>(p->tmap[i]), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                        const_cast<void*>(planes[i]), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

cudaError_t launch_step_tcs(const TcsPlan& p, const Segment* segs, const int* seg_ptr, const float* Z,
                            int64_t z_stride, float* P, int d, int* status, cudaStream_t s) {
  TcsArgs a;
  a.segs = segs;
  a.seg_ptr = seg_ptr;
  a.Z = Z;
  a.z_stride = z_stride;
  a.P = P;
  a.d = d;
  a.status = status;
  a.ncd = p.ncd;
  a.ring = p.ring;
  a.lag = p.lag;
  a.issuers = p.issuers;
  a.prefetch = p.prefetch;
  a.hints = p.hints;
  a.off_B1 = p.off_B1;
  a.off_B2 = p.off_B2;
  a.off_W = p.off_W;
  a.off_Wrecv = p.off_Wrecv;
  a.off_bar = p.off_bar;
  a.tmem_cols = p.tmem_cols;
  if (p.planes == 1) {
    if (p.K == 8) return launch_tcs_t<8, 1>(p, a, s);
    if (p.K == 16) return launch_tcs_t<16, 1>(p, a, s);
    return launch_tcs_t<32, 1>(p, a, s);
  }
  if (p.K == 8) return launch_tcs_t<8, 2>(p, a, s);
  if (p.K == 16) return launch_tcs_t<16, 2>(p, a, s);
  return launch_tcs_t<32, 2>(p, a, s);
}

}  // namespace lp
