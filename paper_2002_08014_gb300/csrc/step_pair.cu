// Fused local power step on the 5th-generation tensor cores, the two passes
// split over the two CTAs of a cluster (two SMs):
//   P[slot] = A_seg^T (A_seg Z_i)   (the unscaled local product of eq. (2)),
// FP32 accumulation in tensor memory, A stored as one BF16 plane or as two
// (hi = RNE_bf16(a), lo = RNE_bf16(a - hi), the FP32 data of the partition).
//
// Why split.  Both products need the same 128-row tile: W = A_t Z needs whole
// rows, and A_t^T W needs W.  A tile of the FP32 workload (128 rows x 1,024
// columns x two planes) is 512 KB, far more than shared memory, so the tile
// streams through shared memory twice, the second time from L2.  On one SM
// the resident Z slice leaves room for only four 32 KB units and the MMA
// issuer stalls on every tile's W; streaming measurements on GB300 show the
// two-pass pattern holding 6.7-7.2 TB/s only while the L2 re-read follows the
// first read within ~256 KB per SM and the ring keeps enough bytes in flight.
// Here each pass has an SM of its own:
//   rank 0  streams the tile from HBM through its ring (evict_last), holds
//           [Z_hi | Z_lo] for all d columns, accumulates
//             D1 += A_u [Z_hi | Z_lo]        (M = 128 rows, N = 2K)
//           in one of two TMEM buffers, and its epilogue forms
//             W = D1[:, :K] + D1[:, K:]  (rows past the segment zeroed)
//           as the BF16 operand [W_hi | W_lo] and copies it (one bulk copy
//           through distributed shared memory) into rank 1's W buffer;
//   rank 1  re-reads the same units from L2 (evict_first) one tile behind,
//           with a deeper ring (no Z), and accumulates
//             D2[b] += A_u^T [W_hi | W_lo]   (M = 128 columns, N = 2K)
//           over the segment in one of two TMEM buffers, which its epilogue
//           drains into P[slot] (Y slice = D2[:, :K] + D2[:, K:]) while the
//           next segment accumulates into the other.
// W moves one way, once per tile; neither pass waits on the other except
// through two W buffers (rank 0 may run up to two tiles ahead).  With Z and W
// split hi/lo the products carry FP32-level accuracy on BF16 operands, and the
// sums are formed in the same order as the single-SM streaming kernel's.
//
// Roles (384 threads per CTA): warp 0 lane 0 issues TMA; lane 0 of warps 1-4
// issue MMAs (four issuers: one thread issues a small-N MMA about every 55
// cycles and much slower when it also polls barriers between MMAs, while four
// threads in four warps keep the tensor pipe fed; rank 0's issuers take units
// round-robin, each into its own partial D1 that the epilogue sums in issuer
// order, rank 1's take 128-column blocks round-robin, each block its own D2);
// warps 8-11 (one per TMEM lane quadrant) run the epilogue; on rank 1, warp 5
// lane 0 recycles W buffers; on rank 0 all warps stage Z when the partition
// changes.  Every wait is bounded: on expiry the CTA records
// ST_TIMEOUT, stops issuing, waits (bounded) for its own copies in flight and
// for W copies addressed to it, retires its MMAs, frees tensor memory and
// returns; the partner's own bounded waits then expire the same way.
#include "lp_internal.cuh"
#include "tc_ptx.cuh"

namespace lp {
namespace {

using namespace tc;

constexpr int kUnitBytes = 2 * kChunkBytes;  // 128 rows x 128 columns of one BF16 plane
constexpr int kPairThreads = 384;
constexpr int kIssuers = 4;    // MMA-issuing threads: lane 0 of warps 1 .. kIssuers
constexpr int kIssuers1 = 3;   // rank 1 uses at most three (its ring of six units splits 3 x 2)
constexpr int kRecycler = 5;   // rank 1: warp of the W-buffer recycler
constexpr int kEpiWarp0 = 8;   // warps 8-11: epilogue (warp % 4 = TMEM lane quadrant)
constexpr int kMaxRing = 8;
constexpr int kSmemLimit = 232448;

enum PairBar {
  R0_D1FULL = 0,     // [2] rank 0: MMA -> epilogue, D1 of a tile complete
  R0_D1EMPTY = 2,    // [2] rank 0: epilogue (4 warps) -> MMA, D1 read out
  R0_B2FREE = 4,     // [2] rank 0: rank 1's W buffer may be overwritten (remote arrive)
  R0_ZDRAIN = 6,     // rank 0: MMAs of a run retired (before Z is restaged)
  R1_B2FULL = 7,     // [2] rank 1: W bytes landed (bulk copy from rank 0, counted in bytes)
  R1_B2USED = 9,     // [2] rank 1: MMA -> recycler, a tile's pass-2 MMAs retired
  R1_D2FULL = 11,    // [2] rank 1: MMA -> epilogue, a segment's Y slice complete
  R1_D2EMPTY = 13,   // [2] rank 1: epilogue (4 warps) -> MMA issuers, Y slice read out
  B_EPI = 15,        // the 128 epilogue threads (bounded barrier)
  B_DONE = 16,       // teardown: every MMA retired
  B_NEVER = 17,      // completed by nothing: the test hook's wait (LP test_stall_cycles)
  B_RING0 = 18       // FULL[s] = B_RING0 + s, EMPTY[s] = B_RING0 + kMaxRing + s
};
constexpr int kNumBars = B_RING0 + 2 * kMaxRing;

struct PairArgs {
  const Segment* segs;
  const int* seg_ptr;  // per cluster
  const float* Z;
  int64_t z_stride;
  float* P;
  int d;
  int* status;
  int ncd;    // 64-column chunks covering d (even)
  int ring0;  // rank 0 ring units
  int ring1;  // rank 1 ring units
  int nd2;    // rank 1 Y-slice buffers in TMEM (1 or 2)
  int hints;  // 1: rank 0 loads evict_last, rank 1 loads evict_first
  int prefetch;  // rank 0: units brought into L2 this far ahead of their load (0: none)
  int map3d;     // 1: the maps are (64 columns, row, chunk) and one box brings a whole unit
  long long stall;  // test hook: > 0 makes rank 0's producer wait this many cycles on B_NEVER
  uint32_t off_Z, off_stage, off_bar, tmem0, tmem1;
};

__device__ __forceinline__ void mbar_arrive_remote(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
__device__ __forceinline__ void st_cluster_u32(uint32_t cluster_addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(cluster_addr), "r"(v) : "memory");
}

template <int K, int PL>
__global__ void __launch_bounds__(kPairThreads, 1)
    step_pair_kernel(const __grid_constant__ CUtensorMap map0, const __grid_constant__ CUtensorMap map1, PairArgs a) {
  constexpr int N = 2 * K;
  constexpr uint32_t B2BUF = 2 * N * 128;  // [W_hi | W_lo]^T: N rows x 128 k (two 64-k chunks)
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* sRing = base;
  unsigned char* sZ = base + a.off_Z;
  unsigned char* sStage = base + a.off_stage;  // rank 0: staging of W; rank 1: the W buffers
  uint64_t* bar = reinterpret_cast<uint64_t*>(base + a.off_bar);
  uint32_t* tmem_holder = reinterpret_cast<uint32_t*>(bar + kNumBars);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_holder + 1);
  volatile uint32_t* sent_slot = tmem_holder + 2;      // rank 1: W copies rank 0 issued (written by rank 0)
  volatile uint32_t* consumed_slot = tmem_holder + 4;  // rank 1, per issuer: W buffers whose arrival it waited for

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t rank = cluster_rank();
  const int cluster_id = blockIdx.x >> 1;
  const int NB = a.ncd / 2;
  const int U = NB * PL;
  const int R = rank == 0 ? a.ring0 : a.ring1;
  const uint32_t tmem_cols = rank == 0 ? a.tmem0 : a.tmem1;
  // Active issuers: rank 0 deals units round-robin, rank 1 deals 128-column blocks.
  // The ring's slots are dealt to the issuers as well: issuer h owns slots
  // [h * RH, (h + 1) * RH) and consumes its units strictly in order, so no thread
  // ever waits on a slot phase more than one past the slot's last completed
  // phase (an mbarrier parity wait further ahead would succeed at once).
  const int HE = rank == 0 ? min(min(U, kIssuers), R) : min(min(NB, kIssuers1), R);
  const int RH = R / HE;
  const int h = warp - 1;  // issuer index on warps 1 .. kIssuers
  const bool issuer = lane == 0 && warp >= 1 && warp <= kIssuers;
  auto issuer_of = [&](int u) { return rank == 0 ? u % HE : (u / PL) % HE; };

  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&bar[R0_D1FULL + s], HE);
      mbar_init(&bar[R0_D1EMPTY + s], 4);
      mbar_init(&bar[R0_B2FREE + s], 1);
      mbar_init(&bar[R1_B2FULL + s], 1);
      mbar_init(&bar[R1_B2USED + s], HE);
      mbar_init(&bar[R1_D2FULL + s], HE);
      mbar_init(&bar[R1_D2EMPTY + s], 4);
    }
    mbar_init(&bar[R0_ZDRAIN], HE);
    mbar_init(&bar[B_EPI], 128);
    mbar_init(&bar[B_DONE], kIssuers);
    mbar_init(&bar[B_NEVER], 1);
    for (int s = 0; s < kMaxRing; ++s) {
      mbar_init(&bar[B_RING0 + s], 1);
      mbar_init(&bar[B_RING0 + kMaxRing + s], 1);
    }
    *abort_flag = 0;
    *sent_slot = 0;
    for (int i = 0; i < kIssuers; ++i) consumed_slot[i] = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_holder)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  cluster_sync_all();  // both CTAs' barriers initialised before any remote arrive or copy
  tc_fence_after();
  const uint32_t tmem = *tmem_holder;

  // A CTA that gives up also raises its partner's flag (both CTAs live until the
  // teardown's cluster barrier), so the partner stops at its next wait.
  auto give_up = [&]() {
    *abort_flag = 1;
    st_cluster_u32(mapa(su32(const_cast<int*>(abort_flag)), rank ^ 1u), 1u);
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
  auto bounded_drain = [&](int id, uint32_t parity) {
    const uint32_t addr = su32(&bar[id]);
    const long long t0 = clock64();
    while (!mbar_try_cluster(addr, parity) && clock64() - t0 < kTimeoutCycles) {
    }
  };

  const int sb = a.seg_ptr[cluster_id], se = a.seg_ptr[cluster_id + 1];
  auto tiles_of = [&](int s) { return static_cast<int>((a.segs[s].row1 - a.segs[s].row0 + kBM - 1) / kBM); };
  uint32_t total_tiles = 0;
  for (int s = sb; s < se; ++s) total_tiles += static_cast<uint32_t>(tiles_of(s));

  // TMA producer over the segments [s0, s1): every unit of every tile, in order,
  // each into the next slot of the issuer that consumes it, optionally bringing
  // the unit PF places ahead into L2 first.  pcnt[h] counts the units dealt to
  // issuer h, fills[s] the fills of slot s.  Returns false after an abort.
  uint32_t pcnt[kIssuers] = {0u, 0u, 0u, 0u};
  uint32_t issued_total = 0;
  uint32_t fills[kMaxRing] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
  auto produce = [&](int s0, int s1, uint64_t policy, int PF) -> bool {
    for (int s = s0; s < s1; ++s) {
      const Segment sg = a.segs[s];
      const int nt = tiles_of(s);
      auto prefetch_unit = [&](int q) {
        const int t2 = q / U, u2 = q % U, b2 = u2 / PL, pl2 = u2 % PL;
        if (a.map3d) {
          tma_prefetch_3d(pl2 ? &map1 : &map0, 0, static_cast<int>(sg.row0) + t2 * kBM, 2 * b2);
          return;
        }
        for (int j = 0; j < 2; ++j)
          tma_prefetch_2d(pl2 ? &map1 : &map0, 64 * (2 * b2 + j), static_cast<int>(sg.row0) + t2 * kBM);
      };
      for (int q = 0; q < PF && q < nt * U; ++q) prefetch_unit(q);
      for (int t = 0; t < nt; ++t)
        for (int u = 0; u < U; ++u) {
          if (PF > 0 && t * U + u + PF < nt * U) prefetch_unit(t * U + u + PF);
          const int hh = issuer_of(u);
          const uint32_t k = pcnt[hh];
          const uint32_t slot = static_cast<uint32_t>(hh * RH) + k % RH;
          if (!wait(B_RING0 + kMaxRing + slot, ((k / RH) + 1) & 1, false)) return false;
          pcnt[hh] = k + 1;
          ++fills[slot];
          mbar_expect_tx(&bar[B_RING0 + slot], kUnitBytes);
          issued_total += 1;
          const int b = u / PL, pl = u % PL;
          const int row = static_cast<int>(sg.row0) + t * kBM;
          const CUtensorMap* map = pl ? &map1 : &map0;
          if (a.map3d) {
            // chunks 2b and 2b + 1 as one box (a chunk past d is out of range: zeros)
            const uint32_t dst = su32(sRing + slot * kUnitBytes);
            if (a.hints) tma_load_3d_hint(dst, map, 0, row, 2 * b, &bar[B_RING0 + slot], policy);
            else tma_load_3d(dst, map, 0, row, 2 * b, &bar[B_RING0 + slot]);
          } else {
            for (int j = 0; j < 2; ++j) {
              const uint32_t dst = su32(sRing + slot * kUnitBytes + j * kChunkBytes);
              if (a.hints) tma_load_2d_hint(dst, map, 64 * (2 * b + j), row, &bar[B_RING0 + slot], policy);
              else tma_load_2d(dst, map, 64 * (2 * b + j), row, &bar[B_RING0 + slot]);
            }
          }
          // Test hook: after rank 0's first ring fill (copies in flight, MMAs started),
          // a wait that nothing can complete runs out its short limit and aborts.
          if (a.stall > 0 && rank == 0 && issued_total == static_cast<uint32_t>(R)) {
            const long long t0 = clock64();
            while (!mbar_try(su32(&bar[B_NEVER]), 0)) {
              if (clock64() - t0 > a.stall) {
                give_up();
                return false;
              }
            }
          }
        }
    }
    return true;
  };
  // After an abort: copies still in flight land before the CTA's shared memory
  // goes (the last fill of every slot; earlier fills were waited for by then).
  auto drain_ring = [&]() {
    for (int q = 0; q < HE * RH; ++q)
      if (fills[q] > 0) bounded_drain(B_RING0 + q, (fills[q] - 1) & 1);
  };

  if (rank == 0) {
    // ===================================================================== rank 0: W = A_t Z
    constexpr uint32_t idesc1 = idesc_bf16(128, N, false, false);
    const int DC = 64 * a.ncd;
    uint32_t c_mma = 0, T_epi = 0, T_mma = 0, epi_phase = 0, sent = 0, run = 0;
    bool prod_ok = true;
    int si = sb;
    const uint64_t pol = a.hints ? l2_policy_evict_last() : 0;
    while (si < se) {
      // a run: consecutive segments of one partition share Z_i
      const int part = a.segs[si].part;
      int sj = si + 1;
      while (sj < se && a.segs[sj].part == part) ++sj;
      __syncthreads();  // every role finished the previous run (its MMAs retired: ZDRAIN)
      if (*abort_flag) break;
      if (run == 0 || a.z_stride != 0) {
        const float* Zg = a.Z + a.z_stride * part;
        for (int e = tid; e < DC * K; e += kPairThreads) {
          const int c = e / K, j = e % K;
          const float z = c < a.d ? Zg[static_cast<int64_t>(c) * K + j] : 0.f;
          const uint16_t hi = bf16_bits(z);
          const uint16_t lo = bf16_bits(z - bf16_val(hi));
          *reinterpret_cast<uint16_t*>(sZ + sw128_off(j, c, N)) = hi;
          *reinterpret_cast<uint16_t*>(sZ + sw128_off(K + j, c, N)) = lo;
        }
      }
      fence_async_smem();
      __syncthreads();

      if (warp == 0 && lane == 0) {
        if (prod_ok) prod_ok = produce(si, sj, pol, a.prefetch);
      } else if (issuer && h < HE) {
        // ------------------------------------------------ MMA issuers, pass 1: issuer h takes units
        // u = h, h + HE, ... of every tile into its partial D1[buf][h]
        const int u_last = h + ((U - 1 - h) / HE) * HE;
        bool ok = true;
        for (int s = si; ok && s < sj; ++s) {
          const int nt = tiles_of(s);
          for (int t = 0; ok && t < nt; ++t, ++T_mma) {
            const uint32_t buf = T_mma & 1;
            if (!(ok = wait(R0_D1EMPTY + buf, ((T_mma >> 1) + 1) & 1, false))) break;
            for (int u = h; u < U; u += HE, ++c_mma) {
              const uint32_t slot = static_cast<uint32_t>(h * RH) + c_mma % RH;
              if (!(ok = wait(B_RING0 + slot, (c_mma / RH) & 1, false))) break;
              tc_fence_after();
              const int b = u / PL;
              const uint32_t aS = su32(sRing + slot * kUnitBytes);
              const uint32_t bS = su32(sZ);
#pragma unroll
              for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                  const uint64_t ad = sdesc(aS + j * kChunkBytes + kk * 32, 16, 1024);
                  const uint64_t bd = sdesc(bS + (2 * b + j) * N * 128 + kk * 32, 16, 1024);
                  mma_bf16(tmem + (buf * kIssuers + h) * N, ad, bd, idesc1, (u != h || j != 0 || kk != 0) ? 1u : 0u);
                }
              mma_commit(&bar[B_RING0 + kMaxRing + slot]);
              if (u == u_last) mma_commit(&bar[R0_D1FULL + buf]);
            }
          }
        }
        // every MMA of the run retired before the next run restages Z
        mma_commit(&bar[R0_ZDRAIN]);
        wait(R0_ZDRAIN, run & 1, false);
      } else if (warp >= kEpiWarp0) {
        // ------------------------------------------------ epilogue: D1 -> [W_hi | W_lo] -> rank 1
        const int r = (warp - kEpiWarp0) * 32 + lane;
        const uint32_t lane_base = static_cast<uint32_t>((warp & 3) * 32) << 16;
        bool ok = true;
        auto epi_sync = [&]() -> bool {
          mbar_arrive(&bar[B_EPI]);
          return wait(B_EPI, (epi_phase++) & 1, false);
        };
        for (int s = si; ok && s < sj; ++s) {
          const Segment sg = a.segs[s];
          const int nt = tiles_of(s);
          for (int t = 0; ok && t < nt; ++t, ++T_epi) {
            const uint32_t buf = T_epi & 1;
            if (!(ok = wait(R0_D1FULL + buf, (T_epi >> 1) & 1, false))) break;
            tc_fence_after();
            // W = sum over the issuers' partials, each [hi part | lo part] (fixed order)
            float w[K];
#pragma unroll
            for (int j = 0; j < K; ++j) w[j] = 0.f;
            for (int hh = 0; hh < HE; ++hh) {
#pragma unroll
              for (int q = 0; q < N / 16; ++q) {
                float v[16];
                tmem_ld16(tmem + lane_base + (buf * kIssuers + hh) * N + q * 16, v);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                  const int col = q * 16 + i;
                  w[col < K ? col : col - K] += v[i];
                }
              }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&bar[R0_D1EMPTY + buf]);
            if (!(sg.row0 + static_cast<int64_t>(t) * kBM + r < sg.row1)) {
#pragma unroll
              for (int j = 0; j < K; ++j) w[j] = 0.f;
            }
            // staging[buf] was last read by the copy of tile T_epi - 2, which thread
            // r == 0 waited for before joining the previous tile's barrier
            unsigned char* stg = sStage + buf * B2BUF;
#pragma unroll
            for (int j = 0; j < K; ++j) {
              const uint16_t hi = bf16_bits(w[j]);
              const uint16_t lo = bf16_bits(w[j] - bf16_val(hi));
              *reinterpret_cast<uint16_t*>(stg + sw128_off(j, r, N)) = hi;
              *reinterpret_cast<uint16_t*>(stg + sw128_off(K + j, r, N)) = lo;
            }
            fence_async_smem();
            if (!(ok = epi_sync())) break;
            if (r == 0) {
              if (!(ok = wait(R0_B2FREE + buf, (T_epi >> 1) & 1, true))) break;
              bulk_s2s_cluster(mapa(su32(stg), 1), su32(stg), B2BUF, mapa(su32(&bar[R1_B2FULL + buf]), 1));
              bulk_commit();
              bulk_wait_read0();
              ++sent;
            }
          }
        }
      }
      ++run;
      si = sj;
    }
    if (warp == 0 && lane == 0) drain_ring();
    if (warp == kEpiWarp0 && lane == 0) st_cluster_u32(mapa(su32(const_cast<uint32_t*>(sent_slot)), 1), sent);
  } else {
    // ===================================================================== rank 1: Y += A_t^T W
    constexpr uint32_t idesc2 = idesc_bf16(128, N, true, false);
    if (warp == 0 && lane == 0) {
      produce(sb, se, a.hints ? l2_policy_evict_first() : 0, 0);
      drain_ring();
    } else if (issuer && h < HE) {
      // ------------------------------------------------ MMA issuers, pass 2: issuer h takes the
      // 128-column blocks b = h, h + HE, ... (both planes of each), each into its own D2 slice
      const int b_last = h + ((NB - 1 - h) / HE) * HE;
      const int u_first = h * PL, u_last = b_last * PL + PL - 1;
      bool ok = true;
      uint32_t c = 0, T = 0, consumed = 0;
      for (int s = sb, pi = 0; ok && s < se; ++s, ++pi) {
        const int pb = pi % a.nd2;
        const uint32_t use = static_cast<uint32_t>(pi / a.nd2);
        const int nt = tiles_of(s);
        for (int t = 0; ok && t < nt; ++t, ++T) {
          const uint32_t buf = T & 1;
          for (int u = u_first; u <= u_last; u = ((u % PL) == PL - 1) ? u + (HE - 1) * PL + 1 : u + 1, ++c) {
            const uint32_t slot = static_cast<uint32_t>(h * RH) + c % RH;
            if (!(ok = wait(B_RING0 + slot, (c / RH) & 1, false))) break;
            if (u == u_first) {
              if (!(ok = wait(R1_B2FULL + buf, (T >> 1) & 1, true))) break;
              consumed = T + 1;
              if (t == 0 && !(ok = wait(R1_D2EMPTY + pb, (use + 1) & 1, false))) break;
            }
            tc_fence_after();
            const int b = u / PL, pl = u % PL;
            const uint32_t aS = su32(sRing + slot * kUnitBytes);
            const uint32_t bS = su32(sStage + buf * B2BUF);
#pragma unroll
            for (int kk = 0; kk < 8; ++kk) {
              // A^T: M = 128 columns (two 64-column chunks, LBO apart), K = 16 rows (two 8-row groups, SBO apart)
              const uint64_t ad = sdesc(aS + kk * 2048, kChunkBytes, 1024);
              const uint64_t bd = sdesc(bS + (kk >> 2) * N * 128 + (kk & 3) * 32, 16, 1024);
              mma_bf16(tmem + (pb * NB + b) * N, ad, bd, idesc2, (t == 0 && pl == 0 && kk == 0) ? 0u : 1u);
            }
            mma_commit(&bar[B_RING0 + kMaxRing + slot]);
            if (u == u_last) {
              mma_commit(&bar[R1_B2USED + buf]);
              if (t == nt - 1) mma_commit(&bar[R1_D2FULL + pb]);
            }
          }
        }
      }
      consumed_slot[h] = consumed;
    } else if (warp == kRecycler && lane == 0) {
      // ------------------------------------------------ W buffer recycler
      for (uint32_t b = 0; b < 2 && b < total_tiles; ++b) {
        mbar_expect_tx(&bar[R1_B2FULL + b], B2BUF);
        mbar_arrive_remote(mapa(su32(&bar[R0_B2FREE + b]), 0));
      }
      for (uint32_t T = 0; T < total_tiles; ++T) {
        const uint32_t buf = T & 1;
        if (!wait(R1_B2USED + buf, (T >> 1) & 1, false)) break;
        if (T + 2 < total_tiles) {
          mbar_expect_tx(&bar[R1_B2FULL + buf], B2BUF);
          mbar_arrive_remote(mapa(su32(&bar[R0_B2FREE + buf]), 0));
        }
      }
    } else if (warp >= kEpiWarp0) {
      // ------------------------------------------------ epilogue: Y slices -> P[slot]
      for (int s = sb, pi = 0; s < se; ++s, ++pi) {
        const int pb = pi % a.nd2;
        const uint32_t use = static_cast<uint32_t>(pi / a.nd2);
        if (!wait(R1_D2FULL + pb, use & 1, false)) break;
        tc_fence_after();
        float* Pd = a.P + static_cast<int64_t>(a.segs[s].slot) * a.d * K;
        for (int b = 0; b < NB; ++b) {
          float y[K];
#pragma unroll
          for (int q = 0; q < N / 16; ++q) {
            float v[16];
            tmem_ld16(tmem + (static_cast<uint32_t>((warp & 3) * 32) << 16) + (pb * NB + b) * N + q * 16, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
              const int col = q * 16 + i;
              if (col < K) y[col] = v[i];
              else y[col - K] += v[i];
            }
          }
          const int dcol = b * 128 + (warp & 3) * 32 + lane;
          if (dcol < a.d) {
            float4* dst = reinterpret_cast<float4*>(Pd + static_cast<int64_t>(dcol) * K);
#pragma unroll
            for (int j = 0; j < K; j += 4) dst[j / 4] = make_float4(y[j], y[j + 1], y[j + 2], y[j + 3]);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&bar[R1_D2EMPTY + pb]);
      }
    }
  }

  // ---- teardown: MMAs retired, W copies addressed to rank 1 landed, then free TMEM
  if (issuer) mma_commit(&bar[B_DONE]);  // every issuer's MMAs (none for an idle issuer)
  __syncthreads();
  if (warp == 0 && lane == 0) bounded_drain(B_DONE, 0);
  __syncthreads();
  cluster_sync_all();  // rank 0's sent count is visible to rank 1; no remote traffic starts after this
  if (rank == 1 && tid == 0) {
    const uint32_t sent = *sent_slot;
    uint32_t consumed = consumed_slot[0];
    for (int i = 1; i < HE; ++i) consumed = consumed_slot[i] < consumed ? consumed_slot[i] : consumed;
    for (uint32_t T = consumed; T < sent; ++T) bounded_drain(R1_B2FULL + (T & 1), (T >> 1) & 1);
  }
  __syncthreads();
  cluster_sync_all();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

template <int K, int PL>
cudaLaunchConfig_t pair_config(unsigned grid, size_t smem, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1, 1);
  cfg.blockDim = dim3(kPairThreads, 1, 1);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

template <int K, int PL>
int pair_active_clusters(size_t smem) {
  if (allow_max_dynamic_smem(reinterpret_cast<const void*>(step_pair_kernel<K, PL>)) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config<K, PL>(2, smem, nullptr, attr);
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, step_pair_kernel<K, PL>, &cfg) != cudaSuccess) {
    (void)cudaGetLastError();
    return 0;
  }
  return n;
}

int pair_active_for(int K, int planes, size_t smem) {
  if (planes == 1)
    return K == 8 ? pair_active_clusters<8, 1>(smem) : K == 16 ? pair_active_clusters<16, 1>(smem)
                                                             : pair_active_clusters<32, 1>(smem);
  return K == 8 ? pair_active_clusters<8, 2>(smem) : K == 16 ? pair_active_clusters<16, 2>(smem)
                                                           : pair_active_clusters<32, 2>(smem);
}

template <int K, int PL>
cudaError_t launch_pair_t(const TcsPlan& p, const PairArgs& a, cudaStream_t s) {
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(step_pair_kernel<K, PL>));
  if (e != cudaSuccess) return e;
  cudaLaunchAttribute attr[1];
  cudaLaunchConfig_t cfg = pair_config<K, PL>(static_cast<unsigned>(2 * p.nclusters), p.smem, s, attr);
  const CUtensorMap* m0 = reinterpret_cast<const CUtensorMap*>(p.tmap[0]);
  const CUtensorMap* m1 = reinterpret_cast<const CUtensorMap*>(p.tmap[PL > 1 ? 1 : 0]);
  return cudaLaunchKernelEx(&cfg, step_pair_kernel<K, PL>, *m0, *m1, a);
}

}  // namespace

bool pair_plan(int d, int k, int planes, int sms, const TcsTuning& tune, TcsPlan* p) {
  if (planes != 1 && planes != 2) return false;
  const int K = k <= 8 ? 8 : (k <= 16 ? 16 : 32);
  const int N = 2 * K;
  int ncd = (d + 63) / 64;
  ncd += ncd & 1;
  const int NB = ncd / 2;
  if (NB * N > 512) return false;  // rank 1's Y slice must fit tensor memory
  const uint32_t zbytes = static_cast<uint32_t>(ncd) * N * 128;
  const uint32_t stage = 2u * (2u * N * 128);
  const uint32_t bars = kNumBars * 8 + 32;  // barriers, TMEM holder, abort flag, sent, consumed[kIssuers]
  const int avail = kSmemLimit - 1024 - static_cast<int>(stage + bars);
  int ring0 = (avail - static_cast<int>(zbytes)) / kUnitBytes;
  int ring1 = avail / kUnitBytes;
  if (ring0 > kMaxRing) ring0 = kMaxRing;
  if (ring1 > kMaxRing) ring1 = kMaxRing;
  if (tune.ring_units > 0) {
    if (ring0 > tune.ring_units) ring0 = tune.ring_units;
    if (ring1 > tune.ring_units) ring1 = tune.ring_units;
  }
  if (ring0 < 2 || ring1 < 2) return false;
  p->pair = 1;
  p->K = K;
  p->planes = planes;
  p->ncd = ncd;
  p->cluster = 2;
  p->ring = ring0;
  p->ring1 = ring1;
  p->lag = 0;
  p->prefetch = tune.prefetch_units > 0 ? tune.prefetch_units : 0;
  p->stall = tune.test_stall_cycles;
  p->hints = 1;  // rank 0 evict_last, rank 1 evict_first (measured best for the two-pass pattern)
  // layout: ring region (rank 1 uses it all), Z (rank 0), W staging / W buffers, barriers
  const uint32_t ring_region = static_cast<uint32_t>(ring1 > ring0 ? ring1 : ring0) * kUnitBytes;
  p->off_B1 = static_cast<uint32_t>(ring0) * kUnitBytes;  // Z
  p->off_B2 = ring_region > p->off_B1 + zbytes ? ring_region : p->off_B1 + zbytes;  // staging / W buffers
  p->off_bar = p->off_B2 + stage;
  p->off_W = p->off_Wrecv = 0;
  p->smem = p->off_bar + bars + 1024;
  if (p->smem > static_cast<size_t>(kSmemLimit)) return false;
  uint32_t c0 = 32;
  while (c0 < static_cast<uint32_t>(2 * kIssuers * N)) c0 *= 2;  // D1[2][kIssuers]
  if (c0 > 512) return false;
  p->tmem_cols = c0;
  p->nd2 = 2 * NB * N <= 512 ? 2 : 1;
  uint32_t c1 = 32;
  while (c1 < static_cast<uint32_t>(p->nd2 * NB * N)) c1 *= 2;
  p->tmem_cols1 = c1;
  const int active = pair_active_for(K, planes, p->smem);
  p->nclusters = sms / 2;
  if (active > 0 && active < p->nclusters) p->nclusters = active;
  return p->nclusters >= 1;
}

cudaError_t launch_step_pair(const TcsPlan& p, const Segment* segs, const int* seg_ptr, const float* Z,
                             int64_t z_stride, float* P, int d, int* status, cudaStream_t s) {
  PairArgs a;
  a.segs = segs;
  a.seg_ptr = seg_ptr;
  a.Z = Z;
  a.z_stride = z_stride;
  a.P = P;
  a.d = d;
  a.status = status;
  a.ncd = p.ncd;
  a.ring0 = p.ring;
  a.ring1 = p.ring1;
  a.nd2 = p.nd2;
  a.hints = p.hints;
  a.prefetch = p.prefetch;
  a.map3d = p.map3d;
  a.stall = p.stall;
  a.off_Z = p.off_B1;
  a.off_stage = p.off_B2;
  a.off_bar = p.off_bar;
  a.tmem0 = p.tmem_cols;
  a.tmem1 = p.tmem_cols1;
  if (p.planes == 1) {
    if (p.K == 8) return launch_pair_t<8, 1>(p, a, s);
    if (p.K == 16) return launch_pair_t<16, 1>(p, a, s);
    return launch_pair_t<32, 1>(p, a, s);
  }
  if (p.K == 8) return launch_pair_t<8, 2>(p, a, s);
  if (p.K == 16) return launch_pair_t<16, 2>(p, a, s);
  return launch_pair_t<32, 2>(p, a, s);
}

}  // namespace lp
