// The d x k and k x k kernels around the fused power step:
//   reduce     Y_i = (1/s_i) sum of the step kernel's per-CTA partials (fixed order)
//   cholqr2    Z = orth(Y) by two passes of Gram / Cholesky / triangular solve
//   align      sign-fixing (eq. (4)) or orthogonal Procrustes (eq. (3)) matrices
//   aggregate  Y = sum_i p_i Y_i D_i (Alg. 1 aggregation)
//   ritz       Rayleigh-Ritz on span(Z): ordered basis and sigma_j = sqrt(n lambda_j)
//   split      FP32 rows -> hi / lo BF16 planes (load time)
//   rho        residual error of Def. 3 per partition (traced solves)
// Precision, by default: the d-sized work (Gram, solves, averaging) and the k x k
// Jacobi SVD / eigen-solves are FP32; the Cholesky factor is FP32 when its pivots
// allow (else FP64); the Ritz matrix H and the sign-fix inner products that
// decide D_i are accumulated in FP64.  GB300's FP64 pipe is a small fraction of
// its FP32 pipe, and these k x k steps are serial latency on every round.  With
// LP_FLAG_KXK_FP64 the k x k work is FP64 throughout: the CholQR2 Gram (summed in
// FP64) and its Cholesky, the Procrustes SVD and the Ritz eigen-solve.
#include <algorithm>
#include <cfloat>
#include <mutex>
#include <unordered_set>

#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kT = 256;

// FP64 1/sqrt(x) by Newton-Raphson iteration from an FP32 seed
// (y <- y (3 - x y^2) / 2); each step doubles the number of correct bits, so two
// steps take the FP32 seed (about 2^-22) past FP64 precision.  An FP64 square
// root is a long instruction sequence on this GPU; this is a few FMAs on the
// FP64 Cholesky's critical path.  Arguments outside the FP32 normal range take
// the plain sqrt.
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = static_cast<double>(rsqrtf(static_cast<float>(x)));
  const double hx = 0.5 * x;
  y = y * (1.5 - hx * y * y);
  y = y * (1.5 - hx * y * y);
  return y;
}

// ---------------------------------------------------------------- pack / unpack
// FP32 rows -> two BF16 planes: hi = RNE(a), lo = RNE(a - hi).  a - hi is exact
// in FP32, so hi + lo matches a to within half an ulp of lo (<= 2^-17 |a|).
__global__ void split_planes_kernel(const float* __restrict__ src, int64_t src_ld, int64_t rows, int d,
                                    uint16_t* __restrict__ hi, uint16_t* __restrict__ lo, int64_t ld) {
  const int64_t total = rows * ld;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t r = e / ld;
    const int c = static_cast<int>(e - r * ld);
    const float a = c < d ? src[r * src_ld + c] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(a);
    const __nv_bfloat16 l = __float2bfloat16_rn(a - __bfloat162float(h));
    hi[e] = __bfloat16_as_ushort(h);
    lo[e] = __bfloat16_as_ushort(l);
  }
}

__global__ void pack_kernel(const double* __restrict__ src, float* __restrict__ dst, int batch, int d, int k, int K) {
  const int64_t total = int64_t(batch) * d * K;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(e % K);
    const int64_t row = e / K;  // b * d + c
    dst[e] = j < k ? static_cast<float>(src[row * k + j]) : 0.f;
  }
}
__global__ void unpack_kernel(const float* __restrict__ src, double* __restrict__ dst, int batch, int d, int k, int K) {
  const int64_t total = int64_t(batch) * d * k;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int j = static_cast<int>(e % k);
    const int64_t row = e / k;
    dst[e] = static_cast<double>(src[row * K + j]);
  }
}

// ---------------------------------------------------------------- reduce
// G adjacent threads share one float4 of Y_i: thread g of the group sums slots
// sb + g, sb + g + G, ... in order (four loads in flight), then the group adds
// its G partials by an xor butterfly.  The order is fixed for a given G, so
// results are reproducible; G > 1 only when partitions have many slots (small
// problems spread over many CTAs), where it cuts the chain of dependent loads.
template <int G>
__global__ void reduce_kernel(const float* __restrict__ P, const int* __restrict__ slot_begin,
                              const float* __restrict__ scale, int d, int K, float* __restrict__ Y) {
  const int i = blockIdx.y;
  const int64_t n4 = int64_t(d) * K / 4;
  const int g = threadIdx.x % G;
  const int64_t e = blockIdx.x * int64_t(blockDim.x / G) + threadIdx.x / G;
  const bool live = e < n4;
  if (G == 1 && !live) return;
  const int sb = slot_begin[i], se = slot_begin[i + 1];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (live) {
    int s = sb + g;
    for (; s + 3 * G < se; s += 4 * G) {
      float4 v[4];
#pragma unroll
      for (int q = 0; q < 4; ++q) v[q] = reinterpret_cast<const float4*>(P + int64_t(s + q * G) * d * K)[e];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        acc.x += v[q].x; acc.y += v[q].y; acc.z += v[q].z; acc.w += v[q].w;
      }
    }
    for (; s < se; s += G) {
      const float4 v = reinterpret_cast<const float4*>(P + int64_t(s) * d * K)[e];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
  }
#pragma unroll
  for (int o = 1; o < G; o <<= 1) {
    acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
    acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    acc.z += __shfl_xor_sync(0xffffffffu, acc.z, o);
    acc.w += __shfl_xor_sync(0xffffffffu, acc.w, o);
  }
  if (!live || g != 0) return;
  const float sc = scale[i];
  acc.x *= sc; acc.y *= sc; acc.z *= sc; acc.w *= sc;
  reinterpret_cast<float4*>(Y + int64_t(i) * d * K)[e] = acc;
}

// ---------------------------------------------------------------- k x k helpers
__device__ __forceinline__ float warp_sumf(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Thresholds of the Jacobi sweeps per precision: a pair (p, q) is rotated while
// |c_p . c_q| > tol ||c_p|| ||c_q|| (tol a few units of the type's rounding
// error times k, so the last sweep only sees rounding noise below it); `tiny`
// skips pairs whose product underflows; beyond `huge` t = 1 / (2 |zeta|) avoids
// squaring zeta.
template <typename T> struct JacobiLimits;
template <> struct JacobiLimits<float> {
  static constexpr float tol = 1e-6f, tiny = 1e-35f, huge = 1e15f;
};
template <> struct JacobiLimits<double> {
  static constexpr double tol = 1e-13, tiny = 1e-300, huge = 1e150;
};

// One-sided (Hestenes) Jacobi on the k x k matrix C (stride K, in shared memory),
// accumulating the rotations in V, in precision T: on return C's columns are
// mutually orthogonal, C_in V = C_out, so C_in = U Sigma V^T with
// sigma_j = ||C_out[:, j]|| and U[:, j] = C_out[:, j] / sigma_j.  FP32 by
// default because GB300's FP64 pipe is a small fraction of its FP32 pipe and
// these k x k problems sit on serial critical paths (the aligners and Ritz
// values stay within 1e-7 of FP64 factorisations on the FP32 workload's
// spectrum); FP64 under LP_FLAG_KXK_FP64.
//
// All kT threads of the CTA call it.  A sweep visits every column pair once in
// the round-robin (circle) order: with np = k rounded up to even (the extra
// column a dummy whose pairs are skipped), step s pairs column np - 1 with s and
// (s + j) mod (np - 1) with (s - j) mod (np - 1) for j = 1 .. np/2 - 1, which
// makes each step a set of disjoint pairs and each sweep np - 1 steps.  Pair
// slot j of a step belongs to half-warp j; its 16 lanes hold rows h and h + 16
// of the two columns, sum the three inner products over the half-warp and
// rotate their rows.  One barrier per step; the sweeps stop when a whole sweep
// rotated nothing.  Returns false if the sweep limit was hit.
template <typename T>
__device__ bool cta_jacobi(T* C, T* V, int k, int K) {
  using L = JacobiLimits<T>;
  const int t = threadIdx.x;
  const int slot = t >> 4, h = t & 15;
  const int np = k + (k & 1);
  for (int e = t; e < K * K; e += kT) V[e] = (e / K == e % K) ? T(1) : T(0);
  __syncthreads();
  for (int sweep = 0; sweep < 40; ++sweep) {
    int rotated = 0;
    for (int s = 0; s < np - 1; ++s) {
      int p = 0, q = 0;
      bool live = slot < np / 2;
      if (live) {
        if (slot == 0) {
          p = s;
          q = np - 1;
        } else {
          p = (s + slot) % (np - 1);
          q = (s - slot + np - 1) % (np - 1);
        }
        live = p < k && q < k;
      }
      T a = 0, b = 0, g = 0;
      if (live)
        for (int r = h; r < k; r += 16) {
          const T cp = C[r * K + p], cq = C[r * K + q];
          a += cp * cp;
          b += cq * cq;
          g += cp * cq;
        }
      // every lane takes part in the shuffles; offsets below 16 stay in the half-warp
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        g += __shfl_xor_sync(0xffffffffu, g, o);
      }
      if (live && fabs(g) > L::tol * sqrt(a * b) && fabs(g) > L::tiny) {
        rotated = 1;
        // zeta = (b - a) / 2g, t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2)
        const T zeta = (b - a) / (T(2) * g);
        const T az = fabs(zeta);
        const T tn = (zeta >= T(0) ? T(1) : T(-1)) / (az > L::huge ? T(2) * az : az + sqrt(T(1) + zeta * zeta));
        const T c = T(1) / sqrt(T(1) + tn * tn);
        const T sn = c * tn;
        for (int r = h; r < k; r += 16) {
          const T cp = C[r * K + p], cq = C[r * K + q];
          C[r * K + p] = c * cp - sn * cq;
          C[r * K + q] = sn * cp + c * cq;
          const T vp = V[r * K + p], vq = V[r * K + q];
          V[r * K + p] = c * vp - sn * vq;
          V[r * K + q] = sn * vp + c * vq;
        }
      }
      __syncthreads();
    }
    if (!__syncthreads_or(rotated)) return true;
  }
  return false;
}

// The orthogonal Procrustes factor O = U V^T of eq. (3) from a finished one-sided
// Jacobi (C holds U Sigma, V the rotations): U's columns are normalised in
// place, then O is formed entry by entry into Gi (K x K, zero beyond k).  A
// column with no norm leaves O short of orthogonal and sets ST_JACOBI.  All
// threads call it; `inv` holds K values of scratch.
template <typename T>
__device__ void procrustes_factor(T* C, const T* V, T* inv, int k, int K, float* Gi, int* status) {
  const int t = threadIdx.x;
  const T small = sizeof(T) == 8 ? T(1e-300) : T(1e-37);
  if (t < k) {
    T nrm = 0;
    for (int r = 0; r < k; ++r) nrm += C[r * K + t] * C[r * K + t];
    inv[t] = nrm > small ? T(1) / sqrt(nrm) : T(0);
    if (!(nrm > small)) atomicOr(status, ST_JACOBI);
  }
  __syncthreads();
  for (int e = t; e < k * K; e += kT)
    if (e % K < k) C[e] *= inv[e % K];
  __syncthreads();
  for (int e = t; e < K * K; e += kT) {
    const int a = e / K, b = e % K;
    T sum = 0;
    if (a < k && b < k)
      for (int j = 0; j < k; ++j) sum = fma(C[a * K + j], V[b * K + j], sum);
    Gi[e] = static_cast<float>(sum);
  }
}

// ---------------------------------------------------------------- CholQR2
// One CTA per block, two passes of:
//   G = Y^T Y        FP32 products and partial sums over row slices, combined in FP32
//   G = L L^T        right-looking Cholesky on warp 0: FP32, or FP64 when an FP32
//                    pivot is too small to trust
//   Z = Y L^{-T}     per-row forward substitution in FP32, one thread per row
// The column space is Y's whatever the precision of L; the second pass restores
// orthonormality lost to the FP32 Gram.  A pivot that is not positive and finite
// sets ST_CHOL (the pivot is then taken as 1 so the kernel can finish).
// G = Y^T Y: thread (block (bi, bj) of 4 x 4 entries, row slice) accumulates
// Y[r][4bi..4bi+3]^T Y[r][4bj..4bj+3] over its rows in FP32 registers (16 FMAs
// per two 16-byte loads); the slices are added in FP32 through shared memory.
template <int K>
__device__ void gram_fp32(const float* Y, int d, float* red, double* G) {
  constexpr int NB = K / 4, NBB = NB * NB, S = kT / NBB;
  const int t = threadIdx.x;
  const int blk = t % NBB, sl = t / NBB;
  const int bi = blk / NB, bj = blk % NB;
  float acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
  // eight rows per trip, all loads issued before the FMAs: one block reads the
  // whole d x K block with ~16 loads in flight per thread instead of one
  constexpr int U = 8;
  for (int r0 = sl; r0 < d; r0 += S * U) {
    float4 u[U], v[U];
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const int r = r0 + q * S;
      u[q] = r < d ? *reinterpret_cast<const float4*>(Y + int64_t(r) * K + 4 * bi) : make_float4(0.f, 0.f, 0.f, 0.f);
      v[q] = r < d ? *reinterpret_cast<const float4*>(Y + int64_t(r) * K + 4 * bj) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int q = 0; q < U; ++q) {
      const float uu[4] = {u[q].x, u[q].y, u[q].z, u[q].w}, vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(uu[a], vv[b], acc[a][b]);
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) red[(sl * NBB + blk) * 16 + 4 * a + b] = acc[a][b];
  __syncthreads();
  for (int e = t; e < K * K; e += kT) {
    const int i = e / K, j = e % K;
    const int bb = (i / 4) * NB + j / 4, el = 4 * (i % 4) + j % 4;
    // four interleaved FP32 partial sums in slice order, then pairwise: short
    // dependency chains (the factorisation reads the Gram in FP32 first)
    float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
    int q = 0;
    for (; q + 4 <= S; q += 4) {
      s0 += red[(q * NBB + bb) * 16 + el];
      s1 += red[((q + 1) * NBB + bb) * 16 + el];
      s2 += red[((q + 2) * NBB + bb) * 16 + el];
      s3 += red[((q + 3) * NBB + bb) * 16 + el];
    }
    for (; q < S; ++q) s0 += red[(q * NBB + bb) * 16 + el];
    G[e] = static_cast<double>((s0 + s1) + (s2 + s3));
  }
  __syncthreads();
}

// G = Y^T Y in FP64 (LP_FLAG_KXK_FP64): the upper triangle of 4 x 4 blocks, one
// per thread of a row slice; each FP32 product is exact in FP64 (two 24-bit
// significands need 48 of its 53 bits) and is summed in FP64 over the slice's
// rows; the slices are added in slice order and the lower triangle mirrored.
template <int K>
__device__ void gram_fp64(const float* Y, int d, double* red, double* G) {
  constexpr int NB = K / 4, NBU = NB * (NB + 1) / 2, S = kT / NBU;
  const int t = threadIdx.x;
  const int blk = t % NBU, sl = t / NBU;
  int bi = 0, rem = blk;
  while (rem >= NB - bi) {
    rem -= NB - bi;
    ++bi;
  }
  const int bj = bi + rem;
  if (sl < S) {
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    constexpr int U = 4;
    for (int r0 = sl; r0 < d; r0 += S * U) {
      float4 u[U], v[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int r = r0 + q * S;
        u[q] = r < d ? *reinterpret_cast<const float4*>(Y + int64_t(r) * K + 4 * bi) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[q] = r < d ? *reinterpret_cast<const float4*>(Y + int64_t(r) * K + 4 * bj) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const double uu[4] = {u[q].x, u[q].y, u[q].z, u[q].w}, vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fma(uu[a], vv[b], acc[a][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) red[(sl * NBU + blk) * 16 + 4 * a + b] = acc[a][b];
  }
  __syncthreads();
  for (int e = t; e < K * K; e += kT) {
    const int i = e / K, j = e % K;
    const int a = i < j ? i : j, b = i < j ? j : i;
    const int ba = a / 4, bb = b / 4;
    const int idx = ba * NB - ba * (ba - 1) / 2 + (bb - ba);
    const int el = 4 * (a % 4) + b % 4;
    double sum = 0.0;
    for (int q = 0; q < S; ++q) sum += red[(q * NBU + idx) * 16 + el];
    G[e] = sum;
  }
  __syncthreads();
}

// One-warp right-looking Cholesky with the matrix in registers: lane l holds
// column l (rows 0..K-1) of the symmetric Gram; at pivot j lane j scales its
// column into L[:, j], the other lanes receive L[i][j] from lane j by shuffles,
// lane l keeps L[l][j] when i reaches l and updates its rows i >= l:
// G[i][l] -= L[i][j] L[l][j].  Every entry of the lower triangle sees the same
// operations in the same order as the textbook shared-memory form; the upper
// rows of a column (i < l) are never read.  No index arithmetic by k in the
// inner loops (the shared-memory form divided by the trailing size for every
// entry, which dominated CholQR2 at K = 32).

// FP64 factor of the FP64 Gram G (k x k, stride K; not modified).  Writes L in FP32
// (lower, stride K) and 1 / L[j][j] in FP32; returns false on breakdown (a pivot
// that is not positive and finite is then taken as 1 so the kernel can finish).
template <int K>
__device__ bool warp_cholesky_rl(const double* G, float* Lf, float* invd, int k) {
  const int lane = threadIdx.x & 31;
  double col[K];
#pragma unroll
  for (int i = 0; i < K; ++i) col[i] = (i < k && lane < k) ? G[i * K + lane] : 0.0;
  bool ok = true;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j >= k) continue;  // (not break: the loop stays unrolled, col[] in registers)
    double piv = __shfl_sync(0xffffffffu, col[j], j);
    if (!(piv > 0.0) || !isfinite(piv)) {
      ok = false;
      piv = 1.0;
    }
    const double inv = rsqrt_nr(piv);
    const double ljj = piv * inv;
    if (lane == j) {
      col[j] = ljj;
#pragma unroll
      for (int i = j + 1; i < K; ++i) col[i] *= inv;
      invd[j] = static_cast<float>(inv);
    }
    double my = 0.0;  // L[lane][j], known once i reaches lane
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      const double lij = __shfl_sync(0xffffffffu, col[i], j);
      if (i == lane) my = lij;
      if (lane > j && i >= lane) col[i] -= lij * my;
    }
  }
  if (lane < K) {
#pragma unroll
    for (int i = 0; i < K; ++i) Lf[i * K + lane] = (i < k && lane <= i) ? static_cast<float>(col[i]) : 0.f;
  }
  __syncwarp();
  return ok;
}

// FP32 factor of the FP64 Gram (read in FP32) on one warp, written to Lf (lower,
// stride K) and invd.  Returns false (G untouched, for warp_cholesky_rl) when a
// pivot is not above 1e-6 of the largest diagonal entry or not finite: GB300's
// FP64 pipe is a small fraction of its FP32 pipe, and the FP32 factor serves both
// CholQR passes whenever the Gram allows it (the column space is that of Y for
// any invertible factor; the second pass restores orthonormality).
template <int K>
__device__ bool warp_cholesky_f32(const double* G, float* Lf, float* invd, int k) {
  const int lane = threadIdx.x & 31;
  float col[K];
#pragma unroll
  for (int i = 0; i < K; ++i) col[i] = (i < k && lane < k) ? static_cast<float>(G[i * K + lane]) : 0.f;
  float dmax = lane < k ? static_cast<float>(G[lane * K + lane]) : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dmax = fmaxf(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
  if (!(dmax > 0.f) || !isfinite(dmax)) return false;
  const float floor = 1e-6f * dmax;
  bool good = true;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    if (j >= k || !good) continue;  // (not break / return: the loop stays unrolled, col[] in registers)
    const float piv = __shfl_sync(0xffffffffu, col[j], j);
    if (!(piv > floor) || !isfinite(piv)) {
      good = false;
      continue;
    }
    const float ljj = sqrtf(piv);
    const float inv = 1.0f / ljj;
    if (lane == j) {
      col[j] = ljj;
#pragma unroll
      for (int i = j + 1; i < K; ++i) col[i] *= inv;
      invd[j] = inv;
    }
    float my = 0.f;  // L[lane][j], known once i reaches lane
#pragma unroll
    for (int i = j + 1; i < K; ++i) {
      const float lij = __shfl_sync(0xffffffffu, col[i], j);
      if (i == lane) my = lij;
      if (lane > j && i >= lane) col[i] -= lij * my;
    }
  }
  if (!good) return false;
  if (lane < K) {
#pragma unroll
    for (int i = 0; i < K; ++i) Lf[i * K + lane] = (i < k && lane <= i) ? col[i] : 0.f;
  }
  __syncwarp();
  return true;
}

// Z[r][:] = Y[r][:] L^{-T}: z_j = (y_j - sum_{p<j} z_p L[j][p]) / L[j][j].  Each
// thread solves four rows at once, column j outermost, so a row of L read from
// shared memory serves four independent FMA chains.
template <int K>
__device__ void forward_rows(const float* Yin, float* Zout, const float* Lf, const float* invd, int d, int k) {
  constexpr int RPT = 4;
  for (int rb = 0; rb < d; rb += RPT * kT) {
    asm volatile("" ::: "memory");  // keep the L reads inside this iteration
    float y[RPT][K];
#pragma unroll
    for (int g = 0; g < RPT; ++g) {
      const int r = rb + threadIdx.x + g * kT;
#pragma unroll
      for (int q = 0; q < K / 4; ++q) {
        const float4 v = r < d ? reinterpret_cast<const float4*>(Yin + int64_t(r) * K)[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        y[g][4 * q] = v.x; y[g][4 * q + 1] = v.y; y[g][4 * q + 2] = v.z; y[g][4 * q + 3] = v.w;
      }
    }
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float inv = j < k ? invd[j] : 0.f;
#pragma unroll
      for (int g = 0; g < RPT; ++g) {
        float s = y[g][j];
#pragma unroll
        for (int p = 0; p < j; ++p) s = fmaf(-y[g][p], Lf[j * K + p], s);
        y[g][j] = s * inv;
      }
    }
#pragma unroll
    for (int g = 0; g < RPT; ++g) {
      const int r = rb + threadIdx.x + g * kT;
      if (r < d) {
        float4* dst = reinterpret_cast<float4*>(Zout + int64_t(r) * K);
#pragma unroll
        for (int q = 0; q < K / 4; ++q) dst[q] = make_float4(y[g][4 * q], y[g][4 * q + 1], y[g][4 * q + 2], y[g][4 * q + 3]);
      }
    }
  }
}

// Z = orth(Y) of one d x K block by the CTA: the first pass writes Zmid from Y,
// the second Zout from Zmid (Zmid may be Y itself: each thread solves its own
// rows in place; or Zout).  Any of them may have been written earlier in the same
// kernel.  F64: Gram and Cholesky in FP64 (LP_FLAG_KXK_FP64); else the FP32 Gram
// and FP32 Cholesky with the FP64 factorisation as fallback.  The d x k forward
// substitution is FP32 either way.
template <int K, bool F64>
__device__ void cholqr2_block(const float* Y, float* Zmid, float* Zout, int d, int k, int* status) {
  __shared__ __align__(16) double G[K * K];
  __shared__ __align__(16) float Lf[K * K];
  __shared__ float invd[K];
  __shared__ __align__(16) unsigned char red[(F64 ? 8 : 4) * kT * 16];
  for (int pass = 0; pass < 2; ++pass) {
    const float* src = pass == 0 ? Y : Zmid;
    if (F64) {
      gram_fp64<K>(src, d, reinterpret_cast<double*>(red), G);
      if (threadIdx.x < 32) {
        const bool ok = warp_cholesky_rl<K>(G, Lf, invd, k);
        if (!ok && threadIdx.x == 0) atomicOr(status, ST_CHOL);
      }
    } else {
      gram_fp32<K>(src, d, reinterpret_cast<float*>(red), G);
      if (threadIdx.x < 32 && !warp_cholesky_f32<K>(G, Lf, invd, k)) {
        const bool ok = warp_cholesky_rl<K>(G, Lf, invd, k);
        if (!ok && threadIdx.x == 0) atomicOr(status, ST_CHOL);
      }
    }
    __syncthreads();
    forward_rows<K>(src, pass == 0 ? Zmid : Zout, Lf, invd, d, k);
    __syncthreads();
  }
}

// One CTA per block.  STAGED: the d x K block is copied into shared memory once
// (eight 16-byte loads in flight per thread), both Grams and the first solve
// work there (the first pass's Z overwrites Y in place) and only the second
// pass writes global memory; otherwise each pass reads global memory (blocks
// larger than kCholStageBytes).
constexpr size_t kCholStageBytes = size_t(128) << 10;

template <int K, bool F64, bool STAGED>
__global__ void __launch_bounds__(kT) cholqr2_kernel(const float* __restrict__ Yall, float* __restrict__ Zall, int d,
                                                     int k, int* status) {
  const float* Y = Yall + int64_t(blockIdx.x) * d * K;
  float* Z = Zall + int64_t(blockIdx.x) * d * K;
  if constexpr (STAGED) {
    extern __shared__ __align__(16) float4 stage4[];
    const float4* Y4 = reinterpret_cast<const float4*>(Y);
    const int n4 = d * (K / 4);
    constexpr int UL = 8;
    for (int e0 = threadIdx.x; e0 < n4; e0 += kT * UL) {
      float4 v[UL];
#pragma unroll
      for (int q = 0; q < UL; ++q) {
        const int e = e0 + q * kT;
        v[q] = e < n4 ? Y4[e] : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < UL; ++q) {
        const int e = e0 + q * kT;
        if (e < n4) stage4[e] = v[q];
      }
    }
    __syncthreads();
    float* stage = reinterpret_cast<float*>(stage4);
    cholqr2_block<K, F64>(stage, stage, Z, d, k, status);
  } else {
    cholqr2_block<K, F64>(Y, Z, Z, d, k, status);
  }
}

template <int K, bool F64>
cudaError_t launch_cholqr2_t(const float* Y, float* Z, int batch, int d, int k, int* status, cudaStream_t s) {
  const size_t bytes = size_t(d) * K * 4;
  if (bytes <= kCholStageBytes) {
    const cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(cholqr2_kernel<K, F64, true>));
    if (e != cudaSuccess) return e;
    cholqr2_kernel<K, F64, true><<<batch, kT, bytes, s>>>(Y, Z, d, k, status);
  } else {
    cholqr2_kernel<K, F64, false><<<batch, kT, 0, s>>>(Y, Z, d, k, status);
  }
  return cudaGetLastError();
}


// ---------------------------------------------------------------- align
// One CTA per partition.  G_i (K x K float, row-major) = D_i (sign) or O_i (OPT).
__global__ void __launch_bounds__(kT) align_kernel(const float* __restrict__ Zl, int64_t z_stride,
                                                   const float* __restrict__ Zb_one, int d, int k, int K,
                                                   int base_one, const int* __restrict__ part_base, int opt, int f64,
                                                   float* __restrict__ Gout, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  double* C = reinterpret_cast<double*>(sm);   // K*K
  double* V = C + K * K;                        // K*K
  double* part = V + K * K;                     // kT x 16 floats
  const int i = blockIdx.x;
  const int t = threadIdx.x;
  // the base of partition i's problem: one for the context, or per partition (batch groups)
  const int base = part_base ? part_base[i] : base_one;
  const float* Zb = part_base ? Zl + z_stride * base : Zb_one;
  float* Gi = Gout + int64_t(i) * K * K;
  if (i == base) {
    for (int e = t; e < K * K; e += kT) Gi[e] = ((e / K) == (e % K) && (e / K) < k) ? 1.f : 0.f;
    return;
  }
  const float* Zi = Zl + z_stride * i;
  if (!opt) {
    // sgn <Z_i[:, j], Z_b[:, j]> with FP64 accumulation; sgn(0) = +1.
    const int j = t % K, sl = t / K, RS = kT / K;
    double s = 0.0;
    for (int r = sl; r < d; r += RS) s += static_cast<double>(Zi[int64_t(r) * K + j]) * Zb[int64_t(r) * K + j];
    part[t] = s;
    __syncthreads();
    if (t < K) {
      double tot = 0.0;
      for (int q = 0; q < RS; ++q) tot += part[q * K + t];
      part[kT - K + t] = tot;  // scratch beyond the first RS*K entries is not re-read
    }
    __syncthreads();
    for (int e = t; e < K * K; e += kT) {
      const int a = e / K, b = e % K;
      float v = 0.f;
      if (a == b && a < k) v = part[kT - K + a] < 0.0 ? -1.f : 1.f;
      Gi[e] = v;
    }
    return;
  }
  // OPT: C = Z_i^T Z_b.  Thread (4 x 4 block (bi, bj) of C, row slice sl) sums
  // FP32 products of rows sl, sl + S, ... in FP32; the slices are added in FP64
  // in slice order.  Then the Procrustes SVD by the CTA's Jacobi.
  float* red = reinterpret_cast<float*>(part);  // kT x 16 partial blocks
  {
    const int NB = K / 4, NBB = NB * NB, S = kT / NBB;
    const int blk = t % NBB, sl = t / NBB;
    const int bi = blk / NB, bj = blk % NB;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = 0.f;
    constexpr int U = 4;  // rows per trip, loads issued before the FMAs
    for (int r0 = sl; r0 < d; r0 += S * U) {
      float4 u[U], v[U];
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const int r = r0 + q * S;
        u[q] = r < d ? *reinterpret_cast<const float4*>(Zi + int64_t(r) * K + 4 * bi) : make_float4(0.f, 0.f, 0.f, 0.f);
        v[q] = r < d ? *reinterpret_cast<const float4*>(Zb + int64_t(r) * K + 4 * bj) : make_float4(0.f, 0.f, 0.f, 0.f);
      }
#pragma unroll
      for (int q = 0; q < U; ++q) {
        const float uu[4] = {u[q].x, u[q].y, u[q].z, u[q].w}, vv[4] = {v[q].x, v[q].y, v[q].z, v[q].w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(uu[a], vv[b], acc[a][b]);
      }
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) red[t * 16 + 4 * a + b] = acc[a][b];
    __syncthreads();
    for (int e = t; e < K * K; e += kT) {
      const int a = e / K, b = e % K;
      const int bb = (a / 4) * NB + b / 4, el = 4 * (a % 4) + b % 4;
      double sum = 0.0;
      for (int q = 0; q < S; ++q) sum += red[(q * NBB + bb) * 16 + el];
      C[e] = sum;
    }
    __syncthreads();
  }
  if (f64) {
    // k x k Procrustes SVD in FP64 (LP_FLAG_KXK_FP64): C = U Sigma V^T, O = U V^T
    const bool ok = cta_jacobi<double>(C, V, k, K);
    if (!ok && t == 0) atomicOr(status, ST_JACOBI);
    procrustes_factor<double>(C, V, part, k, K, Gi, status);
  } else {
    // FP32 copies in the V area (2 K*K floats fit in K*K doubles)
    float* Cf = reinterpret_cast<float*>(V);
    float* Vf = Cf + K * K;
    for (int e = t; e < K * K; e += kT) Cf[e] = static_cast<float>(C[e]);
    __syncthreads();
    const bool ok = cta_jacobi<float>(Cf, Vf, k, K);
    if (!ok && t == 0) atomicOr(status, ST_JACOBI);
    procrustes_factor<float>(Cf, Vf, reinterpret_cast<float*>(part), k, K, Gi, status);
  }
}

// C and V (K x K doubles each), then the partial-block area (kT x 16 floats; it
// also holds the column scales of the Procrustes factor, and the sign path's
// kT doubles)
size_t align_smem(int K) { return size_t(2) * K * K * 8 + size_t(kT) * 16 * 4 + 16; }

// ---------------------------------------------------------------- residual error
// rho_i = ||Z_i G_i - Z_b||_2 (Def. 3) for one partition per CTA: E = Z_i G_i - Z_b
// is formed 64 rows at a time in shared memory (G_i the aligner: K x K, diagonal
// for sign-fixing, nullptr for none); E^T E is summed in FP32 over a chunk and in
// FP64 across chunks; its largest eigenvalue comes from the one-sided Jacobi.
constexpr int kRhoRows = 64;

__global__ void __launch_bounds__(kT) rho_kernel(const float* __restrict__ Zl, int64_t z_stride,
                                                 const float* __restrict__ Zb, const float* __restrict__ G,
                                                 int diag_only, int base, int d, int k, int K,
                                                 double* __restrict__ out, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  double* C = reinterpret_cast<double*>(sm);  // K*K Gram, then Jacobi workspace
  double* V = C + K * K;                       // K*K
  float* E = reinterpret_cast<float*>(V + K * K);  // kRhoRows x K
  const int i = blockIdx.x, t = threadIdx.x;
  if (i == base) {
    if (t == 0) out[i] = 0.0;
    return;
  }
  const float* Zi = Zl + z_stride * i;
  const float* Gi = G ? G + int64_t(i) * K * K : nullptr;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // entries e = t + j * kT of the K x K Gram
  for (int r0 = 0; r0 < d; r0 += kRhoRows) {
    const int nr = min(kRhoRows, d - r0);
    __syncthreads();
    for (int e = t; e < nr * K; e += kT) {
      const int r = r0 + e / K, j = e % K;
      float v;
      if (!Gi) {
        v = Zi[int64_t(r) * K + j];
      } else if (diag_only) {
        v = Zi[int64_t(r) * K + j] * Gi[j * K + j];
      } else {
        v = 0.f;
        for (int l = 0; l < K; ++l) v = fmaf(Zi[int64_t(r) * K + l], Gi[l * K + j], v);
      }
      E[e] = v - Zb[int64_t(r) * K + j];
    }
    __syncthreads();
    for (int q = 0; q < 4; ++q) {
      const int e = t + q * kT;
      if (e >= K * K) break;
      const int a = e / K, b = e % K;
      float s = 0.f;
      if (a < k && b < k)
        for (int r = 0; r < nr; ++r) s = fmaf(E[r * K + a], E[r * K + b], s);
      acc[q] += s;
    }
  }
  __syncthreads();
  for (int q = 0; q < 4; ++q) {
    const int e = t + q * kT;
    if (e < K * K) C[e] = acc[q];
  }
  __syncthreads();
  // E^T E is symmetric positive semidefinite: the one-sided Jacobi's column norms are its eigenvalues
  float* Cf = reinterpret_cast<float*>(V);
  float* Vf = Cf + K * K;
  for (int e = t; e < K * K; e += kT) Cf[e] = static_cast<float>(C[e]);
  __syncthreads();
  const bool ok = cta_jacobi<float>(Cf, Vf, k, K);
  if (!ok && t == 0) atomicOr(status, ST_JACOBI);
  if (t < 32) {
    float top = 0.f;
    for (int j = 0; j < k; ++j) {
      float v = 0.f;
      if (t < k) v = Cf[t * K + j] * Cf[t * K + j];
      v = warp_sumf(v);
      top = fmaxf(top, v);
    }
    if (t == 0) out[i] = sqrt(sqrt(static_cast<double>(top)));  // sqrt(lambda_max(E^T E))
  }
}

// ---------------------------------------------------------------- aggregate
// Y = sum_i w_i Y_i G_i over each problem's partitions (Alg. 1 aggregation; G_i
// the aligner: K x K, diagonal for sign-fixing, or none).  Thread (slice sl,
// row, group jg of four columns) sums the partitions i0 + sl, i0 + sl + S, ... in
// order into four FP32 accumulators, then the S slices are added in slice order
// through shared memory: a fixed summation order for a given S.  RPB = kT /
// (S K/4) rows per CTA; problem q = blockIdx.y sums its own partitions
// [i0, i1) into its own d x K block of Y.
template <int K>
__global__ void __launch_bounds__(kT) aggregate_kernel(const float* __restrict__ Yl, const float* __restrict__ w,
                                                       const float* __restrict__ G, int diag_only, int m, int d, int S,
                                                       const int* __restrict__ prob_begin, float* __restrict__ Y) {
  constexpr int JG = K / 4;
  __shared__ float4 red[kT];
  const int t = threadIdx.x;
  const int RPB = kT / (JG * S);
  const int jg = t % JG, row = (t / JG) % RPB, sl = t / (JG * RPB);
  const int r = blockIdx.x * RPB + row;
  const int q = blockIdx.y;
  const int i0 = prob_begin ? prob_begin[q] : 0, i1 = prob_begin ? prob_begin[q + 1] : m;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  if (r < d) {
    for (int i = i0 + sl; i < i1; i += S) {
      const float* yi = Yl + (int64_t(i) * d + r) * K;
      float4 v;
      if (G == nullptr) {
        v = *reinterpret_cast<const float4*>(yi + 4 * jg);
      } else if (diag_only) {
        const float* gi = G + int64_t(i) * K * K + (4 * jg) * (K + 1);
        const float4 y = *reinterpret_cast<const float4*>(yi + 4 * jg);
        v = make_float4(y.x * gi[0], y.y * gi[K + 1], y.z * gi[2 * (K + 1)], y.w * gi[3 * (K + 1)]);
      } else {
        const float* gi = G + int64_t(i) * K * K + 4 * jg;
        float yr[K];
#pragma unroll
        for (int l = 0; l < K; l += 4) {
          const float4 y = *reinterpret_cast<const float4*>(yi + l);
          yr[l] = y.x;
          yr[l + 1] = y.y;
          yr[l + 2] = y.z;
          yr[l + 3] = y.w;
        }
        v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int l = 0; l < K; ++l) {
          const float4 g = *reinterpret_cast<const float4*>(gi + l * K);
          v.x = fmaf(yr[l], g.x, v.x);
          v.y = fmaf(yr[l], g.y, v.y);
          v.z = fmaf(yr[l], g.z, v.z);
          v.w = fmaf(yr[l], g.w, v.w);
        }
      }
      const float wi = w[i];
      acc.x = fmaf(wi, v.x, acc.x);
      acc.y = fmaf(wi, v.y, acc.y);
      acc.z = fmaf(wi, v.z, acc.z);
      acc.w = fmaf(wi, v.w, acc.w);
    }
  }
  red[t] = acc;
  __syncthreads();
  if (t < RPB * JG) {
    const int row2 = t / JG, jg2 = t % JG;
    const int r2 = blockIdx.x * RPB + row2;
    float4 sum = red[t];
    for (int s2 = 1; s2 < S; ++s2) {
      const float4 o = red[(s2 * RPB + row2) * JG + jg2];
      sum.x += o.x;
      sum.y += o.y;
      sum.z += o.z;
      sum.w += o.w;
    }
    if (r2 < d) reinterpret_cast<float4*>(Y + int64_t(q) * d * K + int64_t(r2) * K)[jg2] = sum;
  }
}

// Zl[i] = Z[part_prob[i]]: each partition's copy of its problem's d x K block
// (batch groups, where the first step of a round multiplies per-problem bases).
__global__ void broadcast_kernel(const float4* __restrict__ Z, const int* __restrict__ part_prob, int m,
                                 int64_t blk4, float4* __restrict__ Zl) {
  const int64_t total = int64_t(m) * blk4;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t i = e / blk4, off = e - i * blk4;
    Zl[e] = Z[int64_t(part_prob[i]) * blk4 + off];
  }
}

// ---------------------------------------------------------------- Ritz
// H = Z^T (M Z) in FP64, split over row slices: block g adds the products of
// its rows (staged in shared memory) into Hpart[g]; ritz_solve adds the slices
// in slice order (deterministic), symmetrises, diagonalises (Jacobi: FP32, or
// FP64 under LP_FLAG_KXK_FP64),
// orders by descending Ritz value and writes sigma and the reordered V;
// ritz_rotate forms Zout = Z V row by row.
constexpr int kRitzRows = 64;  // rows per slice

__global__ void __launch_bounds__(kT) ritz_partial_kernel(const float* __restrict__ Z, const float* __restrict__ MZ,
                                                          int d, int k, int K, double* __restrict__ Hpart) {
  __shared__ float zs[kRitzRows * LP_MAX_K], ms[kRitzRows * LP_MAX_K];
  const int t = threadIdx.x;
  const int r0 = blockIdx.x * kRitzRows;
  // problem blockIdx.y: its d x K blocks and its slices of the scratch
  Z += int64_t(blockIdx.y) * d * K;
  MZ += int64_t(blockIdx.y) * d * K;
  Hpart += int64_t(blockIdx.y) * gridDim.x * K * K;
  const int nr = min(kRitzRows, d - r0);
  for (int e = t; e < nr * K; e += kT) {
    zs[e] = Z[int64_t(r0) * K + e];
    ms[e] = MZ[int64_t(r0) * K + e];
  }
  __syncthreads();
  double* H = Hpart + int64_t(blockIdx.x) * K * K;
  for (int e = t; e < K * K; e += kT) {
    const int a = e / K, b = e % K;
    double sum = 0.0;
    if (a < k && b < k)
      for (int r = 0; r < nr; ++r) sum += static_cast<double>(zs[r * K + a]) * ms[r * K + b];
    H[e] = sum;
  }
}

__global__ void __launch_bounds__(kT) ritz_solve_kernel(const double* __restrict__ Hpart, int slices, int k, int K,
                                                        double n_one, const double* __restrict__ n_of, int f64,
                                                        double* __restrict__ Vo, double* __restrict__ sigma,
                                                        int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  // problem blockIdx.x: its slices, its V and sigma, its row count
  const int qp = blockIdx.x;
  Hpart += int64_t(qp) * slices * K * K;
  Vo += int64_t(qp) * K * K;
  sigma += int64_t(qp) * LP_MAX_K;
  const double n = n_of ? n_of[qp] : n_one;
  double* H = reinterpret_cast<double*>(sm);  // K*K
  double* V = H + K * K;                       // K*K
  double* lam = V + K * K;                     // K
  int* order = reinterpret_cast<int*>(lam + K);
  const int t = threadIdx.x;
  for (int e = t; e < K * K; e += kT) {
    double sum = 0.0;
    for (int g = 0; g < slices; ++g) sum += Hpart[int64_t(g) * K * K + e];
    H[e] = sum;
  }
  __syncthreads();
  // symmetrise: the thread of entry (a, b), a < b, writes both halves
  for (int e = t; e < K * K; e += kT) {
    const int a = e / K, b = e % K;
    if (a < b) {
      const double v = 0.5 * (H[a * K + b] + H[b * K + a]);
      H[a * K + b] = v;
      H[b * K + a] = v;
    }
  }
  __syncthreads();
  // H is symmetric positive semidefinite: its one-sided Jacobi SVD is its
  // eigendecomposition, in FP64 under LP_FLAG_KXK_FP64, else on FP32 copies in
  // the V area.
  if (f64) {
    const bool ok = cta_jacobi<double>(H, V, k, K);
    if (!ok && t == 0) atomicOr(status, ST_JACOBI);
    if (t < k) {
      double v = 0.0;
      for (int r = 0; r < k; ++r) v += H[r * K + t] * H[r * K + t];
      lam[t] = v > 0.0 ? sqrt(v) : 0.0;
    }
  } else {
    float* Hf = reinterpret_cast<float*>(V);
    float* Vf = Hf + K * K;
    for (int e = t; e < K * K; e += kT) Hf[e] = static_cast<float>(H[e]);
    __syncthreads();
    const bool ok = cta_jacobi<float>(Hf, Vf, k, K);
    if (!ok && t == 0) atomicOr(status, ST_JACOBI);
    if (t < k) {
      float v = 0.f;
      for (int r = 0; r < k; ++r) v += Hf[r * K + t] * Hf[r * K + t];
      lam[t] = v > 0.f ? sqrt(static_cast<double>(v)) : 0.0;
    }
  }
  __syncthreads();
  if (t == 0) {
    for (int j = 0; j < k; ++j) order[j] = j;
    for (int a = 0; a < k; ++a)
      for (int b = a + 1; b < k; ++b)
        if (lam[order[b]] > lam[order[a]]) {
          const int tmp = order[a];
          order[a] = order[b];
          order[b] = tmp;
        }
    for (int j = 0; j < k; ++j) sigma[j] = sqrt(n * lam[order[j]]);
  }
  __syncthreads();
  for (int e = t; e < K * K; e += kT) {
    const int l = e / K, j = e % K;
    Vo[e] = j >= k ? 0.0
                   : f64 ? V[l * K + order[j]]
                         : static_cast<double>(reinterpret_cast<const float*>(V)[K * K + l * K + order[j]]);
  }
}

__global__ void ritz_rotate_kernel(const float* __restrict__ Z, const double* __restrict__ Vo, int d, int k, int K,
                                   int nprob, double* __restrict__ Zout) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= int64_t(nprob) * d * k) return;
  // problem q's d x k output block follows problem q - 1's
  const int q = static_cast<int>(e / (int64_t(d) * k));
  const int64_t el = e - int64_t(q) * d * k;
  Z += int64_t(q) * d * K;
  Vo += int64_t(q) * K * K;
  const int r = static_cast<int>(el / k), j = static_cast<int>(el % k);
  double sum = 0.0;
  for (int l = 0; l < k; ++l) sum += static_cast<double>(Z[int64_t(r) * K + l]) * Vo[l * K + j];
  Zout[e] = sum;
}

}  // namespace

cudaError_t allow_max_dynamic_smem(const void* kern) {
  static std::mutex mu;
  static std::unordered_set<const void*> done;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count(kern)) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaFuncAttributes fa{};
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kern);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - static_cast<int>(fa.sharedSizeBytes));
  if (e == cudaSuccess) done.insert(kern);
  return e;
}

cudaError_t launch_split_planes(const float* src, int64_t src_ld, int64_t rows, int d, uint16_t* hi, uint16_t* lo,
                                int64_t ld, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  const int64_t total = rows * ld;
  const int64_t blocks = std::min<int64_t>((total + kT - 1) / kT, 4096);
  split_planes_kernel<<<static_cast<unsigned>(blocks), kT, 0, s>>>(src, src_ld, rows, d, hi, lo, ld);
  return cudaGetLastError();
}

cudaError_t launch_pack(const double* src, float* dst, int batch, int d, int k, int K, cudaStream_t s) {
  const int64_t total = int64_t(batch) * d * K;
  const int64_t nb = (total + kT - 1) / kT;
  const int blocks = static_cast<int>(nb < 4096 ? (nb > 0 ? nb : 1) : 4096);
  pack_kernel<<<blocks, kT, 0, s>>>(src, dst, batch, d, k, K);
  return cudaGetLastError();
}

cudaError_t launch_unpack(const float* src, double* dst, int batch, int d, int k, int K, cudaStream_t s) {
  const int64_t total = int64_t(batch) * d * k;
  const int64_t nb = (total + kT - 1) / kT;
  const int blocks = static_cast<int>(nb < 4096 ? (nb > 0 ? nb : 1) : 4096);
  unpack_kernel<<<blocks, kT, 0, s>>>(src, dst, batch, d, k, K);
  return cudaGetLastError();
}

cudaError_t launch_reduce(const float* P, const int* slot_begin, const float* scale, int m, int d, int K, float* Y,
                          cudaStream_t s, int max_slots) {
  const int64_t n4 = int64_t(d) * K / 4;
  int G = 1;
  while (G < 32 && max_slots > 4 * G) G <<= 1;
  dim3 grid(static_cast<unsigned>((n4 + kT / G - 1) / (kT / G)), static_cast<unsigned>(m));
  switch (G) {
    case 1: reduce_kernel<1><<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y); break;
    case 2: reduce_kernel<2><<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y); break;
    case 4: reduce_kernel<4><<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y); break;
    case 8: reduce_kernel<8><<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y); break;
    case 16: reduce_kernel<16><<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y); break;
    default: reduce_kernel<32><<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_cholqr2(const float* Y, float* Z, int batch, int d, int k, int K, int* status, cudaStream_t s,
                           bool kxk_fp64) {
  switch (K * 2 + (kxk_fp64 ? 1 : 0)) {
    case 16: return launch_cholqr2_t<8, false>(Y, Z, batch, d, k, status, s);
    case 17: return launch_cholqr2_t<8, true>(Y, Z, batch, d, k, status, s);
    case 32: return launch_cholqr2_t<16, false>(Y, Z, batch, d, k, status, s);
    case 33: return launch_cholqr2_t<16, true>(Y, Z, batch, d, k, status, s);
    case 64: return launch_cholqr2_t<32, false>(Y, Z, batch, d, k, status, s);
    case 65: return launch_cholqr2_t<32, true>(Y, Z, batch, d, k, status, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_align(const float* Zl, int64_t z_stride, const float* Zb, int m, int d, int k, int K, int base,
                         lp_aggregator agg, float* G, int* status, cudaStream_t s, bool kxk_fp64,
                         const int* part_base) {
  align_kernel<<<m, kT, align_smem(K), s>>>(Zl, z_stride, Zb, d, k, K, base, part_base, agg == LP_AGG_OPT ? 1 : 0,
                                            kxk_fp64 ? 1 : 0, G, status);
  return cudaGetLastError();
}

cudaError_t launch_aggregate(const float* Yl, const float* w, const float* G, int diag_only, int m, int d, int K,
                             float* Y, cudaStream_t s, const int* prob_begin, int nprob) {
  // slices: a power of two up to the partitions per problem, at most 16
  const int per = nprob > 0 ? m / nprob : m;
  int S = 1;
  while (S * 2 <= per && S * 2 <= 16) S *= 2;
  const int rpb = kT / (K / 4 * S);
  const dim3 grid((d + rpb - 1) / rpb, nprob);
  switch (K) {
    case 4: aggregate_kernel<4><<<grid, kT, 0, s>>>(Yl, w, G, diag_only, m, d, S, prob_begin, Y); break;
    case 8: aggregate_kernel<8><<<grid, kT, 0, s>>>(Yl, w, G, diag_only, m, d, S, prob_begin, Y); break;
    case 16: aggregate_kernel<16><<<grid, kT, 0, s>>>(Yl, w, G, diag_only, m, d, S, prob_begin, Y); break;
    case 32: aggregate_kernel<32><<<grid, kT, 0, s>>>(Yl, w, G, diag_only, m, d, S, prob_begin, Y); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_broadcast(const float* Z, const int* part_prob, int m, int d, int K, float* Zl, cudaStream_t s) {
  const int64_t blk4 = int64_t(d) * K / 4;
  const int64_t total = int64_t(m) * blk4;
  const int blocks = static_cast<int>(std::min<int64_t>((total + kT - 1) / kT, 4096));
  broadcast_kernel<<<blocks > 0 ? blocks : 1, kT, 0, s>>>(reinterpret_cast<const float4*>(Z), part_prob, m, blk4,
                                                          reinterpret_cast<float4*>(Zl));
  return cudaGetLastError();
}

cudaError_t launch_ritz(const float* Z, const float* MZ, int d, int k, int K, double n, double* Zout, double* sigma,
                        double* scratch, int* status, cudaStream_t s, bool kxk_fp64, int nprob, const double* n_of) {
  const int slices = (d + kRitzRows - 1) / kRitzRows;
  double* Hpart = scratch;
  double* Vo = scratch + size_t(nprob) * slices * K * K;
  ritz_partial_kernel<<<dim3(slices, nprob), kT, 0, s>>>(Z, MZ, d, k, K, Hpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = size_t(2) * K * K * 8 + size_t(K) * 8 + size_t(K) * 4 + 16;
  ritz_solve_kernel<<<nprob, kT, sm, s>>>(Hpart, slices, k, K, n, n_of, kxk_fp64 ? 1 : 0, Vo, sigma, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t total = int64_t(nprob) * d * k;
  ritz_rotate_kernel<<<static_cast<unsigned>((total + kT - 1) / kT), kT, 0, s>>>(Z, Vo, d, k, K, nprob, Zout);
  return cudaGetLastError();
}

cudaError_t launch_rho(const float* Zl, int64_t z_stride, const float* Zb, const float* G, int diag_only, int base,
                       int m, int d, int k, int K, double* out, int* status, cudaStream_t s) {
  const size_t sm = size_t(2) * K * K * 8 + size_t(kRhoRows) * K * 4;
  rho_kernel<<<m, kT, sm, s>>>(Zl, z_stride, Zb, G, diag_only, base, d, k, K, out, status);
  return cudaGetLastError();
}

size_t ritz_scratch_bytes(int d, int K, int nprob) {
  const int slices = (d + kRitzRows - 1) / kRitzRows;
  return size_t(nprob) * (size_t(slices) + 1) * K * K * 8;
}

}  // namespace lp
