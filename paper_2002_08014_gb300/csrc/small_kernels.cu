// The d x k and k x k kernels around the fused power step:
//   reduce     Y_i = (1/s_i) sum of the step kernel's per-CTA partials (fixed order)
//   cholqr2    Z = orth(Y) by two passes of Gram / Cholesky / triangular solve
//   align      sign-fixing (eq. (4)) or orthogonal Procrustes (eq. (3)) matrices
//   aggregate  Y = sum_i p_i Y_i D_i (Alg. 1 aggregation)
//   ritz       Rayleigh-Ritz on span(Z): ordered basis and sigma_j = sqrt(n lambda_j)
// Precision: the d-sized work (Gram, solves, averaging) is FP32; the k x k
// factorisations (Cholesky, triangular inverse, Jacobi SVD / eigen) are FP64,
// as are the sign-fix inner products that decide D_i.
#include <algorithm>
#include <cfloat>

#include <cuda_bf16.h>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP64 1/sqrt(x) and 1/x by Newton-Raphson iteration from FP32 seeds
// (y <- y (3 - x y^2) / 2 and y <- y (2 - x y)); each step doubles the number of
// correct bits, so two steps take the FP32 seed (about 2^-22) past FP64
// precision.  FP64 square roots and divisions are long instruction sequences on
// this GPU; these are a few FMAs on the short k x k critical paths.  Arguments
// outside the FP32 normal range take the plain sqrt / division.
__device__ __forceinline__ double rsqrt_nr(double x) {
  if (!(x > 1e-30 && x < 1e30)) return 1.0 / sqrt(x);
  double y = static_cast<double>(rsqrtf(static_cast<float>(x)));
  const double hx = 0.5 * x;
  y = y * (1.5 - hx * y * y);
  y = y * (1.5 - hx * y * y);
  return y;
}
__device__ __forceinline__ double recip_nr(double x) {
  const double ax = fabs(x);
  if (!(ax > 1e-30 && ax < 1e30)) return 1.0 / x;
  double y = static_cast<double>(__frcp_rn(static_cast<float>(x)));
  y = y * (2.0 - x * y);
  y = y * (2.0 - x * y);
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
__global__ void reduce_kernel(const float* __restrict__ P, const int* __restrict__ slot_begin,
                              const float* __restrict__ scale, int d, int K, float* __restrict__ Y) {
  const int i = blockIdx.y;
  const int64_t n4 = int64_t(d) * K / 4;
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= n4) return;
  const int sb = slot_begin[i], se = slot_begin[i + 1];
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int s = sb; s < se; ++s) {
    const float4 v = reinterpret_cast<const float4*>(P + int64_t(s) * d * K)[e];
    acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
  }
  const float sc = scale[i];
  acc.x *= sc; acc.y *= sc; acc.z *= sc; acc.w *= sc;
  reinterpret_cast<float4*>(Y + int64_t(i) * d * K)[e] = acc;
}

// ---------------------------------------------------------------- k x k helpers (warp 0, FP64)
// One-sided (Hestenes) Jacobi on the k x k matrix C (stride K, in smem), accumulating the
// rotations in V.  On return C's columns are mutually orthogonal: C_in V = C_out, so
// C_in = U Sigma V^T with sigma_j = ||C_out[:, j]||, U[:, j] = C_out[:, j] / sigma_j.
// Returns false if the sweep limit was hit.
__device__ bool warp_jacobi(double* C, double* V, int k, int K) {
  const int lane = threadIdx.x & 31;
  for (int r = lane; r < k; r += 32)
    for (int j = 0; j < k; ++j) V[r * K + j] = (r == j) ? 1.0 : 0.0;
  __syncwarp();
  const double tol = 1e-14;
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int p = 0; p < k - 1; ++p) {
      for (int q = p + 1; q < k; ++q) {
        double a = 0.0, b = 0.0, g = 0.0;
        if (lane < k) {
          const double cp = C[lane * K + p], cq = C[lane * K + q];
          a = cp * cp;
          b = cq * cq;
          g = cp * cq;
        }
        a = warp_sum(a);
        b = warp_sum(b);
        g = warp_sum(g);
        if (g * g > tol * tol * (a * b) && fabs(g) > 1e-300) {
          rotated = 1;
          // zeta = (b - a) / 2g, t = sgn(zeta) / (|zeta| + sqrt(1 + zeta^2)), c = 1 / sqrt(1 + t^2)
          const double zeta = (b - a) * recip_nr(2.0 * g);
          const double q2 = 1.0 + zeta * zeta;
          const double t = (zeta >= 0.0 ? 1.0 : -1.0) * recip_nr(fabs(zeta) + q2 * rsqrt_nr(q2));
          const double c = rsqrt_nr(1.0 + t * t);
          const double s = c * t;
          if (lane < k) {
            const double cp = C[lane * K + p], cq = C[lane * K + q];
            C[lane * K + p] = c * cp - s * cq;
            C[lane * K + q] = s * cp + c * cq;
            const double vp = V[lane * K + p], vq = V[lane * K + q];
            V[lane * K + p] = c * vp - s * vq;
            V[lane * K + q] = s * vp + c * vq;
          }
          __syncwarp();
        }
      }
    }
    if (!rotated) return true;
  }
  return false;
}

// ---------------------------------------------------------------- CholQR2
// One CTA per block, two passes of:
//   G = Y^T Y        FP32 products and partial sums over row slices, combined in FP64
//   G = L L^T        FP64 right-looking Cholesky on warp 0 (parallel trailing updates)
//   Z = Y L^{-T}     per-row forward substitution in FP32, one thread per row
// The column space is Y's whatever the precision of L; the second pass restores
// orthonormality lost to the FP32 Gram.  A pivot that is not positive and finite
// sets ST_CHOL (the pivot is then taken as 1 so the kernel can finish).
// G = Y^T Y: thread (block (bi, bj) of 4 x 4 entries, row slice) accumulates
// Y[r][4bi..4bi+3]^T Y[r][4bj..4bj+3] over its rows in FP32 registers (16 FMAs
// per two 16-byte loads); the slices are added in FP64 through shared memory.
template <int K>
__device__ void gram_fp32(const float* __restrict__ Y, int d, float* red, double* G) {
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
    double s = 0.0;
    for (int q = 0; q < S; ++q) s += red[(q * NBB + bb) * 16 + el];
    G[e] = s;
  }
  __syncthreads();
}

// Right-looking Cholesky of G (k x k, stride K, FP64, overwritten) by one warp.
// Writes L in FP32 (lower, stride K) and 1 / L[j][j] in FP32; returns false on breakdown.
template <int K>
__device__ bool warp_cholesky_rl(double* G, float* Lf, float* invd, int k) {
  const int lane = threadIdx.x & 31;
  bool ok = true;
  for (int j = 0; j < k; ++j) {
    double piv = G[j * K + j];
    if (!(piv > 0.0) || !isfinite(piv)) {
      ok = false;
      piv = 1.0;
    }
    const double inv = rsqrt_nr(piv);
    const double ljj = piv * inv;
    // column j below the diagonal
    for (int i = j + 1 + lane; i < k; i += 32) G[i * K + j] *= inv;
    if (lane == 0) {
      G[j * K + j] = ljj;
      invd[j] = static_cast<float>(inv);
    }
    __syncwarp();
    // trailing update G[i][l] -= L[i][j] L[l][j] for j < l <= i < k
    const int m = k - j - 1;
    for (int e = lane; e < m * m; e += 32) {
      const int i = j + 1 + e / m, l = j + 1 + e % m;
      if (l <= i) G[i * K + l] -= G[i * K + j] * G[l * K + j];
    }
    __syncwarp();
  }
  for (int e = lane; e < K * K; e += 32) {
    const int i = e / K, l = e % K;
    Lf[e] = (i < k && l <= i) ? static_cast<float>(G[e]) : 0.f;
  }
  __syncwarp();
  return ok;
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

template <int K>
__global__ void __launch_bounds__(kT) cholqr2_kernel(const float* __restrict__ Yall, float* __restrict__ Zall, int d,
                                                     int k, int* status) {
  __shared__ __align__(16) double G[K * K];
  __shared__ __align__(16) float Lf[K * K];
  __shared__ float invd[K];
  __shared__ __align__(16) float red[kT * 16];
  const float* Y = Yall + int64_t(blockIdx.x) * d * K;
  float* Z = Zall + int64_t(blockIdx.x) * d * K;
  for (int pass = 0; pass < 2; ++pass) {
    const float* src = pass == 0 ? Y : Z;
    gram_fp32<K>(src, d, red, G);
    if (threadIdx.x < 32) {
      const bool ok = warp_cholesky_rl<K>(G, Lf, invd, k);
      if (!ok && threadIdx.x == 0) atomicOr(status, ST_CHOL);
    }
    __syncthreads();
    forward_rows<K>(src, Z, Lf, invd, d, k);
    __syncthreads();
  }
}

// ---------------------------------------------------------------- align
// One CTA per partition.  G_i (K x K float, row-major) = D_i (sign) or O_i (OPT).
__global__ void __launch_bounds__(kT) align_kernel(const float* __restrict__ Zl, int64_t z_stride,
                                                   const float* __restrict__ Zb, int d, int k, int K, int base,
                                                   int opt, float* __restrict__ Gout, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
  double* C = reinterpret_cast<double*>(sm);   // K*K
  double* V = C + K * K;                        // K*K
  double* part = V + K * K;                     // kT doubles
  const int i = blockIdx.x;
  const int t = threadIdx.x;
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
  // OPT: C = Z_i^T Z_b (FP32 products, FP32 partial sums, FP64 combine), SVD by Jacobi.
  const int NP = K * K;
  const int RS = NP >= kT ? 1 : kT / NP;
  const int PP = NP >= kT ? NP / kT : 1;
  for (int pp = 0; pp < PP; ++pp) {
    const int idx = t + kT * pp;
    const int pair = idx % NP, sl = idx / NP;
    const int a = pair / K, b = pair % K;
    float s = 0.f;
    if (sl < RS)
      for (int r = sl; r < d; r += RS) s = fmaf(Zi[int64_t(r) * K + a], Zb[int64_t(r) * K + b], s);
    if (RS > 1) part[t] = s;
    else C[idx] = s;
  }
  __syncthreads();
  if (RS > 1) {
    if (t < NP) {
      double s = 0.0;
      for (int sl = 0; sl < RS; ++sl) s += part[sl * NP + t];
      C[t] = s;
    }
    __syncthreads();
  }
  if (t < 32) {
    const bool ok = warp_jacobi(C, V, k, K);
    if (!ok && t == 0) atomicOr(status, ST_JACOBI);
    // U[:, j] = C[:, j] / sigma_j ; O = U V^T
    for (int j = 0; j < k; ++j) {
      double nrm = 0.0;
      if (t < k) nrm = C[t * K + j] * C[t * K + j];
      nrm = warp_sum(nrm);  // squared norm
      const double inv = nrm > 1e-300 ? rsqrt_nr(nrm) : 0.0;
      if (t < k) C[t * K + j] *= inv;
      if (!(nrm > 1e-300) && t == 0) atomicOr(status, ST_JACOBI);
    }
    __syncwarp();
    for (int e = t; e < K * K; e += 32) {
      const int a = e / K, b = e % K;
      double s = 0.0;
      if (a < k && b < k)
        for (int j = 0; j < k; ++j) s += C[a * K + j] * V[b * K + j];
      Gi[e] = static_cast<float>(s);
    }
  }
}

size_t align_smem(int K) { return size_t(2) * K * K * 8 + size_t(kT) * 8 + 16; }

// ---------------------------------------------------------------- aggregate
__global__ void aggregate_kernel(const float* __restrict__ Yl, const float* __restrict__ w,
                                 const float* __restrict__ G, int diag_only, int m, int d, int K,
                                 float* __restrict__ Y) {
  const int t = threadIdx.x;
  const int j = t % K;
  const int r = blockIdx.x * (kT / K) + t / K;
  if (r >= d) return;
  float acc = 0.f;
  for (int i = 0; i < m; ++i) {
    const float* yi = Yl + (int64_t(i) * d + r) * K;
    float v;
    if (G == nullptr) {
      v = yi[j];
    } else if (diag_only) {
      v = yi[j] * G[int64_t(i) * K * K + j * K + j];
    } else {
      const float* gi = G + int64_t(i) * K * K;
      v = 0.f;
      for (int l = 0; l < K; ++l) v = fmaf(yi[l], gi[l * K + j], v);
    }
    acc = fmaf(w[i], v, acc);
  }
  Y[int64_t(r) * K + j] = acc;
}

// ---------------------------------------------------------------- Ritz
// H = Z^T (M Z) in FP64, split over row slices: block g adds the products of
// its rows (staged in shared memory) into Hpart[g]; ritz_solve adds the slices
// in slice order (deterministic), symmetrises, diagonalises (FP64 Jacobi),
// orders by descending Ritz value and writes sigma and the reordered V;
// ritz_rotate forms Zout = Z V row by row.
constexpr int kRitzRows = 64;  // rows per slice

__global__ void __launch_bounds__(kT) ritz_partial_kernel(const float* __restrict__ Z, const float* __restrict__ MZ,
                                                          int d, int k, int K, double* __restrict__ Hpart) {
  __shared__ float zs[kRitzRows * LP_MAX_K], ms[kRitzRows * LP_MAX_K];
  const int t = threadIdx.x;
  const int r0 = blockIdx.x * kRitzRows;
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
                                                        double n, double* __restrict__ Vo,
                                                        double* __restrict__ sigma, int* status) {
  extern __shared__ __align__(16) unsigned char sm[];
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
  if (t < 32) {
    // symmetrise
    for (int e = t; e < K * K; e += 32) {
      const int a = e / K, b = e % K;
      if (a < b) {
        const double v = 0.5 * (H[a * K + b] + H[b * K + a]);
        H[a * K + b] = v;
        H[b * K + a] = v;
      }
    }
    __syncwarp();
    // H is symmetric positive semidefinite: its one-sided Jacobi SVD is its eigendecomposition.
    const bool ok = warp_jacobi(H, V, k, K);
    if (!ok && t == 0) atomicOr(status, ST_JACOBI);
    for (int j = 0; j < k; ++j) {
      double v = 0.0;
      if (t < k) v = H[t * K + j] * H[t * K + j];
      v = warp_sum(v);
      if (t == 0) lam[j] = v > 0.0 ? v * rsqrt_nr(v) : 0.0;
    }
    __syncwarp();
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
    __syncwarp();
  }
  __syncthreads();
  for (int e = t; e < K * K; e += kT) {
    const int l = e / K, j = e % K;
    Vo[e] = j < k ? V[l * K + order[j]] : 0.0;
  }
}

__global__ void ritz_rotate_kernel(const float* __restrict__ Z, const double* __restrict__ Vo, int d, int k, int K,
                                   double* __restrict__ Zout) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= int64_t(d) * k) return;
  const int r = static_cast<int>(e / k), j = static_cast<int>(e % k);
  double sum = 0.0;
  for (int l = 0; l < k; ++l) sum += static_cast<double>(Z[int64_t(r) * K + l]) * Vo[l * K + j];
  Zout[e] = sum;
}

}  // namespace

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
                          cudaStream_t s) {
  const int64_t n4 = int64_t(d) * K / 4;
  dim3 grid(static_cast<unsigned>((n4 + kT - 1) / kT), static_cast<unsigned>(m));
  reduce_kernel<<<grid, kT, 0, s>>>(P, slot_begin, scale, d, K, Y);
  return cudaGetLastError();
}

cudaError_t launch_cholqr2(const float* Y, float* Z, int batch, int d, int k, int K, int* status, cudaStream_t s) {
  switch (K) {
    case 8: cholqr2_kernel<8><<<batch, kT, 0, s>>>(Y, Z, d, k, status); break;
    case 16: cholqr2_kernel<16><<<batch, kT, 0, s>>>(Y, Z, d, k, status); break;
    case 32: cholqr2_kernel<32><<<batch, kT, 0, s>>>(Y, Z, d, k, status); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_align(const float* Zl, int64_t z_stride, const float* Zb, int m, int d, int k, int K, int base,
                         lp_aggregator agg, float* G, int* status, cudaStream_t s) {
  align_kernel<<<m, kT, align_smem(K), s>>>(Zl, z_stride, Zb, d, k, K, base, agg == LP_AGG_OPT ? 1 : 0, G, status);
  return cudaGetLastError();
}

cudaError_t launch_aggregate(const float* Yl, const float* w, const float* G, int diag_only, int m, int d, int K,
                             float* Y, cudaStream_t s) {
  const int rpb = kT / K;
  aggregate_kernel<<<(d + rpb - 1) / rpb, kT, 0, s>>>(Yl, w, G, diag_only, m, d, K, Y);
  return cudaGetLastError();
}

cudaError_t launch_ritz(const float* Z, const float* MZ, int d, int k, int K, double n, double* Zout, double* sigma,
                        double* scratch, int* status, cudaStream_t s) {
  const int slices = (d + kRitzRows - 1) / kRitzRows;
  double* Hpart = scratch;
  double* Vo = scratch + size_t(slices) * K * K;
  ritz_partial_kernel<<<slices, kT, 0, s>>>(Z, MZ, d, k, K, Hpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t sm = size_t(2) * K * K * 8 + size_t(K) * 8 + size_t(K) * 4 + 16;
  ritz_solve_kernel<<<1, kT, sm, s>>>(Hpart, slices, k, K, n, Vo, sigma, status);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  const int64_t total = int64_t(d) * k;
  ritz_rotate_kernel<<<static_cast<unsigned>((total + kT - 1) / kT), kT, 0, s>>>(Z, Vo, d, k, K, Zout);
  return cudaGetLastError();
}

size_t ritz_scratch_bytes(int d, int K) {
  const int slices = (d + kRitzRows - 1) / kRitzRows;
  return (size_t(slices) + 1) * K * K * 8;
}

}  // namespace lp
