// The local-approximation measure of Def. 2 (Sec. 4):
//   eta = max_i ||M_i - M||_2 / ||M||_2,  M_i = (1/s_i) A_i^T A_i,  M = sum_i p_i M_i.
// The M_i come from the fused step kernel itself: a step on Z = columns
// [c0, c0 + K) of the identity returns M_i Z, i.e. K columns of every M_i, so
// ceil(d / K) steps over A give all of them, in the precision of a solve's
// steps.  The kernels here turn those blocks into the matrices whose norms are
// wanted and measure the norms:
//   identity_block   Z = [e_c0 .. e_{c0+K-1}]
//   scatter_columns  the step's Y_i blocks -> rows c0.. of the d x d slots
//   deviations       M = sum_i p_i sym(M_i) (FP64 sums) into slot m, D_i = sym(M_i) - M in place
//   lanczos_norms    ||D_i||_2 and ||M||_2: one CTA per matrix runs Lanczos with
//                    full reorthogonalisation (FP32 vectors); the extreme
//                    eigenvalues of its tridiagonal matrix come from Sturm-count
//                    bisection in FP64.
#include <algorithm>
#include <cfloat>
#include <cstdint>

#include "lp_internal.cuh"

namespace lp {
namespace {

constexpr int kLzThreads = 512;
constexpr int kLzWarps = kLzThreads / 32;
constexpr int kMaxLanczos = 256;

__global__ void identity_block_kernel(float* __restrict__ Z, int d, int K, int c0) {
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= int64_t(d) * K) return;
  const int r = static_cast<int>(e / K), j = static_cast<int>(e % K);
  Z[e] = r == c0 + j ? 1.f : 0.f;
}

// Slot i row (c0 + j) = column j of Y_i (d x K block); M_i is symmetric, so the
// slot holds M_i^T until the deviation pass symmetrises it.
__global__ void scatter_columns_kernel(const float* __restrict__ Y, float* __restrict__ Mall, int d, int K, int c0,
                                       int ncols) {
  const int i = blockIdx.y;
  const int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x;
  if (e >= int64_t(ncols) * d) return;
  const int j = static_cast<int>(e / d), r = static_cast<int>(e % d);
  const size_t dd = size_t(d) * d;
  Mall[i * dd + size_t(c0 + j) * d + r] = Y[(size_t(i) * d + r) * K + j];
}

// One thread per unordered pair (r <= c): reads entries (r, c) and (c, r) of
// every slot, writes both, so no two threads touch the same element.
__global__ void deviations_kernel(float* __restrict__ Mall, const float* __restrict__ w, int m, int d) {
  const size_t dd = size_t(d) * d;
  for (size_t e = blockIdx.x * size_t(blockDim.x) + threadIdx.x; e < dd; e += size_t(gridDim.x) * blockDim.x) {
    const int r = static_cast<int>(e / d), c = static_cast<int>(e % d);
    if (r > c) continue;
    const size_t rc = size_t(r) * d + c, cr = size_t(c) * d + r;
    double mean = 0.0;
    for (int i = 0; i < m; ++i)
      mean += double(w[i]) * 0.5 * (double(Mall[i * dd + rc]) + double(Mall[i * dd + cr]));
    for (int i = 0; i < m; ++i) {
      const double s = 0.5 * (double(Mall[i * dd + rc]) + double(Mall[i * dd + cr]));
      const float dv = static_cast<float>(s - mean);
      Mall[i * dd + rc] = dv;
      Mall[i * dd + cr] = dv;
    }
    Mall[size_t(m) * dd + rc] = static_cast<float>(mean);
    Mall[size_t(m) * dd + cr] = static_cast<float>(mean);
  }
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum over the CTA, returned to every thread.  `red` holds kLzWarps + 1 floats.
__device__ float block_sum(float v, float* red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  v = warp_sum(v);
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    float t = lane < kLzWarps ? red[lane] : 0.f;
    t = warp_sum(t);
    if (lane == 0) red[kLzWarps] = t;
  }
  __syncthreads();
  const float s = red[kLzWarps];
  __syncthreads();
  return s;
}

// Number of eigenvalues of the symmetric tridiagonal (a, b) below x (Sturm
// sequence of the LDL^T pivots).
__device__ int sturm_below(const double* a, const double* b, int n, double x, double pivmin) {
  int cnt = 0;
  double q = a[0] - x;
  for (int i = 0;;) {
    if (q < 0.0) ++cnt;
    if (++i == n) break;
    if (fabs(q) < pivmin) q = -pivmin;
    q = a[i] - x - b[i - 1] * b[i - 1] / q;
  }
  return cnt;
}

// The idx-th smallest eigenvalue (0-based) by bisection inside [lo, hi].
__device__ double tridiag_eig(const double* a, const double* b, int n, int idx, double lo, double hi, double pivmin) {
  for (int it = 0; it < 120 && hi - lo > 1e-15 * fmax(fabs(lo), fabs(hi)) + 1e-300; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (sturm_below(a, b, n, mid, pivmin) > idx) hi = mid;
    else lo = mid;
  }
  return 0.5 * (lo + hi);
}

// A fixed pseudo-random start vector entry in [-1, 1) (splitmix64 of the index).
__device__ __forceinline__ float start_entry(int c) {
  uint64_t z = 0x9E3779B97F4A7C15ull * (uint64_t(c) + 1);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return static_cast<float>(static_cast<double>(z >> 11) * (2.0 / 9007199254740992.0) - 1.0);
}

// out[mat] = ||S||_2 of the symmetric d x d matrix S = Mall slot `mat`: the
// largest |eigenvalue| of the Lanczos tridiagonal after min(L, breakdown) steps.
// V holds the Lanczos vectors (L x d per matrix).
__global__ void __launch_bounds__(kLzThreads) lanczos_norms_kernel(const float* __restrict__ Mall, int d, int L,
                                                                   float* __restrict__ Vall, double* __restrict__ out) {
  extern __shared__ __align__(16) float lz[];
  float* v = lz;       // current Lanczos vector
  float* w = v + d;    // S v, then the next residual
  float* h = w + d;    // reorthogonalisation coefficients (L)
  __shared__ float red[kLzWarps + 1];
  __shared__ double alpha[kMaxLanczos], beta[kMaxLanczos];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int mat = blockIdx.x;
  const float* S = Mall + size_t(mat) * d * d;
  float* V = Vall + size_t(mat) * L * d;

  float ss = 0.f;
  for (int c = tid; c < d; c += kLzThreads) {
    const float x = start_entry(c);
    v[c] = x;
    ss += x * x;
  }
  const float inv0 = rsqrtf(block_sum(ss, red));
  for (int c = tid; c < d; c += kLzThreads) v[c] *= inv0;
  __syncthreads();

  int steps = 0;
  float anorm = 0.f;
  for (int j = 0; j < L; ++j) {
    for (int c = tid; c < d; c += kLzThreads) V[size_t(j) * d + c] = v[c];
    // w = S v (a warp per row, coalesced along the row)
    for (int r = warp; r < d; r += kLzWarps) {
      const float* row = S + size_t(r) * d;
      float s = 0.f;
      for (int c = lane; c < d; c += 32) s = fmaf(row[c], v[c], s);
      s = warp_sum(s);
      if (lane == 0) w[r] = s;
    }
    __syncthreads();
    float part = 0.f;
    for (int c = tid; c < d; c += kLzThreads) part = fmaf(v[c], w[c], part);
    const float a = block_sum(part, red);
    if (tid == 0) alpha[j] = a;
    const float bprev = j > 0 ? static_cast<float>(beta[j - 1]) : 0.f;
    for (int c = tid; c < d; c += kLzThreads) {
      float x = w[c] - a * v[c];
      if (j > 0) x -= bprev * V[size_t(j - 1) * d + c];
      w[c] = x;
    }
    __syncthreads();
    // full reorthogonalisation against v_0 .. v_j, twice (classical Gram-Schmidt)
    for (int pass = 0; pass < 2; ++pass) {
      for (int i = warp; i <= j; i += kLzWarps) {
        const float* vi = V + size_t(i) * d;
        float s = 0.f;
        for (int c = lane; c < d; c += 32) s = fmaf(vi[c], w[c], s);
        s = warp_sum(s);
        if (lane == 0) h[i] = s;
      }
      __syncthreads();
      for (int c = tid; c < d; c += kLzThreads) {
        float t = 0.f;
        for (int i = 0; i <= j; ++i) t = fmaf(h[i], V[size_t(i) * d + c], t);
        w[c] -= t;
      }
      __syncthreads();
    }
    part = 0.f;
    for (int c = tid; c < d; c += kLzThreads) part = fmaf(w[c], w[c], part);
    const float b = sqrtf(block_sum(part, red));
    anorm = fmaxf(anorm, fabsf(a) + b + bprev);
    steps = j + 1;
    // breakdown: the Krylov space is invariant (exact for d steps, or S = 0)
    if (j + 1 == L || !(b > 1e-6f * anorm)) break;
    if (tid == 0) beta[j] = b;
    const float inv = 1.f / b;
    for (int c = tid; c < d; c += kLzThreads) v[c] = w[c] * inv;
    __syncthreads();
  }
  __syncthreads();

  // extreme eigenvalues of the steps x steps tridiagonal; Gershgorin bounds
  __shared__ double ext[2];
  if (tid == 0 || tid == 32) {
    double lo = DBL_MAX, hi = -DBL_MAX, scale = 0.0;
    for (int i = 0; i < steps; ++i) {
      const double off = (i > 0 ? fabs(beta[i - 1]) : 0.0) + (i + 1 < steps ? fabs(beta[i]) : 0.0);
      lo = fmin(lo, alpha[i] - off);
      hi = fmax(hi, alpha[i] + off);
      scale = fmax(scale, fabs(alpha[i]) + off);
    }
    const double pad = 1e-12 * scale + 1e-300;
    const double pivmin = 1e-290 + 1e-30 * scale * scale;
    ext[tid == 0 ? 0 : 1] = tridiag_eig(alpha, beta, steps, tid == 0 ? 0 : steps - 1, lo - pad, hi + pad, pivmin);
  }
  __syncthreads();
  if (tid == 0) {
    const double e = fmax(fabs(ext[0]), fabs(ext[1]));
    out[mat] = isfinite(ext[0]) && isfinite(ext[1]) && isfinite(anorm) ? e : NAN;
  }
}

}  // namespace

int lanczos_steps(int d) { return d < kMaxLanczos ? d : kMaxLanczos; }

size_t lanczos_smem(int d) { return size_t(4) * (2 * size_t(d) + kMaxLanczos); }

cudaError_t launch_identity_block(float* Z, int d, int K, int c0, cudaStream_t s) {
  const int64_t total = int64_t(d) * K;
  identity_block_kernel<<<static_cast<unsigned>((total + 255) / 256), 256, 0, s>>>(Z, d, K, c0);
  return cudaGetLastError();
}

cudaError_t launch_scatter_columns(const float* Y, float* Mall, int m, int d, int K, int c0, int ncols,
                                   cudaStream_t s) {
  const int64_t total = int64_t(ncols) * d;
  scatter_columns_kernel<<<dim3(static_cast<unsigned>((total + 255) / 256), m), 256, 0, s>>>(Y, Mall, d, K, c0,
                                                                                              ncols);
  return cudaGetLastError();
}

cudaError_t launch_deviations(float* Mall, const float* w, int m, int d, cudaStream_t s) {
  const size_t dd = size_t(d) * d;
  const unsigned blocks = static_cast<unsigned>(std::min<size_t>((dd + 255) / 256, 152 * 32));
  deviations_kernel<<<blocks, 256, 0, s>>>(Mall, w, m, d);
  return cudaGetLastError();
}

cudaError_t launch_lanczos_norms(const float* Mall, int nmat, int d, float* V, double* out, cudaStream_t s) {
  const size_t smem = lanczos_smem(d);
  cudaError_t e = allow_max_dynamic_smem(reinterpret_cast<const void*>(lanczos_norms_kernel));
  if (e != cudaSuccess) return e;
  lanczos_norms_kernel<<<nmat, kLzThreads, smem, s>>>(Mall, d, lanczos_steps(d), V, out);
  return cudaGetLastError();
}

}  // namespace lp
