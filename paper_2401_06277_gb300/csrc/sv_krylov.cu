// sv_krylov.cu -- FP64 kernels of FGMRES (Section 6.8): fused multi-dot
// products (classical Gram-Schmidt, applied twice), fused multi-axpy, scaling,
// Givens rotations and the small triangular solve.  Reductions are two-stage
// (warp shuffles, then one CTA over the per-block partials in a fixed order),
// so every result is deterministic.
#include <cuda_runtime.h>

#include <cmath>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int DOT_NT = 256;
constexpr int DOT_KMAX = 16;   // vectors per multi-dot pass
constexpr int DOT_BLOCKS = 152 * 4;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// partials[k * npart + blockIdx.x] = sum over this block's elements of V_k[i] w[i]
__global__ void __launch_bounds__(DOT_NT) k_multidot(const double* __restrict__ V, long long ld,
                                                     int nk, const double* __restrict__ w,
                                                     long long N, double* __restrict__ partials,
                                                     int npart) {
  double acc[DOT_KMAX];
#pragma unroll
  for (int k = 0; k < DOT_KMAX; ++k) acc[k] = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(DOT_NT) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * DOT_NT) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < DOT_KMAX; ++k)
      if (k < nk) acc[k] = fma(V[k * ld + i], wi, acc[k]);
  }
  __shared__ double red[DOT_NT / 32][DOT_KMAX];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < DOT_KMAX; ++k) {
    if (k < nk) {
      const double v = warp_sum(acc[k]);
      if (lane == 0) red[wid][k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x < nk) {
    double s = 0.0;
    for (int q = 0; q < DOT_NT / 32; ++q) s += red[q][threadIdx.x];
    partials[static_cast<long long>(threadIdx.x) * npart + blockIdx.x] = s;
  }
}

// out[k] (+)= sum_b partials[k * npart + b]; one CTA per k
__global__ void k_reduce(const double* __restrict__ partials, int npart, double* __restrict__ out,
                         int accumulate) {
  const int k = blockIdx.x;
  double s = 0.0;
  for (int b = threadIdx.x; b < npart; b += blockDim.x) s += partials[static_cast<long long>(k) * npart + b];
  __shared__ double red[32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    v = warp_sum(v);
    if (threadIdx.x == 0) out[k] = accumulate ? out[k] + v : v;
  }
}

__global__ void k_multiaxpy(double* __restrict__ w, const double* __restrict__ V, long long ld,
                            int nk, const double* __restrict__ coef, double sign, long long N) {
  __shared__ double c[64];
  if (threadIdx.x < nk) c[threadIdx.x] = sign * coef[threadIdx.x];
  __syncthreads();
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    double s = w[i];
    for (int k = 0; k < nk; ++k) s = fma(c[k], V[k * ld + i], s);
    w[i] = s;
  }
}

__global__ void k_scale(double* __restrict__ y, const double* __restrict__ x,
                        const double* __restrict__ den, double scal, long long N) {
  double f = scal;
  if (den != nullptr) {
    const double d = *den;
    f = (d != 0.0) ? 1.0 / d : 0.0;
  }
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = x[i] * f;
}

__global__ void k_fill(double* __restrict__ p, double v, long long N) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    p[i] = v;
}

// *p = sqrt(*src)
__global__ void k_sqrt(double* p, const double* src) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *p = sqrt(*src);
}

// Column j of the Hessenberg matrix: H[0..j] = hcol, H[j+1] = hnorm.  Apply the
// previous rotations, build rotation j, update g; est = |g[j+1]|.
__global__ void k_givens(double* H, int ldh, double* cs, double* sn, double* g,
                         const double* hcol, const double* hnorm, int j, double* est) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double* h = H + static_cast<long long>(j) * ldh;
  for (int i = 0; i <= j; ++i) h[i] = hcol[i];
  h[j + 1] = *hnorm;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * h[i] + sn[i] * h[i + 1];
    h[i + 1] = -sn[i] * h[i] + cs[i] * h[i + 1];
    h[i] = t;
  }
  const double d = hypot(h[j], h[j + 1]);
  double c = 1.0, s = 0.0;
  if (d != 0.0) {
    c = h[j] / d;
    s = h[j + 1] / d;
  }
  cs[j] = c;
  sn[j] = s;
  h[j] = d;
  h[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  *est = fabs(g[j + 1]);
}

// Solve the k x k upper-triangular system H y = g (columns of H have stride ldh).
__global__ void k_backsolve(const double* H, int ldh, const double* g, int k, double* y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[static_cast<long long>(c) * ldh + i] * y[c];
    const double d = H[static_cast<long long>(i) * ldh + i];
    y[i] = (d != 0.0) ? s / d : 0.0;
  }
}

__global__ void k_add_small(double* a, const double* b, int n) {
  if (threadIdx.x < n) a[threadIdx.x] += b[threadIdx.x];
}

__global__ void k_dirichlet_copy(LevelDev L, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = L.N;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x) {
    double v = 0.0;
    if (i < 2 * L.nv) {
      const long long k = i % L.nv;
      const int J = static_cast<int>(k / L.nq), I = static_cast<int>(k - static_cast<long long>(J) * L.nq);
      if (I == 0 || J == 0 || I == L.nq - 1 || J == L.nq - 1) v = src[i];
    }
    dst[i] = v;
  }
}

// partials[b] = sum over this block's elements of x (deterministic two-stage sum with k_reduce)
__global__ void __launch_bounds__(DOT_NT) k_partial_sum(const double* __restrict__ x, long long N,
                                                        double* __restrict__ partials) {
  double acc = 0.0;
  for (long long i = blockIdx.x * static_cast<long long>(DOT_NT) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * DOT_NT)
    acc += x[i];
  acc = warp_sum(acc);
  __shared__ double red[DOT_NT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < DOT_NT / 32; ++q) s += red[q];
    partials[blockIdx.x] = s;
  }
}

// y = x, with the pressure block shifted by -(*sum)/np2 (zero mean)
__global__ void k_copy_shift_pressure(const double* __restrict__ x, double* __restrict__ y, long long N,
                                      long long p0, const double* __restrict__ sum, double inv_np2) {
  const double m = *sum * inv_np2;
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    y[i] = (i >= p0) ? x[i] - m : x[i];
}

int grid_for(long long N, int nt) {
  long long b = (N + nt - 1) / nt;
  if (b > 152 * 8) b = 152 * 8;
  if (b < 1) b = 1;
  return static_cast<int>(b);
}

}  // namespace

std::atomic<long long> g_launches{0};

int dot_blocks() { return DOT_BLOCKS; }

void launch_multidot(const double* V, long long ld, int nk, const double* w, long long N,
                     double* partials, int npart, double* out, int accumulate, cudaStream_t s) {
  for (int k0 = 0; k0 < nk; k0 += DOT_KMAX) {
    const int kk = (nk - k0 < DOT_KMAX) ? nk - k0 : DOT_KMAX;
    count_launches(2);
    k_multidot<<<npart, DOT_NT, 0, s>>>(V + k0 * ld, ld, kk, w, N, partials, npart);
    k_reduce<<<kk, 256, 0, s>>>(partials, npart, out + k0, accumulate);
  }
}

void launch_multiaxpy(double* w, const double* V, long long ld, int nk, const double* coef,
                      double sign, long long N, cudaStream_t s) {
  count_launches(1);
  k_multiaxpy<<<grid_for(N, 256), 256, 0, s>>>(w, V, ld, nk, coef, sign, N);
}

void launch_scale(double* y, const double* x, const double* den, double scal, long long N,
                  cudaStream_t s) {
  count_launches(1);
  k_scale<<<grid_for(N, 256), 256, 0, s>>>(y, x, den, scal, N);
}

void launch_givens(double* H, int ldh, double* cs, double* sn, double* g, const double* hcol,
                   const double* hnorm, int j, double* est, cudaStream_t s) {
  count_launches(1);
  k_givens<<<1, 32, 0, s>>>(H, ldh, cs, sn, g, hcol, hnorm, j, est);
}

void launch_backsolve(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t s) {
  count_launches(1);
  k_backsolve<<<1, 32, 0, s>>>(H, ldh, g, k, y);
}

void launch_fill(double* p, double v, long long N, cudaStream_t s) {
  count_launches(1);
  k_fill<<<grid_for(N, 256), 256, 0, s>>>(p, v, N);
}

void launch_set_scalar(double* p, const double* src_sqrt, cudaStream_t s) {
  count_launches(1);
  k_sqrt<<<1, 32, 0, s>>>(p, src_sqrt);
}

void launch_add_small(double* a, const double* b, int n, cudaStream_t s) {
  count_launches(1);
  k_add_small<<<1, 64, 0, s>>>(a, b, n);
}

void launch_project_pressure(const LevelDev& L, const double* x, double* y, double* partials, int npart,
                             double* sum, cudaStream_t s) {
  count_launches(3);
  const long long p0 = 2 * L.nv, np2 = static_cast<long long>(L.np) * L.np;
  k_partial_sum<<<npart, DOT_NT, 0, s>>>(x + p0, np2, partials);
  k_reduce<<<1, 256, 0, s>>>(partials, npart, sum, 0);
  k_copy_shift_pressure<<<grid_for(L.N, 256), 256, 0, s>>>(x, y, L.N, p0, sum, 1.0 / static_cast<double>(np2));
}

void launch_dirichlet_copy(const LevelDev& L, const double* src, double* dst, cudaStream_t s) {
  count_launches(1);
  k_dirichlet_copy<<<grid_for(L.N, 256), 256, 0, s>>>(L, src, dst);
}

}  // namespace sv
