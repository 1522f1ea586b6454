// sv_krylov.cu -- FP64 kernels of FGMRES (Section 6.8): the Arnoldi step's
// Gram-Schmidt, either modified (one launch per basis vector: the previous
// vector's update fused with the next one's dot) or classical as two fused
// passes (all dots plus ||w||^2 in one read of V and w; the update w -= V h
// plus the new ||w||^2 in another), with a second pass only when the first lost
// more than half of ||w||^2 (the DGKS test, decided on the device); scaling,
// Givens rotations and the small triangular solve.  Every reduction is
// two-stage (warp shuffles, then the last block to finish sums the per-block
// partials in block order), so each result is deterministic.
#include <cuda_runtime.h>

#include <cmath>

#include "sv_internal.h"

namespace sv {
namespace {

constexpr int DOT_NT = 256;
constexpr int ORTH_KMAX = 16;  // basis vectors per fused Gram-Schmidt launch
constexpr int DOT_BLOCKS = 152 * 4;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---- fused Gram-Schmidt passes ----
// Loads kept in flight per thread: U elements of each of the K + 1 vectors.
template <int K>
constexpr int orth_unroll() { return K <= 1 ? 4 : (K <= 4 ? 2 : 1); }

// Reduces acc[0..NO) over the block into partials[t * npart + blockIdx.x] and
// returns, in every thread, whether this block is the last of the grid to
// finish (its partials then see all others').  The last block resets *ticket.
template <int NO>
__device__ __forceinline__ bool block_partials(const double (&acc)[NO], double* __restrict__ partials,
                                               int npart, unsigned* ticket) {
  __shared__ double red[DOT_NT / 32][NO];
  __shared__ unsigned last;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NO; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) red[wid][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NO) {
    double s = 0.0;
#pragma unroll
    for (int q = 0; q < DOT_NT / 32; ++q) s += red[q][threadIdx.x];
    partials[static_cast<long long>(threadIdx.x) * npart + blockIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(ticket, 1u) == gridDim.x - 1) ? 1u : 0u;
  __syncthreads();
  return last != 0u;
}

// In the last block: tot[t] = sum over blocks b (in a fixed order) of
// partials[t * npart + b], t < NO; one warp per output.
template <int NO>
__device__ __forceinline__ void total_partials(const double* __restrict__ partials, int npart,
                                               double (&tot)[NO]) {
  __shared__ double sh[NO];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = wid; t < NO; t += DOT_NT / 32) {
    double v = 0.0;
    for (int b = lane; b < npart; b += 32) v += __ldcg(partials + static_cast<long long>(t) * npart + b);
    v = warp_sum(v);
    if (lane == 0) sh[t] = v;
  }
  __syncthreads();
#pragma unroll
  for (int t = 0; t < NO; ++t) tot[t] = sh[t];
}

// Pass 1 of Gram-Schmidt: dots[k] = <V_k, w> (k < K) and, if NORM,
// norm2[0] = <w, w>, norm2[1] = sqrt(norm2[0]).  Skipped when *gate == 0.
template <int K, bool NORM>
__global__ void __launch_bounds__(DOT_NT) k_orth_dots(const double* __restrict__ V, long long ld,
                                                      const double* __restrict__ w, long long N,
                                                      double* __restrict__ partials, int npart,
                                                      unsigned* ticket, double* __restrict__ dots,
                                                      double* __restrict__ norm2,
                                                      const double* __restrict__ gate) {
  pdl_begin();
  if (gate != nullptr && *gate == 0.0) return;
  constexpr int NO = K + (NORM ? 1 : 0);
  constexpr int U = orth_unroll<K>();
  double acc[NO];
#pragma unroll
  for (int k = 0; k < NO; ++k) acc[k] = 0.0;
  const long long stride = static_cast<long long>(gridDim.x) * DOT_NT;
  long long i = blockIdx.x * static_cast<long long>(DOT_NT) + threadIdx.x;
  for (; i + (U - 1) * stride < N; i += U * stride) {
    double wv[U], vv[U][K > 0 ? K : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wv[u] = w[i + u * stride];
#pragma unroll
      for (int k = 0; k < K; ++k) vv[u][k] = V[k * ld + i + u * stride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fma(vv[u][k], wv[u], acc[k]);
      if (NORM) acc[NO - 1] = fma(wv[u], wv[u], acc[NO - 1]);
    }
  }
  for (; i < N; i += stride) {
    const double wi = w[i];
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fma(V[k * ld + i], wi, acc[k]);
    if (NORM) acc[NO - 1] = fma(wi, wi, acc[NO - 1]);
  }
  if (!block_partials<NO>(acc, partials, npart, ticket)) return;
  double tot[NO];
  total_partials<NO>(partials, npart, tot);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) dots[k] = tot[k];
    if (NORM) {
      norm2[0] = tot[NO - 1];
      norm2[1] = sqrt(tot[NO - 1]);
    }
    *ticket = 0u;
  }
}

// Pass 2 of Gram-Schmidt: w -= sum_{k<K} coef[k] V_k and, if NORM, norm2[0] =
// <w, w> of the updated w, norm2[1] = its square root.  In the last block,
// when dgks_ref is given, *flag = 1 if norm2[0] < dgks_ref / 2 (re-orthogonalise)
// else 0; when hacc is given, hacc[t] += coef_all[t] for t < nacc.  Skipped
// when *gate == 0.
template <int K, bool NORM>
__global__ void __launch_bounds__(DOT_NT) k_orth_update(double* __restrict__ w, const double* __restrict__ V,
                                                        long long ld, const double* __restrict__ coef,
                                                        long long N, double* __restrict__ partials, int npart,
                                                        unsigned* ticket, double* __restrict__ norm2,
                                                        const double* __restrict__ gate,
                                                        const double* __restrict__ dgks_ref,
                                                        double* __restrict__ flag, double* __restrict__ hacc,
                                                        const double* __restrict__ coef_all, int nacc) {
  pdl_begin();
  if (gate != nullptr && *gate == 0.0) return;
  constexpr int U = orth_unroll<K>();
  double c[K > 0 ? K : 1];
#pragma unroll
  for (int k = 0; k < K; ++k) c[k] = coef[k];
  double acc[1] = {0.0};
  const long long stride = static_cast<long long>(gridDim.x) * DOT_NT;
  long long i = blockIdx.x * static_cast<long long>(DOT_NT) + threadIdx.x;
  for (; i + (U - 1) * stride < N; i += U * stride) {
    double wv[U], vv[U][K > 0 ? K : 1];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wv[u] = w[i + u * stride];
#pragma unroll
      for (int k = 0; k < K; ++k) vv[u][k] = V[k * ld + i + u * stride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      double x = wv[u];
#pragma unroll
      for (int k = 0; k < K; ++k) x = fma(-c[k], vv[u][k], x);
      w[i + u * stride] = x;
      if (NORM) acc[0] = fma(x, x, acc[0]);
    }
  }
  for (; i < N; i += stride) {
    double x = w[i];
#pragma unroll
    for (int k = 0; k < K; ++k) x = fma(-c[k], V[k * ld + i], x);
    w[i] = x;
    if (NORM) acc[0] = fma(x, x, acc[0]);
  }
  if (!block_partials<1>(acc, partials, npart, ticket)) return;
  double tot[1];
  total_partials<1>(partials, npart, tot);
  if (threadIdx.x == 0) {
    if (NORM) {
      norm2[0] = tot[0];
      norm2[1] = sqrt(tot[0]);
      if (dgks_ref != nullptr) *flag = (tot[0] < 0.5 * *dgks_ref) ? 1.0 : 0.0;
    }
    if (hacc != nullptr)
      for (int t = 0; t < nacc; ++t) hacc[t] += coef_all[t];
    *ticket = 0u;
  }
}

// Pass 1's update fused with pass 2's dots: w' = w - sum_{k<K} coef[k] V_k,
// dots[k] = <V_k, w'>, norm2[0] = <w', w'>, norm2[1] = its square root, and
// *flag = 1 if norm2[0] < dgks_ref / 2 (re-orthogonalise) else 0.  Each w'
// element is formed in registers next to the V elements that it is dotted with,
// so V is read once for both; the values equal those of the two passes run
// apart.
template <int K>
__global__ void __launch_bounds__(DOT_NT) k_orth_update_dots(double* __restrict__ w, const double* __restrict__ V,
                                                             long long ld, const double* __restrict__ coef,
                                                             long long N, double* __restrict__ partials,
                                                             int npart, unsigned* ticket,
                                                             double* __restrict__ dots,
                                                             double* __restrict__ norm2,
                                                             const double* __restrict__ dgks_ref,
                                                             double* __restrict__ flag) {
  pdl_begin();
  constexpr int NO = K + 1;
  constexpr int U = orth_unroll<K>();
  double c[K];
#pragma unroll
  for (int k = 0; k < K; ++k) c[k] = coef[k];
  double acc[NO];
#pragma unroll
  for (int k = 0; k < NO; ++k) acc[k] = 0.0;
  const long long stride = static_cast<long long>(gridDim.x) * DOT_NT;
  long long i = blockIdx.x * static_cast<long long>(DOT_NT) + threadIdx.x;
  for (; i + (U - 1) * stride < N; i += U * stride) {
    double wv[U], vv[U][K];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      wv[u] = w[i + u * stride];
#pragma unroll
      for (int k = 0; k < K; ++k) vv[u][k] = V[k * ld + i + u * stride];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      double x = wv[u];
#pragma unroll
      for (int k = 0; k < K; ++k) x = fma(-c[k], vv[u][k], x);
      w[i + u * stride] = x;
#pragma unroll
      for (int k = 0; k < K; ++k) acc[k] = fma(vv[u][k], x, acc[k]);
      acc[K] = fma(x, x, acc[K]);
    }
  }
  for (; i < N; i += stride) {
    double vk[K];
#pragma unroll
    for (int k = 0; k < K; ++k) vk[k] = V[k * ld + i];
    double x = w[i];
#pragma unroll
    for (int k = 0; k < K; ++k) x = fma(-c[k], vk[k], x);
    w[i] = x;
#pragma unroll
    for (int k = 0; k < K; ++k) acc[k] = fma(vk[k], x, acc[k]);
    acc[K] = fma(x, x, acc[K]);
  }
  if (!block_partials<NO>(acc, partials, npart, ticket)) return;
  double tot[NO];
  total_partials<NO>(partials, npart, tot);
  if (threadIdx.x == 0) {
#pragma unroll
    for (int k = 0; k < K; ++k) dots[k] = tot[k];
    norm2[0] = tot[K];
    norm2[1] = sqrt(tot[K]);
    *flag = (tot[K] < 0.5 * *dgks_ref) ? 1.0 : 0.0;
    *ticket = 0u;
  }
}

// One step of modified Gram-Schmidt, in the order of the textbook loop: if UPD,
// w -= coef[0] Va (coef[0] the dot the previous step produced); then, if DOT,
// dots[0] = <Vb, w>, and, if NORM, norm2[0] = <w, w> and norm2[1] = its square
// root, both of the updated w.  Every element costs at most two FP64 FMAs against
// three vectors read and one written, so a step streams HBM: on a GPU whose FP64
// rate is 1/64 of its FP32 rate this is cheaper per basis vector than classical
// Gram-Schmidt with a second pass, which spends four FMAs per element and vector.
template <bool UPD, bool DOT, bool NORM>
__global__ void __launch_bounds__(DOT_NT) k_mgs_step(double* __restrict__ w, const double* __restrict__ Va,
                                                     const double* __restrict__ Vb,
                                                     const double* __restrict__ coef, long long N,
                                                     double* __restrict__ partials, int npart, unsigned* ticket,
                                                     double* __restrict__ dots, double* __restrict__ norm2) {
  pdl_begin();
  constexpr int NO = (DOT ? 1 : 0) + (NORM ? 1 : 0);
  static_assert(NO > 0, "a step produces a dot or a norm");
  constexpr int U = 4;
  const double c = UPD ? coef[0] : 0.0;
  double acc[NO];
#pragma unroll
  for (int k = 0; k < NO; ++k) acc[k] = 0.0;
  auto step = [&](long long i, double x, double va, double vb) {
    if (UPD) {
      x = fma(-c, va, x);
      w[i] = x;
    }
    if (DOT) acc[0] = fma(vb, x, acc[0]);
    if (NORM) acc[NO - 1] = fma(x, x, acc[NO - 1]);
  };
  const long long stride = static_cast<long long>(gridDim.x) * DOT_NT;
  long long i = blockIdx.x * static_cast<long long>(DOT_NT) + threadIdx.x;
  for (; i + (U - 1) * stride < N; i += U * stride) {
    double x[U], va[U], vb[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      x[u] = w[i + u * stride];
      va[u] = UPD ? Va[i + u * stride] : 0.0;
      vb[u] = DOT ? Vb[i + u * stride] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < U; ++u) step(i + u * stride, x[u], va[u], vb[u]);
  }
  for (; i < N; i += stride) step(i, w[i], UPD ? Va[i] : 0.0, DOT ? Vb[i] : 0.0);
  if (!block_partials<NO>(acc, partials, npart, ticket)) return;
  double tot[NO];
  total_partials<NO>(partials, npart, tot);
  if (threadIdx.x == 0) {
    if (DOT) dots[0] = tot[0];
    if (NORM) {
      norm2[0] = tot[NO - 1];
      norm2[1] = sqrt(tot[NO - 1]);
    }
    *ticket = 0u;
  }
}

// out[k] (+)= sum_b partials[k * npart + b]; one CTA per k
__global__ void k_reduce(const double* __restrict__ partials, int npart, double* __restrict__ out,
                         int accumulate) {
  pdl_begin();
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
  pdl_begin();
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
  pdl_begin();
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
  pdl_begin();
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    p[i] = v;
}

// Column j of the Hessenberg matrix: H[0..j] = hcol, H[j+1] = hnorm.  Apply the
// previous rotations, build rotation j, update g; est = |g[j+1]|.
__global__ void k_givens(double* H, int ldh, double* cs, double* sn, double* g,
                         const double* hcol, const double* hnorm, int j, double* est) {
  pdl_begin();
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
  pdl_begin();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[static_cast<long long>(c) * ldh + i] * y[c];
    const double d = H[static_cast<long long>(i) * ldh + i];
    y[i] = (d != 0.0) ? s / d : 0.0;
  }
}

__global__ void k_dirichlet_copy(LevelDev L, const double* __restrict__ src, double* __restrict__ dst) {
  pdl_begin();
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
  pdl_begin();
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
  pdl_begin();
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
std::atomic<long long> g_tc_launches{0};

int dot_blocks() { return DOT_BLOCKS; }

template <int K>
void dots_k(bool norm, const double* V, long long ld, const double* w, long long N, double* partials,
            int npart, unsigned* ticket, double* dots, double* norm2, const double* gate, cudaStream_t s) {
  if constexpr (K == 0) {
    (void)norm;   // zero vectors: only the norm (callers pass norm2)
    launch_pdl(k_orth_dots<0, true>, dim3(npart), dim3(DOT_NT), 0, s, V, ld, w, N, partials, npart, ticket, dots, norm2, gate);
  } else if (norm) {
    launch_pdl(k_orth_dots<K, true>, dim3(npart), dim3(DOT_NT), 0, s, V, ld, w, N, partials, npart, ticket, dots, norm2, gate);
  } else {
    launch_pdl(k_orth_dots<K, false>, dim3(npart), dim3(DOT_NT), 0, s, V, ld, w, N, partials, npart, ticket, dots, norm2, gate);
  }
}

template <int K>
void update_k(bool norm, double* w, const double* V, long long ld, const double* coef, long long N,
              double* partials, int npart, unsigned* ticket, double* norm2, const double* gate,
              const double* dgks_ref, double* flag, double* hacc, const double* coef_all, int nacc,
              cudaStream_t s) {
  if (norm)
    launch_pdl(k_orth_update<K, true>, dim3(npart), dim3(DOT_NT), 0, s, w, V, ld, coef, N, partials, npart, ticket, norm2, gate,
                                                    dgks_ref, flag, hacc, coef_all, nacc);
  else
    launch_pdl(k_orth_update<K, false>, dim3(npart), dim3(DOT_NT), 0, s, w, V, ld, coef, N, partials, npart, ticket, norm2, gate,
                                                     dgks_ref, flag, hacc, coef_all, nacc);
}

template <int K>
void update_dots_k(double* w, const double* V, long long ld, const double* coef, long long N, double* partials,
                   int npart, unsigned* ticket, double* dots, double* norm2, const double* dgks_ref, double* flag,
                   cudaStream_t s) {
  if constexpr (K == 0) {
    (void)w;   // never launched: the caller passes at least one vector
  } else {
    launch_pdl(k_orth_update_dots<K>, dim3(npart), dim3(DOT_NT), 0, s, w, V, ld, coef, N, partials, npart, ticket, dots, norm2,
                                                   dgks_ref, flag);
  }
}

#define SV_ORTH_CASES(F, ...) \
  switch (kk) {                                    \
    case 0: F<0>(__VA_ARGS__); break;              \
    case 1: F<1>(__VA_ARGS__); break;              \
    case 2: F<2>(__VA_ARGS__); break;              \
    case 3: F<3>(__VA_ARGS__); break;              \
    case 4: F<4>(__VA_ARGS__); break;              \
    case 5: F<5>(__VA_ARGS__); break;              \
    case 6: F<6>(__VA_ARGS__); break;              \
    case 7: F<7>(__VA_ARGS__); break;              \
    case 8: F<8>(__VA_ARGS__); break;              \
    case 9: F<9>(__VA_ARGS__); break;              \
    case 10: F<10>(__VA_ARGS__); break;            \
    case 11: F<11>(__VA_ARGS__); break;            \
    case 12: F<12>(__VA_ARGS__); break;            \
    case 13: F<13>(__VA_ARGS__); break;            \
    case 14: F<14>(__VA_ARGS__); break;            \
    case 15: F<15>(__VA_ARGS__); break;            \
    default: F<16>(__VA_ARGS__); break;            \
  }

void launch_orth_dots(const double* V, long long ld, int nk, const double* w, long long N, double* partials,
                      int npart, unsigned* ticket, double* dots, double* norm2, const double* gate,
                      cudaStream_t s) {
  // chunks of ORTH_KMAX vectors; the first chunk also takes ||w||^2
  int k0 = 0;
  do {
    const int kk = (nk - k0 < ORTH_KMAX) ? nk - k0 : ORTH_KMAX;
    const bool norm = (k0 == 0) && norm2 != nullptr;
    count_launches(1);
    SV_ORTH_CASES(dots_k, norm, V + k0 * ld, ld, w, N, partials, npart, ticket, dots + k0, norm2, gate, s)
    k0 += kk;
  } while (k0 < nk);
}

void launch_orth_update(double* w, const double* V, long long ld, int nk, const double* coef, long long N,
                        double* partials, int npart, unsigned* ticket, double* norm2, const double* gate,
                        const double* dgks_ref, double* flag, double* hacc, cudaStream_t s) {
  // chunks of ORTH_KMAX vectors; the last chunk takes the norm, the flag and hacc
  int k0 = 0;
  do {
    const int kk = (nk - k0 < ORTH_KMAX) ? nk - k0 : ORTH_KMAX;
    const bool lastc = (k0 + kk >= nk);
    count_launches(1);
    SV_ORTH_CASES(update_k, lastc && norm2 != nullptr, w, V + k0 * ld, ld, coef + k0, N, partials, npart,
                  ticket, norm2, gate, lastc ? dgks_ref : nullptr, flag, lastc ? hacc : nullptr, coef, nk, s)
    k0 += kk;
  } while (k0 < nk);
}

bool launch_orth_update_dots(double* w, const double* V, long long ld, int nk, const double* coef, long long N,
                             double* partials, int npart, unsigned* ticket, double* dots, double* norm2,
                             const double* dgks_ref, double* flag, cudaStream_t s) {
  if (nk < 1 || nk > ORTH_KMAX) return false;   // one launch holds at most ORTH_KMAX vectors
  const int kk = nk;
  count_launches(1);
  SV_ORTH_CASES(update_dots_k, w, V, ld, coef, N, partials, npart, ticket, dots, norm2, dgks_ref, flag, s)
  return true;
}

#undef SV_ORTH_CASES

void launch_mgs_step(double* w, const double* Va, const double* Vb, const double* coef, long long N,
                     double* partials, int npart, unsigned* ticket, double* dots, double* norm2, cudaStream_t s) {
  if (Va == nullptr && Vb == nullptr) return;   // a step reads at least one basis vector
  count_launches(1);
  const dim3 g(npart), b(DOT_NT);
  if (Va == nullptr)   // the first step: <V_0, w> and ||w||^2
    launch_pdl(k_mgs_step<false, true, true>, g, b, 0, s, w, Va, Vb, coef, N, partials, npart, ticket, dots, norm2);
  else if (Vb == nullptr)   // the last step: w -= h_j V_j and the new ||w||^2
    launch_pdl(k_mgs_step<true, false, true>, g, b, 0, s, w, Va, Vb, coef, N, partials, npart, ticket, dots, norm2);
  else
    launch_pdl(k_mgs_step<true, true, false>, g, b, 0, s, w, Va, Vb, coef, N, partials, npart, ticket, dots, norm2);
}

void launch_multiaxpy(double* w, const double* V, long long ld, int nk, const double* coef,
                      double sign, long long N, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_multiaxpy, dim3(grid_for(N, 256)), dim3(256), 0, s, w, V, ld, nk, coef, sign, N);
}

void launch_scale(double* y, const double* x, const double* den, double scal, long long N,
                  cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_scale, dim3(grid_for(N, 256)), dim3(256), 0, s, y, x, den, scal, N);
}

void launch_givens(double* H, int ldh, double* cs, double* sn, double* g, const double* hcol,
                   const double* hnorm, int j, double* est, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_givens, dim3(1), dim3(32), 0, s, H, ldh, cs, sn, g, hcol, hnorm, j, est);
}

void launch_backsolve(const double* H, int ldh, const double* g, int k, double* y, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_backsolve, dim3(1), dim3(32), 0, s, H, ldh, g, k, y);
}

void launch_fill(double* p, double v, long long N, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_fill, dim3(grid_for(N, 256)), dim3(256), 0, s, p, v, N);
}

void launch_project_pressure(const LevelDev& L, const double* x, double* y, double* partials, int npart,
                             double* sum, cudaStream_t s) {
  count_launches(3);
  const long long p0 = 2 * L.nv, np2 = static_cast<long long>(L.np) * L.np;
  launch_pdl(k_partial_sum, dim3(npart), dim3(DOT_NT), 0, s, x + p0, np2, partials);
  launch_pdl(k_reduce, dim3(1), dim3(256), 0, s, partials, npart, sum, 0);
  launch_pdl(k_copy_shift_pressure, dim3(grid_for(L.N, 256)), dim3(256), 0, s, x, y, L.N, p0, sum, 1.0 / static_cast<double>(np2));
}

void launch_dirichlet_copy(const LevelDev& L, const double* src, double* dst, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_dirichlet_copy, dim3(grid_for(L.N, 256)), dim3(256), 0, s, L, src, dst);
}

}  // namespace sv
