// sv_simple.cu -- "simple Vanka" (Section 4 / 6.2 of the paper): additive
// Vanka relaxation with an explicitly stored inverse for every patch, the
// baseline that the paper's tuned (shared-inverse) Vanka is compared against.
// FP64 only.  Three kernels, one per step of Algorithm 3, with the
// corrections passing through HBM exactly as in the paper's simple GPU code:
//
//   set-up   k_patch_inverse: assemble each patch matrix A_i = V_i A V_i^T from
//            the stencils and invert it by Gauss-Jordan (one warp per patch);
//   sweep    r = b - A x (k_apply), then k_patch_solve: delta_i = A_i^-1 V_i r
//            (one thread per patch, the inverse streamed from HBM), then
//            k_patch_update: x_out = x + sum_i V_i^T W_i delta_i.
//
// Storage is entry-major: entry e of patch p at e * P + p, P = the patch count
// rounded up to a multiple of 32, so a warp of consecutive patches reads 256
// contiguous bytes per entry.  At 2048^2 the finest level holds 4.2 M inverses
// (87 GB); nothing in them is shared, so memory and traffic grow with n as in
// the paper, where this variant stopped at 768^2 on an 80 GB A100.
#include <cuda_runtime.h>

#include "sv_internal.h"
#include "sv_stencil.cuh"
#include "sv_vanka_common.cuh"

namespace sv {
namespace {

constexpr int NS = 51;                 // slots per patch: 25 u_x, 25 u_y, 1 p
constexpr int INV_WARPS = 4;           // patches per CTA in the set-up kernel

__device__ __forceinline__ bool in_grid(int I, int J, int nq) { return I >= 0 && J >= 0 && I < nq && J < nq; }
__device__ __forceinline__ bool free_node(int I, int J, int nq) {
  return I > 0 && J > 0 && I < nq - 1 && J < nq - 1;
}

// Entry (s, t) of the patch matrix of vertex (pi, pj): the Dirichlet-eliminated
// Stokes operator restricted to the patch's slots; slots on Dirichlet nodes or
// outside the grid carry identity rows (their residual is b - x, or 0).
__device__ double patch_entry(const LevelDev& L, int pi, int pj, int s, int t) {
  const int nq = L.nq;
  if (s == NS - 1 && t == NS - 1) return 0.0;
  if (s == NS - 1 || t == NS - 1) {   // pressure coupling b(v, p) = -int p div v
    const int v = (s == NS - 1) ? t : s;
    const int c = v / 25, w = v % 25;
    const int dI = w % 5 - 2, dJ = w / 5 - 2;
    const int I = 2 * pi + dI, J = 2 * pj + dJ;
    if (!free_node(I, J, nq)) return 0.0;
    return L.cb * (c == 0 ? crow(dI) * nrow(dJ) : nrow(dI) * crow(dJ));
  }
  const int cs = s / 25, ct = t / 25, ws = s % 25, wt = t % 25;
  const int Is = 2 * pi + ws % 5 - 2, Js = 2 * pj + ws / 5 - 2;
  const int It = 2 * pi + wt % 5 - 2, Jt = 2 * pj + wt / 5 - 2;
  const bool fs = free_node(Is, Js, nq), ft = free_node(It, Jt, nq);
  if (!fs || !ft) return (s == t) ? 1.0 : 0.0;
  if (cs != ct) return 0.0;
  const int dI = It - Is, dJ = Jt - Js;
  return L.cl * (k1(Is & 1, dI) * m1(Js & 1, dJ) + m1(Is & 1, dI) * k1(Js & 1, dJ));
}

// One warp per patch: assemble A_i in shared memory, invert in place by
// Gauss-Jordan (velocity slots first: their block is SPD or identity, and the
// last pivot is minus the Schur complement b K^-1 b^T, so no pivoting is
// needed), then the CTA writes its INV_WARPS inverses entry-major.
__global__ void __launch_bounds__(32 * INV_WARPS) k_patch_inverse(LevelDev L, int P, double* __restrict__ inv) {
  pdl_begin();
  extern __shared__ double sa[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int np = L.np, npatch = np * np;
  const int p0 = blockIdx.x * INV_WARPS;
  const int p = p0 + warp;
  double* a = sa + warp * NS * NS;
  if (p < npatch) {
    const int pi = p % np, pj = p / np;
    for (int e = lane; e < NS * NS; e += 32) a[e] = patch_entry(L, pi, pj, e / NS, e % NS);
    __syncwarp();
    for (int k = 0; k < NS; ++k) {
      const double piv = 1.0 / a[k * NS + k];
      __syncwarp();
      for (int j = lane; j < NS; j += 32) a[k * NS + j] = (j == k ? 1.0 : a[k * NS + j]) * piv;
      __syncwarp();
      for (int i = lane; i < NS; i += 32) {
        if (i == k) continue;
        const double f = a[i * NS + k];
        a[i * NS + k] = 0.0;
        for (int j = 0; j < NS; ++j) a[i * NS + j] = fma(-f, a[k * NS + j], a[i * NS + j]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // entry-major store: thread t writes patch p0 + t % INV_WARPS, entries t / INV_WARPS + 32 q
  const int w = threadIdx.x % INV_WARPS;
  if (p0 + w < npatch)
    for (int e = threadIdx.x / INV_WARPS; e < NS * NS; e += 32)
      inv[static_cast<long long>(e) * P + p0 + w] = sa[w * NS * NS + e];
}

// delta_i = A_i^-1 r_i for every patch (one thread each); r is the level's
// residual vector, delta is entry-major like the inverses.
__global__ void __launch_bounds__(128) k_patch_solve(LevelDev L, int P, const double* __restrict__ inv,
                                                     const double* __restrict__ r, double* __restrict__ delta) {
  pdl_begin();
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int np = L.np, nq = L.nq;
  if (p >= np * np) return;
  const int pi = p % np, pj = p / np;
  const long long nv = L.nv;
  double ri[NS];
#pragma unroll
  for (int s = 0; s < 50; ++s) {
    const int c = s / 25, w = s % 25;
    const int I = 2 * pi + w % 5 - 2, J = 2 * pj + w / 5 - 2;
    ri[s] = in_grid(I, J, nq) ? r[c * nv + static_cast<long long>(J) * nq + I] : 0.0;
  }
  ri[50] = r[2 * nv + p];
  const double* A = inv + p;
#pragma unroll 1
  for (int o = 0; o < NS; ++o) {
    double acc = 0.0;
#pragma unroll
    for (int k = 0; k < NS; ++k) acc = fma(A[static_cast<long long>(o * NS + k) * P], ri[k], acc);
    delta[static_cast<long long>(o) * P + p] = acc;
  }
}

// x_out = x + sum over the patches holding each dof of (omega / m_j) delta.
// One thread per vertex (a, b): Q2 nodes (2a + PI, 2b + PJ) of both components
// and p(a, b).  A node 2a + PI lies in the windows of patches a - 1 .. a + 1
// (PI = 0) or a .. a + 1 (PI = 1) on each axis, where they exist.
template <typename T, int PI, int PJ>
__device__ __forceinline__ void update_node(const LevelDev& L, int P, const T* __restrict__ delta,
                                            const T* __restrict__ x, T* __restrict__ xo, T omega, int a, int b) {
  const int I = 2 * a + PI, J = 2 * b + PJ, nq = L.nq, n = L.n, np = L.np;
  if (I >= nq || J >= nq) return;
  const int pil = max(0, a - (PI ? 0 : 1)), pih = min(n, a + 1);
  const int pjl = max(0, b - (PJ ? 0 : 1)), pjh = min(n, b + 1);
  const T w = omega * vk::inv_mult<T>((pih - pil + 1) * (pjh - pjl + 1));
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T acc = T(0);
    for (int pj = pjl; pj <= pjh; ++pj)
      for (int pi = pil; pi <= pih; ++pi) {
        const int slot = c * 25 + (J - 2 * pj + 2) * 5 + (I - 2 * pi + 2);
        acc += delta[static_cast<long long>(slot) * P + pj * np + pi];
      }
    const long long k = c * L.nv + static_cast<long long>(J) * nq + I;
    xo[k] = fma(w, acc, x != nullptr ? x[k] : T(0));
  }
}

// The same for a vertex (a, b) with 1 <= a, b <= n - 1: every patch around its
// nodes exists, so the patch ranges, the slots of the node and the multiplicity
// are compile-time constants; the sum runs in the order of update_node.
template <typename T, int PI, int PJ>
__device__ __forceinline__ void update_node_interior(const LevelDev& L, int P, const T* __restrict__ delta,
                                                     const T* __restrict__ x, T* __restrict__ xo, T omega, int a,
                                                     int b) {
  const int I = 2 * a + PI, J = 2 * b + PJ, nq = L.nq, np = L.np;
  const T w = omega * vk::inv_mult<T>((PI ? 2 : 3) * (PJ ? 2 : 3));
  const T* d0 = delta + static_cast<long long>(b) * np + a;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T acc = T(0);
#pragma unroll
    for (int dj = (PJ ? 0 : -1); dj <= 1; ++dj)
#pragma unroll
      for (int di = (PI ? 0 : -1); di <= 1; ++di) {
        const int slot = c * 25 + (PJ - 2 * dj + 2) * 5 + (PI - 2 * di + 2);
        acc += d0[static_cast<long long>(slot) * P + dj * np + di];
      }
    const long long k = c * L.nv + static_cast<long long>(J) * nq + I;
    xo[k] = fma(w, acc, x != nullptr ? x[k] : T(0));
  }
}

template <typename T>
__global__ void k_patch_update(LevelDev L, int P, const T* __restrict__ delta, const T* __restrict__ x,
                               T* __restrict__ xo, T omega) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > L.n || b > L.n) return;
  if (a >= 1 && b >= 1 && a <= L.n - 1 && b <= L.n - 1) {
    update_node_interior<T, 0, 0>(L, P, delta, x, xo, omega, a, b);
    update_node_interior<T, 1, 0>(L, P, delta, x, xo, omega, a, b);
    update_node_interior<T, 0, 1>(L, P, delta, x, xo, omega, a, b);
    update_node_interior<T, 1, 1>(L, P, delta, x, xo, omega, a, b);
  } else {
    update_node<T, 0, 0>(L, P, delta, x, xo, omega, a, b);
    update_node<T, 1, 0>(L, P, delta, x, xo, omega, a, b);
    update_node<T, 0, 1>(L, P, delta, x, xo, omega, a, b);
    update_node<T, 1, 1>(L, P, delta, x, xo, omega, a, b);
  }
  const int p = b * L.np + a;
  const long long k = 2 * L.nv + p;
  xo[k] = fma(omega, delta[static_cast<long long>(NS - 1) * P + p], x != nullptr ? x[k] : T(0));
}

}  // namespace

int patch_stride(const LevelDev& L) {
  const int npatch = L.np * L.np;
  return (npatch + 31) / 32 * 32;
}

size_t patch_inverse_doubles(const LevelDev& L) { return static_cast<size_t>(NS) * NS * patch_stride(L); }

size_t patch_delta_doubles(const LevelDev& L) { return static_cast<size_t>(NS) * patch_stride(L); }

cudaError_t simple_prepare() {
  return cudaFuncSetAttribute(k_patch_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>(INV_WARPS * NS * NS * sizeof(double)));
}

void launch_patch_inverse(const LevelDev& L, double* inv, cudaStream_t s) {
  count_launches(1);
  const int npatch = L.np * L.np;
  launch_pdl(k_patch_inverse, dim3((npatch + INV_WARPS - 1) / INV_WARPS), dim3(32 * INV_WARPS), INV_WARPS * NS * NS * sizeof(double), s, 
      L, patch_stride(L), inv);
}

template <typename T>
void launch_patch_update(const LevelDev& L, int P, const T* delta, const T* x, T* xo, double omega, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  launch_pdl(k_patch_update<T>, dim3(dim3((L.np + 31) / 32, (L.np + 7) / 8)), dim3(blk), 0, s, L, P, delta, x, xo, T(omega));
}
template void launch_patch_update<double>(const LevelDev&, int, const double*, const double*, double*, double,
                                          cudaStream_t);
template void launch_patch_update<float>(const LevelDev&, int, const float*, const float*, float*, double,
                                         cudaStream_t);

void launch_simple_sweep(const LevelDev& L, const double* inv, double* delta, double* rscratch, const double* x,
                         const double* b, double* xo, double omega, cudaStream_t s) {
  const int P = patch_stride(L), npatch = L.np * L.np;
  const double* r = b;
  if (x != nullptr) {
    launch_apply<double>(L, x, b, rscratch, 1, s);
    r = rscratch;
  }
  count_launches(1);
  launch_pdl(k_patch_solve, dim3((npatch + 127) / 128), dim3(128), 0, s, L, P, inv, r, delta);
  launch_patch_update(L, P, delta, x, xo, omega, s);
}

}  // namespace sv
