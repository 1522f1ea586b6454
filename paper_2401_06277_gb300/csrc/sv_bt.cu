// sv_bt.cu -- kernels of the block-triangular preconditioner (Section 3.4,
// Algorithm 5): scalar multigrid on the pressure mass matrix M and on the
// velocity Laplacian L, each smoothed by weighted Jacobi.  Both work on the
// full [u_x | u_y | p] layout with the other block held at zero, so the grid
// transfers of the Stokes V-cycle (block diagonal) serve unchanged; every
// kernel here writes exact zeros into the block it does not own.
//
//   Q1 mass, 1D row of vertex i in units of h/6: [1 4 1] inside, [2 1] / [1 2]
//   at the ends (one element); M = (h/6)^2 (m (x) m).
//   diag(L) on a free Q2 node: nu/90 times 224 / 352 / 512 by node parities; 1 on
//   Dirichlet rows (identity in the eliminated operator).
#include <cuda_runtime.h>

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace sv {
namespace {

__device__ __forceinline__ double q1m(int i, int d, int n) {
  if (d == 0) return (i == 0 || i == n) ? 2.0 : 4.0;
  const int k = i + d;
  return (k < 0 || k > n) ? 0.0 : 1.0;
}

// y_p = b_p - M x_p (x may be nullptr: y_p = b_p); y_u = 0
__global__ void k_mass_resid(LevelDev L, const double* __restrict__ x, const double* __restrict__ b,
                             double* __restrict__ y) {
  pdl_begin();
  const long long N = L.N, p0 = 2 * L.nv;
  const int n = L.n, np = L.np;
  const double c = (L.h / 6.0) * (L.h / 6.0);
  for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < N;
       k += static_cast<long long>(gridDim.x) * blockDim.x) {
    if (k < p0) {
      y[k] = 0.0;
      continue;
    }
    const int v = static_cast<int>(k - p0), i = v % np, j = v / np;
    double s = 0.0;
    if (x != nullptr) {
#pragma unroll
      for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
        for (int di = -1; di <= 1; ++di) {
          const double w = q1m(i, di, n) * q1m(j, dj, n);
          if (w != 0.0) s = fma(w, x[p0 + static_cast<long long>(j + dj) * np + (i + di)], s);
        }
    }
    y[k] = b[k] - c * s;
  }
}

// xo = x + omega D^-1 r on the owned block, 0 on the other (x may be nullptr);
// block 0: velocity (D = diag L), block 1: pressure (D = diag M)
__global__ void k_block_jacobi(LevelDev L, int block, const double* __restrict__ x, const double* __restrict__ r,
                               double* __restrict__ xo, double omega) {
  pdl_begin();
  const long long N = L.N, p0 = 2 * L.nv;
  const int n = L.n, np = L.np, nq = L.nq;
  const double cm = (L.h / 6.0) * (L.h / 6.0);
  for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < N;
       k += static_cast<long long>(gridDim.x) * blockDim.x) {
    const bool vel = k < p0;
    if (vel != (block == 0)) {
      xo[k] = 0.0;
      continue;
    }
    double d;
    if (vel) {
      const long long kk = k % L.nv;
      const int J = static_cast<int>(kk / nq), I = static_cast<int>(kk - static_cast<long long>(J) * nq);
      const bool fr = I > 0 && J > 0 && I < nq - 1 && J < nq - 1;
      d = fr ? L.cl * (k1(I, 0) * m1(J, 0) + m1(I, 0) * k1(J, 0)) : 1.0;
    } else {
      const int v = static_cast<int>(k - p0), i = v % np, j = v / np;
      d = cm * q1m(i, 0, n) * q1m(j, 0, n);
    }
    xo[k] = fma(omega / d, r[k], x != nullptr ? x[k] : 0.0);
  }
}

__global__ void k_add(double* __restrict__ y, const double* __restrict__ x, long long N) {
  pdl_begin();
  for (long long k = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; k < N;
       k += static_cast<long long>(gridDim.x) * blockDim.x)
    y[k] += x[k];
}

int grid_for_bt(long long N) {
  long long b = (N + 255) / 256;
  if (b > 152 * 8) b = 152 * 8;
  return static_cast<int>(b < 1 ? 1 : b);
}

}  // namespace

void launch_mass_resid(const LevelDev& L, const double* x, const double* b, double* y, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_mass_resid, dim3(grid_for_bt(L.N)), dim3(256), 0, s, L, x, b, y);
}

void launch_block_jacobi(const LevelDev& L, int block, const double* x, const double* r, double* xo, double omega,
                         cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_block_jacobi, dim3(grid_for_bt(L.N)), dim3(256), 0, s, L, block, x, r, xo, omega);
}

void launch_add(double* y, const double* x, long long N, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_add, dim3(grid_for_bt(N)), dim3(256), 0, s, y, x, N);
}

}  // namespace sv
