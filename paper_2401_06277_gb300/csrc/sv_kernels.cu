// sv_kernels.cu -- stencil kernels of the hot path on sm_103a, templated on
// the element type (double for the FP64 form and for FGMRES, float inside the
// mixed-precision preconditioner):
//   matrix-free Stokes operator / residual   (Section 2.2, Algorithm 1 residual)
//   FE restriction P^T and prolongation P    (Section 3, Algorithm 1)
//   precision conversions
// and, in FP64 only: right-hand side assembly and its transpose (Section 2.2)
// and the dense coarse solve (Algorithm 1, level 0).
#include <cuda_runtime.h>

#include "sv_internal.h"
#include "sv_level_ops.cuh"
#include "sv_stencil.cuh"

namespace sv {
namespace {

using ops::is_free;

template <typename T>
__global__ void k_apply(LevelDev L, const T* __restrict__ x, const T* __restrict__ b,
                        T* __restrict__ y, int residual) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int bb = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > L.n || bb > L.n) return;
  ops::apply_vertex<T>(L, x, b, y, residual, a, bb);
}

// ---------------------------------------------------------------------------
// Right-hand side b = [M f - L_{.,D} u_D ; u_D on D ; -B_{.,D} u_D].
// ---------------------------------------------------------------------------
// One vertex (a, bb): the four Q2 nodes (2a + PI, 2bb + PJ) of both components.
// b = (h/30)^2 (m (x) m) f on free rows, minus nu/90 (k (x) m + m (x) k) u_D over
// the Dirichlet columns (MASK: vertices within two of the boundary only), and
// b = u_D on Dirichlet rows.  The 6 x 6 f (and u_D) neighbourhood of each
// component is read once; coefficients are compile-time constants.
template <bool MASK>
__device__ __forceinline__ void rhs_vertex(const LevelDev& L, const double* __restrict__ f,
                                           const double* __restrict__ ud, double* __restrict__ b, int a,
                                           int bb) {
  const int nq = L.nq;
  const long long nv = L.nv;
  const int I0 = 2 * a, J0 = 2 * bb;
  const double cm = (L.h / 30.0) * (L.h / 30.0), cl = L.nu / 90.0;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    double F[6][6], U[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int I = I0 - 2 + q, J = J0 - 2 + r;
        const bool in = !MASK || (I >= 0 && J >= 0 && I < nq && J < nq);
        const long long k = c * nv + static_cast<long long>(J) * nq + I;
        F[r][q] = in ? f[k] : 0.0;
        U[r][q] = (MASK && in && !is_free(I, J, nq)) ? ud[k] : 0.0;
      }
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ) {
#pragma unroll
      for (int PI = 0; PI < 2; ++PI) {
        const int I = I0 + PI, J = J0 + PJ;
        if (MASK && (I >= nq || J >= nq)) continue;
        const long long k = c * nv + static_cast<long long>(J) * nq + I;
        if (MASK && !is_free(I, J, nq)) {
          b[k] = ud[k];
          continue;
        }
        double sm = 0.0, sl = 0.0;
#pragma unroll
        for (int dJ = -2; dJ <= 2; ++dJ)
#pragma unroll
          for (int dI = -2; dI <= 2; ++dI) {
            const double mm = m1(PI, dI) * m1(PJ, dJ);
            if (mm != 0.0) sm = fma(mm, F[PJ + dJ + 2][PI + dI + 2], sm);
            if (MASK) {
              const double cf = k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ);
              if (cf != 0.0) sl = fma(cf, U[PJ + dJ + 2][PI + dI + 2], sl);
            }
          }
        b[k] = cm * sm - cl * sl;
      }
    }
  }
}

__global__ void k_rhs_vel(LevelDev L, const double* __restrict__ f, const double* __restrict__ ud,
                          double* __restrict__ b) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int bb = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = L.n;
  if (a > n || bb > n) return;
  if (a >= 2 && a <= n - 2 && bb >= 2 && bb <= n - 2)
    rhs_vertex<false>(L, f, ud, b, a, bb);
  else
    rhs_vertex<true>(L, f, ud, b, a, bb);
}

__global__ void k_rhs_p(LevelDev L, const double* __restrict__ ud, double* __restrict__ b) {
  pdl_begin();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  const int nq = L.nq, np = L.np, n = L.n;
  if (i >= np || j >= np) return;
  const long long nv = L.nv;
  // -B_{.,D} u_D with B = -(C (x) N) h for u_x, -(N (x) C) h for u_y
  double s = 0.0;
  for (int J = 2 * j - 2; J <= 2 * j + 2; ++J) {
    if (J < 0 || J >= nq) continue;
    for (int I = 2 * i - 2; I <= 2 * i + 2; ++I) {
      if (I < 0 || I >= nq || is_free(I, J, nq)) continue;
      const long long kk = static_cast<long long>(J) * nq + I;
      s += c1_full(i, I, n) * n1_full(j, J, n) * ud[kk];
      s += n1_full(i, I, n) * c1_full(j, J, n) * ud[nv + kk];
    }
  }
  b[2 * nv + static_cast<long long>(j) * np + i] = L.h * s;
}

// grad_f = R^T lambda: sum over free velocity rows k of (M)_{k,(I,J)} lambda_k.
__global__ void k_rhs_transpose(LevelDev L, const double* __restrict__ lam, double* __restrict__ g) {
  pdl_begin();
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int nq = L.nq;
  if (I >= nq || J >= nq) return;
  const long long nv = L.nv;
  double sx = 0.0, sy = 0.0;
  for (int dJ = -2; dJ <= 2; ++dJ) {
    const int J2 = J + dJ;
    for (int dI = -2; dI <= 2; ++dI) {
      const int I2 = I + dI;
      if (!is_free(I2, J2, nq)) continue;
      // M is symmetric: M_{(I2,J2),(I,J)} = row of (I2,J2) at offset (-dI, -dJ)
      const double mm = m1(I2, -dI) * m1(J2, -dJ);
      const long long kk = static_cast<long long>(J2) * nq + I2;
      sx = fma(mm, lam[kk], sx);
      sy = fma(mm, lam[nv + kk], sy);
    }
  }
  const double cm = (L.h / 30.0) * (L.h / 30.0);
  const long long k = static_cast<long long>(J) * nq + I;
  g[k] = cm * sx;
  g[nv + k] = cm * sy;
}

// Restriction r_c = P^T r_f and prolongation x_f += P e_c (sv_level_ops.cuh):
// one thread per coarse element (ex, ey), ex, ey in 0..nc.
template <typename T>
__global__ void k_restrict(LevelDev F, LevelDev C, const T* __restrict__ rf, T* __restrict__ rc) {
  pdl_begin();
  const int ex = blockIdx.x * blockDim.x + threadIdx.x;
  const int ey = blockIdx.y * blockDim.y + threadIdx.y;
  if (ex > C.n || ey > C.n) return;
  ops::restrict_elem<T>(F, C, rf, rc, ex, ey);
}

template <typename T>
__global__ void k_prolong_add(LevelDev F, LevelDev C, const T* __restrict__ ec, T* __restrict__ xf) {
  pdl_begin();
  const int ex = blockIdx.x * blockDim.x + threadIdx.x;
  const int ey = blockIdx.y * blockDim.y + threadIdx.y;
  if (ex > C.n || ey > C.n) return;
  ops::prolong_elem<T>(F, C, ec, xf, ex, ey);
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, long long N) {
  pdl_begin();
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = static_cast<TO>(in[i]);
}

// e = G r, G dense N0 x N0: one warp per row, lanes along the row (coalesced),
// summed by a fixed shuffle tree (deterministic)
__global__ void k_coarse(const double* __restrict__ G, int N0, const double* __restrict__ r,
                         double* __restrict__ e) {
  pdl_begin();
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (row >= N0) return;
  const double s = ops::coarse_row<double>(G, N0, r, row, lane);
  if (lane == 0) e[row] = s;
}

dim3 grid2(int nx, int ny, dim3 blk) {
  return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y);
}

}  // namespace

template <typename T>
void launch_apply(const LevelDev& L, const T* x, const T* b, T* y, int residual, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  launch_pdl(k_apply<T>, dim3(grid2(L.np, L.np, blk)), dim3(blk), 0, s, L, x, b, y, residual);
}

void launch_rhs(const LevelDev& L, const double* f, const double* ud, double* b, cudaStream_t s) {
  count_launches(2);
  dim3 blk(32, 8);
  launch_pdl(k_rhs_vel, dim3(grid2(L.np, L.np, blk)), dim3(blk), 0, s, L, f, ud, b);
  launch_pdl(k_rhs_p, dim3(grid2(L.np, L.np, blk)), dim3(blk), 0, s, L, ud, b);
}

void launch_rhs_transpose(const LevelDev& L, const double* lam, double* g, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  launch_pdl(k_rhs_transpose, dim3(grid2(L.nq, L.nq, blk)), dim3(blk), 0, s, L, lam, g);
}

template <typename T>
void launch_restrict(const LevelDev& F, const LevelDev& C, const T* rf, T* rc, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  launch_pdl(k_restrict<T>, dim3(grid2(C.n + 1, C.n + 1, blk)), dim3(blk), 0, s, F, C, rf, rc);
}

template <typename T>
void launch_prolong_add(const LevelDev& F, const LevelDev& C, const T* ec, T* xf, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  launch_pdl(k_prolong_add<T>, dim3(grid2(C.n + 1, C.n + 1, blk)), dim3(blk), 0, s, F, C, ec, xf);
}

template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, long long N, cudaStream_t s) {
  count_launches(1);
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  launch_pdl(k_convert<TI, TO>, dim3(static_cast<int>(blocks)), dim3(256), 0, s, in, out, N);
}

void launch_coarse(const double* G, int N0, const double* r, double* e, cudaStream_t s) {
  count_launches(1);
  launch_pdl(k_coarse, dim3((N0 + 7) / 8), dim3(256), 0, s, G, N0, r, e);
}

template void launch_apply<double>(const LevelDev&, const double*, const double*, double*, int, cudaStream_t);
template void launch_apply<float>(const LevelDev&, const float*, const float*, float*, int, cudaStream_t);
template void launch_restrict<double>(const LevelDev&, const LevelDev&, const double*, double*, cudaStream_t);
template void launch_restrict<float>(const LevelDev&, const LevelDev&, const float*, float*, cudaStream_t);
template void launch_prolong_add<double>(const LevelDev&, const LevelDev&, const double*, double*, cudaStream_t);
template void launch_prolong_add<float>(const LevelDev&, const LevelDev&, const float*, float*, cudaStream_t);
template void launch_convert<double, float>(const double*, float*, long long, cudaStream_t);
template void launch_convert<float, double>(const float*, double*, long long, cudaStream_t);

}  // namespace sv
