// sv_kernels_f64.cu -- FP64 kernels of the hot path on sm_103a:
//   matrix-free Stokes operator / residual   (Section 2.2, Algorithm 1 residual)
//   right-hand side assembly and its transpose (Section 2.2)
//   fused additive Vanka sweep               (Section 3.2, Algorithm 3; Section 6.3)
//   FE restriction P^T and prolongation P    (Section 3, Algorithm 1)
//   dense coarse solve                       (Algorithm 1, level 0)
#include <cuda_runtime.h>

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace sv {
namespace {

__device__ __forceinline__ bool is_free(int I, int J, int nq) {
  return I > 0 && J > 0 && I < nq - 1 && J < nq - 1;
}

// ---------------------------------------------------------------------------
// Operator: y = A x (residual = 0) or y = b - A x (residual = 1).
// One thread per vertex (a, b): the four Q2 nodes (2a..2a+1) x (2b..2b+1) of
// both velocity components and the pressure row of (a, b).  Away from the
// boundary (2 <= a, b <= n-2) every tap is in the free interior and the
// stencil coefficients are compile-time constants (node parities are fixed
// per node); near the boundary a masked generic path drops Dirichlet columns.
// ---------------------------------------------------------------------------
template <int PI, int PJ>
__device__ __forceinline__ double lap_g(const double* __restrict__ xs, int ld) {
  double s = 0.0;
#pragma unroll
  for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
    for (int dI = -2; dI <= 2; ++dI) {
      const double c = k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ);
      if (c != 0.0) s = fma(c, xs[dJ * ld + dI], s);
    }
  }
  return s;
}

template <int PI, int PJ, int COMP>
__device__ __forceinline__ double btp_g(const double* __restrict__ pc, int ld) {
  double g = 0.0;
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const double w = COMP == 0 ? ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj)
                                 : ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj);
      if (w != 0.0) g = fma(w, pc[dj * ld + di], g);
    }
  }
  return g;
}

// generic masked evaluation of (A x) at velocity node (I, J), both components
__device__ __forceinline__ void apply_vel_node(const LevelDev& L, const double* __restrict__ x, int I,
                                               int J, double& ax, double& ay) {
  const int nq = L.nq, np = L.np, n = L.n;
  const long long nv = L.nv;
  const long long k = static_cast<long long>(J) * nq + I;
  if (!is_free(I, J, nq)) {
    ax = x[k];
    ay = x[nv + k];
    return;
  }
  double sx = 0.0, sy = 0.0;
  for (int dJ = -2; dJ <= 2; ++dJ) {
    const int J2 = J + dJ;
    if (J2 <= 0 || J2 >= nq - 1) continue;
    const double mJ = m1(J, dJ), kJ = k1(J, dJ);
    for (int dI = -2; dI <= 2; ++dI) {
      const int I2 = I + dI;
      if (I2 <= 0 || I2 >= nq - 1) continue;
      const double c = k1(I, dI) * mJ + m1(I, dI) * kJ;
      if (c == 0.0) continue;
      const long long kk = static_cast<long long>(J2) * nq + I2;
      sx = fma(c, x[kk], sx);
      sy = fma(c, x[nv + kk], sy);
    }
  }
  const double* p = x + 2 * nv;
  double gx = 0.0, gy = 0.0;
  for (int j = J / 2 - 1; j <= J / 2 + 1; ++j) {
    if (j < 0 || j > n) continue;
    for (int i = I / 2 - 1; i <= I / 2 + 1; ++i) {
      if (i < 0 || i > n) continue;
      const double wx = ccol(I, i) * ncol(J, j), wy = ncol(I, i) * ccol(J, j);
      const double pv = p[static_cast<long long>(j) * np + i];
      if (wx != 0.0) gx = fma(wx, pv, gx);
      if (wy != 0.0) gy = fma(wy, pv, gy);
    }
  }
  const double cl = L.nu / 90.0, cb = -L.h / 18.0;
  ax = cl * sx + cb * gx;
  ay = cl * sy + cb * gy;
}

template <int PI, int PJ>
__device__ __forceinline__ void apply_node(const LevelDev& L, const double* __restrict__ x,
                                           const double* __restrict__ b, double* __restrict__ y,
                                           int residual, bool fast, int a, int bb) {
  const int I = 2 * a + PI, J = 2 * bb + PJ;
  const int nq = L.nq;
  if (I >= nq || J >= nq) return;
  const long long nv = L.nv;
  const long long k = static_cast<long long>(J) * nq + I;
  double ax, ay;
  if (fast) {
    const double cl = L.nu / 90.0, cb = -L.h / 18.0;
    const double* pc = x + 2 * nv + static_cast<long long>(bb) * L.np + a;
    ax = cl * lap_g<PI, PJ>(x + k, nq) + cb * btp_g<PI, PJ, 0>(pc, L.np);
    ay = cl * lap_g<PI, PJ>(x + nv + k, nq) + cb * btp_g<PI, PJ, 1>(pc, L.np);
  } else {
    apply_vel_node(L, x, I, J, ax, ay);
  }
  if (residual) {
    y[k] = b[k] - ax;
    y[nv + k] = b[nv + k] - ay;
  } else {
    y[k] = ax;
    y[nv + k] = ay;
  }
}

__global__ void k_apply(LevelDev L, const double* __restrict__ x, const double* __restrict__ b,
                        double* __restrict__ y, int residual) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int bb = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = L.n, nq = L.nq, np = L.np;
  if (a > n || bb > n) return;
  const bool fast = a >= 2 && a <= n - 2 && bb >= 2 && bb <= n - 2;
  apply_node<0, 0>(L, x, b, y, residual, fast, a, bb);
  apply_node<1, 0>(L, x, b, y, residual, fast, a, bb);
  apply_node<0, 1>(L, x, b, y, residual, fast, a, bb);
  apply_node<1, 1>(L, x, b, y, residual, fast, a, bb);
  // pressure row of vertex (a, bb): (B u)
  const long long nv = L.nv;
  double s = 0.0;
  if (fast) {
    const double* u0 = x + static_cast<long long>(2 * bb) * nq + 2 * a;
#pragma unroll
    for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
      for (int dI = -2; dI <= 2; ++dI) {
        const double cx = crow(dI) * nrow(dJ), cy = nrow(dI) * crow(dJ);
        if (cx != 0.0) s = fma(cx, u0[dJ * nq + dI], s);
        if (cy != 0.0) s = fma(cy, u0[nv + dJ * nq + dI], s);
      }
    }
  } else {
#pragma unroll
    for (int dJ = -2; dJ <= 2; ++dJ) {
      const int J = 2 * bb + dJ;
      if (J <= 0 || J >= nq - 1) continue;
#pragma unroll
      for (int dI = -2; dI <= 2; ++dI) {
        const int I = 2 * a + dI;
        if (I <= 0 || I >= nq - 1) continue;
        const long long kk = static_cast<long long>(J) * nq + I;
        const double cx = crow(dI) * nrow(dJ), cy = nrow(dI) * crow(dJ);
        if (cx != 0.0) s = fma(cx, x[kk], s);
        if (cy != 0.0) s = fma(cy, x[nv + kk], s);
      }
    }
  }
  const double ap = -L.h / 18.0 * s;
  const long long k = 2 * nv + static_cast<long long>(bb) * np + a;
  y[k] = residual ? b[k] - ap : ap;
}

// ---------------------------------------------------------------------------
// Right-hand side b = [M f - L_{.,D} u_D ; u_D on D ; -B_{.,D} u_D].
// ---------------------------------------------------------------------------
__global__ void k_rhs_vel(LevelDev L, const double* __restrict__ f, const double* __restrict__ ud,
                          double* __restrict__ b) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  const int nq = L.nq;
  if (I >= nq || J >= nq) return;
  const long long nv = L.nv;
  const long long k = static_cast<long long>(J) * nq + I;
  if (!is_free(I, J, nq)) {
    b[k] = ud[k];
    b[nv + k] = ud[nv + k];
    return;
  }
  double mx = 0.0, my = 0.0, lx = 0.0, ly = 0.0;
  for (int dJ = -2; dJ <= 2; ++dJ) {
    const int J2 = J + dJ;
    if (J2 < 0 || J2 >= nq) continue;
    for (int dI = -2; dI <= 2; ++dI) {
      const int I2 = I + dI;
      if (I2 < 0 || I2 >= nq) continue;
      const long long kk = static_cast<long long>(J2) * nq + I2;
      const double mm = m1(I, dI) * m1(J, dJ);
      mx = fma(mm, f[kk], mx);
      my = fma(mm, f[nv + kk], my);
      if (!is_free(I2, J2, nq)) {
        const double c = k1(I, dI) * m1(J, dJ) + m1(I, dI) * k1(J, dJ);
        lx = fma(c, ud[kk], lx);
        ly = fma(c, ud[nv + kk], ly);
      }
    }
  }
  const double cm = (L.h / 30.0) * (L.h / 30.0), cl = L.nu / 90.0;
  b[k] = cm * mx - cl * lx;
  b[nv + k] = cm * my - cl * ly;
}

__global__ void k_rhs_p(LevelDev L, const double* __restrict__ ud, double* __restrict__ b) {
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

// ---------------------------------------------------------------------------
// Restriction r_c = P^T r_f and prolongation x_f += P e_c (FE interpolation,
// Dirichlet rows of P (fine) and columns (coarse) zero).
// 1D Q2 weights: coarse node C even: fine 2C + {-3:-1/8, -1:3/8, 0:1, 1:3/8, 3:-1/8};
// C odd: fine 2C + {-1:3/4, 0:1, 1:3/4}.  Q1: fine 2c + {-1:1/2, 0:1, 1:1/2}.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double rq2(int C, int off) {
  if (C & 1) return off == 0 ? 1.0 : ((off == 1 || off == -1) ? 0.75 : 0.0);
  switch (off) {
    case 0: return 1.0;
    case 1: case -1: return 0.375;
    case 3: case -3: return -0.125;
    default: return 0.0;
  }
}
__device__ __forceinline__ double rq1(int off) {
  return off == 0 ? 1.0 : ((off == 1 || off == -1) ? 0.5 : 0.0);
}

__global__ void k_restrict(LevelDev F, LevelDev C, const double* __restrict__ rf,
                           double* __restrict__ rc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  // velocity part over the coarse Q2 grid, pressure over the coarse vertices
  if (I < C.nq && J < C.nq) {
    const long long k = static_cast<long long>(J) * C.nq + I;
    double sx = 0.0, sy = 0.0;
    if (is_free(I, J, C.nq)) {
      for (int dJ = -3; dJ <= 3; ++dJ) {
        const double wJ = rq2(J, dJ);
        const int FJ = 2 * J + dJ;
        if (wJ == 0.0 || !(FJ > 0 && FJ < F.nq - 1)) continue;
        for (int dI = -3; dI <= 3; ++dI) {
          const double wI = rq2(I, dI);
          const int FI = 2 * I + dI;
          if (wI == 0.0 || !(FI > 0 && FI < F.nq - 1)) continue;
          const long long kf = static_cast<long long>(FJ) * F.nq + FI;
          sx = fma(wI * wJ, rf[kf], sx);
          sy = fma(wI * wJ, rf[F.nv + kf], sy);
        }
      }
    }
    rc[k] = sx;
    rc[C.nv + k] = sy;
  }
  if (I < C.np && J < C.np) {
    double s = 0.0;
    for (int dj = -1; dj <= 1; ++dj) {
      const int fj = 2 * J + dj;
      if (fj < 0 || fj >= F.np) continue;
      for (int di = -1; di <= 1; ++di) {
        const int fi = 2 * I + di;
        if (fi < 0 || fi >= F.np) continue;
        s = fma(rq1(di) * rq1(dj), rf[2 * F.nv + static_cast<long long>(fj) * F.np + fi], s);
      }
    }
    rc[2 * C.nv + static_cast<long long>(J) * C.np + I] = s;
  }
}

// weights of the coarse element's local nodes at fine local position k/4 (Q2) or k/2 (Q1)
__device__ __forceinline__ double pq2(int k, int a) {
  // rows k = 0..4 (t = k/4), columns a = 0..2
  const double W[5][3] = {{1.0, 0.0, 0.0},
                          {0.375, 0.75, -0.125},
                          {0.0, 1.0, 0.0},
                          {-0.125, 0.75, 0.375},
                          {0.0, 0.0, 1.0}};
  return W[k][a];
}

__global__ void k_prolong_add(LevelDev F, LevelDev C, const double* __restrict__ ec,
                              double* __restrict__ xf) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I < F.nq && J < F.nq && is_free(I, J, F.nq)) {
    const int ex = min(I / 4, C.n - 1), ey = min(J / 4, C.n - 1);
    const int kx = I - 4 * ex, ky = J - 4 * ey;
    double sx = 0.0, sy = 0.0;
    for (int b = 0; b < 3; ++b) {
      const double wy = pq2(ky, b);
      const int CJ = 2 * ey + b;
      if (wy == 0.0 || CJ <= 0 || CJ >= C.nq - 1) continue;  // coarse Dirichlet row
      for (int a = 0; a < 3; ++a) {
        const double wx = pq2(kx, a);
        const int CI = 2 * ex + a;
        if (wx == 0.0 || !is_free(CI, CJ, C.nq)) continue;
        const long long kc = static_cast<long long>(CJ) * C.nq + CI;
        sx = fma(wx * wy, ec[kc], sx);
        sy = fma(wx * wy, ec[C.nv + kc], sy);
      }
    }
    const long long k = static_cast<long long>(J) * F.nq + I;
    xf[k] += sx;
    xf[F.nv + k] += sy;
  }
  if (I < F.np && J < F.np) {
    const int ex = min(I / 2, C.n - 1), ey = min(J / 2, C.n - 1);
    const int kx = I - 2 * ex, ky = J - 2 * ey;
    double s = 0.0;
    for (int b = 0; b < 2; ++b) {
      const double wy = (b == 0) ? (1.0 - 0.5 * ky) : 0.5 * ky;
      if (wy == 0.0) continue;
      for (int a = 0; a < 2; ++a) {
        const double wx = (a == 0) ? (1.0 - 0.5 * kx) : 0.5 * kx;
        if (wx == 0.0) continue;
        s = fma(wx * wy, ec[2 * C.nv + static_cast<long long>(ey + b) * C.np + (ex + a)], s);
      }
    }
    xf[2 * F.nv + static_cast<long long>(J) * F.np + I] += s;
  }
}

// e = G r, G dense N0 x N0 (one CTA)
__global__ void k_coarse(const double* __restrict__ G, int N0, const double* __restrict__ r,
                         double* __restrict__ e) {
  extern __shared__ double sr_[];
  for (int k = threadIdx.x; k < N0; k += blockDim.x) sr_[k] = r[k];
  __syncthreads();
  for (int row = threadIdx.x; row < N0; row += blockDim.x) {
    double s = 0.0;
    const double* g = G + static_cast<long long>(row) * N0;
    for (int k = 0; k < N0; ++k) s = fma(g[k], sr_[k], s);
    e[row] = s;
  }
}

dim3 grid2(int nx, int ny, dim3 blk) {
  return dim3((nx + blk.x - 1) / blk.x, (ny + blk.y - 1) / blk.y);
}

}  // namespace

void launch_apply(const LevelDev& L, const double* x, const double* b, double* y, int residual,
                  cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_apply<<<grid2(L.np, L.np, blk), blk, 0, s>>>(L, x, b, y, residual);
}

void launch_rhs(const LevelDev& L, const double* f, const double* ud, double* b, cudaStream_t s) {
  count_launches(2);
  dim3 blk(32, 8);
  k_rhs_vel<<<grid2(L.nq, L.nq, blk), blk, 0, s>>>(L, f, ud, b);
  k_rhs_p<<<grid2(L.np, L.np, blk), blk, 0, s>>>(L, ud, b);
}

void launch_rhs_transpose(const LevelDev& L, const double* lam, double* g, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_rhs_transpose<<<grid2(L.nq, L.nq, blk), blk, 0, s>>>(L, lam, g);
}

void launch_restrict(const LevelDev& F, const LevelDev& C, const double* rf, double* rc,
                     cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_restrict<<<grid2(C.nq, C.nq, blk), blk, 0, s>>>(F, C, rf, rc);
}

void launch_prolong_add(const LevelDev& F, const LevelDev& C, const double* ec, double* xf,
                        cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_prolong_add<<<grid2(F.nq, F.nq, blk), blk, 0, s>>>(F, C, ec, xf);
}

void launch_coarse(const double* G, int N0, const double* r, double* e, cudaStream_t s) {
  count_launches(1);
  k_coarse<<<1, 256, N0 * sizeof(double), s>>>(G, N0, r, e);
}

}  // namespace sv
