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
template <typename T, int PI, int PJ>
__device__ __forceinline__ T lap_g(const T* __restrict__ xs, int ld) {
  T s = T(0);
#pragma unroll
  for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
    for (int dI = -2; dI <= 2; ++dI) {
      const T c = T(k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ));
      if (c != T(0)) s = fma(c, xs[dJ * ld + dI], s);
    }
  }
  return s;
}

template <typename T, int PI, int PJ, int COMP>
__device__ __forceinline__ T btp_g(const T* __restrict__ pc, int ld) {
  T g = T(0);
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const T w = T(COMP == 0 ? ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj)
                              : ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj));
      if (w != T(0)) g = fma(w, pc[dj * ld + di], g);
    }
  }
  return g;
}

// generic masked evaluation of (A x) at velocity node (I, J), both components
template <typename T>
__device__ __forceinline__ void apply_vel_node(const LevelDev& L, const T* __restrict__ x, int I,
                                               int J, T& ax, T& ay) {
  const int nq = L.nq, np = L.np, n = L.n;
  const long long nv = L.nv;
  const long long k = static_cast<long long>(J) * nq + I;
  if (!is_free(I, J, nq)) {
    ax = x[k];
    ay = x[nv + k];
    return;
  }
  T sx = T(0), sy = T(0);
  for (int dJ = -2; dJ <= 2; ++dJ) {
    const int J2 = J + dJ;
    if (J2 <= 0 || J2 >= nq - 1) continue;
    const double mJ = m1(J, dJ), kJ = k1(J, dJ);
    for (int dI = -2; dI <= 2; ++dI) {
      const int I2 = I + dI;
      if (I2 <= 0 || I2 >= nq - 1) continue;
      const T c = T(k1(I, dI) * mJ + m1(I, dI) * kJ);
      if (c == T(0)) continue;
      const long long kk = static_cast<long long>(J2) * nq + I2;
      sx = fma(c, x[kk], sx);
      sy = fma(c, x[nv + kk], sy);
    }
  }
  const T* p = x + 2 * nv;
  T gx = T(0), gy = T(0);
  for (int j = J / 2 - 1; j <= J / 2 + 1; ++j) {
    if (j < 0 || j > n) continue;
    for (int i = I / 2 - 1; i <= I / 2 + 1; ++i) {
      if (i < 0 || i > n) continue;
      const T wx = T(ccol(I, i) * ncol(J, j)), wy = T(ncol(I, i) * ccol(J, j));
      const T pv = p[static_cast<long long>(j) * np + i];
      if (wx != T(0)) gx = fma(wx, pv, gx);
      if (wy != T(0)) gy = fma(wy, pv, gy);
    }
  }
  const T cl = T(L.cl), cb = T(L.cb);
  ax = cl * sx + cb * gx;
  ay = cl * sy + cb * gy;
}

template <typename T, int PI, int PJ>
__device__ __forceinline__ void apply_node(const LevelDev& L, const T* __restrict__ x,
                                           const T* __restrict__ b, T* __restrict__ y,
                                           int residual, bool fast, int a, int bb) {
  const int I = 2 * a + PI, J = 2 * bb + PJ;
  const int nq = L.nq;
  if (I >= nq || J >= nq) return;
  const long long nv = L.nv;
  const long long k = static_cast<long long>(J) * nq + I;
  T ax, ay;
  if (fast) {
    const T cl = T(L.cl), cb = T(L.cb);
    const T* pc = x + 2 * nv + static_cast<long long>(bb) * L.np + a;
    ax = cl * lap_g<T, PI, PJ>(x + k, nq) + cb * btp_g<T, PI, PJ, 0>(pc, L.np);
    ay = cl * lap_g<T, PI, PJ>(x + nv + k, nq) + cb * btp_g<T, PI, PJ, 1>(pc, L.np);
  } else {
    apply_vel_node<T>(L, x, I, J, ax, ay);
  }
  if (residual) {
    y[k] = b[k] - ax;
    y[nv + k] = b[nv + k] - ay;
  } else {
    y[k] = ax;
    y[nv + k] = ay;
  }
}

template <typename T>
__global__ void k_apply(LevelDev L, const T* __restrict__ x, const T* __restrict__ b,
                        T* __restrict__ y, int residual) {
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int bb = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = L.n, nq = L.nq, np = L.np;
  if (a > n || bb > n) return;
  const bool fast = a >= 2 && a <= n - 2 && bb >= 2 && bb <= n - 2;
  apply_node<T, 0, 0>(L, x, b, y, residual, fast, a, bb);
  apply_node<T, 1, 0>(L, x, b, y, residual, fast, a, bb);
  apply_node<T, 0, 1>(L, x, b, y, residual, fast, a, bb);
  apply_node<T, 1, 1>(L, x, b, y, residual, fast, a, bb);
  // pressure row of vertex (a, bb): (B u)
  const long long nv = L.nv;
  T s = T(0);
  if (fast) {
    const T* u0 = x + static_cast<long long>(2 * bb) * nq + 2 * a;
#pragma unroll
    for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
      for (int dI = -2; dI <= 2; ++dI) {
        const T cx = T(crow(dI) * nrow(dJ)), cy = T(nrow(dI) * crow(dJ));
        if (cx != T(0)) s = fma(cx, u0[dJ * nq + dI], s);
        if (cy != T(0)) s = fma(cy, u0[nv + dJ * nq + dI], s);
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
        const T cx = T(crow(dI) * nrow(dJ)), cy = T(nrow(dI) * crow(dJ));
        if (cx != T(0)) s = fma(cx, x[kk], s);
        if (cy != T(0)) s = fma(cy, x[nv + kk], s);
      }
    }
  }
  const T ap = T(L.cb) * s;
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
// Dirichlet rows of P (fine) and columns (coarse) zero).  In 1D a fine Q2
// node 2G coincides with coarse node G (weight 1); an odd fine node
// 4e+1 / 4e+3 inside coarse element e takes the coarse quadratic at t = 1/4 /
// 3/4: weights (3/8, 3/4, -1/8) / (-1/8, 3/4, 3/8) on coarse nodes 2e..2e+2.
// Q1: fine vertex 2g <- coarse g; 2g+1 <- (1/2, 1/2) on g, g+1.  All weights
// are computed in registers (no tables).
// ---------------------------------------------------------------------------

// coarse nodes and weights feeding fine Q2 node F on one axis; returns the count (1 or 3)
__device__ __forceinline__ int q2_interp(int F, int nc, int* G, double* w) {
  if ((F & 1) == 0) {
    G[0] = F >> 1;
    w[0] = 1.0;
    return 1;
  }
  int e = F >> 2;
  if (e > nc - 1) e = nc - 1;
  const bool first = (F - 4 * e) == 1;
  G[0] = 2 * e;
  G[1] = 2 * e + 1;
  G[2] = 2 * e + 2;
  w[0] = first ? 0.375 : -0.125;
  w[1] = 0.75;
  w[2] = first ? -0.125 : 0.375;
  return 3;
}

// fine Q2 nodes fed by coarse Q2 node G on one axis (the transpose); returns the count (1, 3 or 5)
__device__ __forceinline__ int q2_restrict(int G, int* F, double* w) {
  if (G & 1) {  // coarse element midpoint: fine nodes 2G-1, 2G, 2G+1
    F[0] = 2 * G - 1;
    F[1] = 2 * G;
    F[2] = 2 * G + 1;
    w[0] = 0.75;
    w[1] = 1.0;
    w[2] = 0.75;
    return 3;
  }
  F[0] = 2 * G - 3;  // coarse vertex: fine 2G-3, 2G-1, 2G, 2G+1, 2G+3
  F[1] = 2 * G - 1;
  F[2] = 2 * G;
  F[3] = 2 * G + 1;
  F[4] = 2 * G + 3;
  w[0] = -0.125;
  w[1] = 0.375;
  w[2] = 1.0;
  w[3] = 0.375;
  w[4] = -0.125;
  return 5;
}

template <typename T>
__global__ void k_restrict(LevelDev F, LevelDev C, const T* __restrict__ rf, T* __restrict__ rc) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I < C.nq && J < C.nq) {
    const long long k = static_cast<long long>(J) * C.nq + I;
    T sx = T(0), sy = T(0);
    if (is_free(I, J, C.nq)) {
      int FI[5], FJ[5];
      double wI[5], wJ[5];
      const int ni = q2_restrict(I, FI, wI), nj = q2_restrict(J, FJ, wJ);
      for (int b = 0; b < nj; ++b) {
        if (FJ[b] <= 0 || FJ[b] >= F.nq - 1) continue;
        for (int a = 0; a < ni; ++a) {
          if (FI[a] <= 0 || FI[a] >= F.nq - 1) continue;
          const long long kf = static_cast<long long>(FJ[b]) * F.nq + FI[a];
          const T w = T(wI[a] * wJ[b]);
          sx = fma(w, rf[kf], sx);
          sy = fma(w, rf[F.nv + kf], sy);
        }
      }
    }
    rc[k] = sx;
    rc[C.nv + k] = sy;
  }
  if (I < C.np && J < C.np) {
    T s = T(0);
    for (int dj = -1; dj <= 1; ++dj) {
      const int fj = 2 * J + dj;
      if (fj < 0 || fj >= F.np) continue;
      for (int di = -1; di <= 1; ++di) {
        const int fi = 2 * I + di;
        if (fi < 0 || fi >= F.np) continue;
        const T w = T((di == 0 ? 1.0 : 0.5) * (dj == 0 ? 1.0 : 0.5));
        s = fma(w, rf[2 * F.nv + static_cast<long long>(fj) * F.np + fi], s);
      }
    }
    rc[2 * C.nv + static_cast<long long>(J) * C.np + I] = s;
  }
}

template <typename T>
__global__ void k_prolong_add(LevelDev F, LevelDev C, const T* __restrict__ ec, T* __restrict__ xf) {
  const int I = blockIdx.x * blockDim.x + threadIdx.x;
  const int J = blockIdx.y * blockDim.y + threadIdx.y;
  if (I < F.nq && J < F.nq && is_free(I, J, F.nq)) {
    int GI[3], GJ[3];
    double wI[3], wJ[3];
    const int ni = q2_interp(I, C.n, GI, wI), nj = q2_interp(J, C.n, GJ, wJ);
    T sx = T(0), sy = T(0);
    for (int b = 0; b < nj; ++b) {
      if (GJ[b] <= 0 || GJ[b] >= C.nq - 1) continue;  // coarse Dirichlet row
      for (int a = 0; a < ni; ++a) {
        if (GI[a] <= 0 || GI[a] >= C.nq - 1) continue;
        const long long kc = static_cast<long long>(GJ[b]) * C.nq + GI[a];
        const T w = T(wI[a] * wJ[b]);
        sx = fma(w, ec[kc], sx);
        sy = fma(w, ec[C.nv + kc], sy);
      }
    }
    const long long k = static_cast<long long>(J) * F.nq + I;
    xf[k] += sx;
    xf[F.nv + k] += sy;
  }
  if (I < F.np && J < F.np) {
    // fine vertex (I, J) <- coarse vertices (I/2 .. (I+1)/2, J/2 .. (J+1)/2), weights 1 or 1/2 per axis
    const int i0 = I >> 1, i1 = (I + 1) >> 1, j0 = J >> 1, j1 = (J + 1) >> 1;
    const T wi = (I & 1) ? T(0.5) : T(1.0), wj = (J & 1) ? T(0.5) : T(1.0);
    const T* p = ec + 2 * C.nv;
    T s = wi * wj * p[static_cast<long long>(j0) * C.np + i0];
    if (I & 1) s = fma(wi * wj, p[static_cast<long long>(j0) * C.np + i1], s);
    if (J & 1) s = fma(wi * wj, p[static_cast<long long>(j1) * C.np + i0], s);
    if ((I & 1) && (J & 1)) s = fma(wi * wj, p[static_cast<long long>(j1) * C.np + i1], s);
    xf[2 * F.nv + static_cast<long long>(J) * F.np + I] += s;
  }
}

template <typename TI, typename TO>
__global__ void k_convert(const TI* __restrict__ in, TO* __restrict__ out, long long N) {
  for (long long i = blockIdx.x * static_cast<long long>(blockDim.x) + threadIdx.x; i < N;
       i += static_cast<long long>(gridDim.x) * blockDim.x)
    out[i] = static_cast<TO>(in[i]);
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

template <typename T>
void launch_apply(const LevelDev& L, const T* x, const T* b, T* y, int residual, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_apply<T><<<grid2(L.np, L.np, blk), blk, 0, s>>>(L, x, b, y, residual);
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

template <typename T>
void launch_restrict(const LevelDev& F, const LevelDev& C, const T* rf, T* rc, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_restrict<T><<<grid2(C.nq, C.nq, blk), blk, 0, s>>>(F, C, rf, rc);
}

template <typename T>
void launch_prolong_add(const LevelDev& F, const LevelDev& C, const T* ec, T* xf, cudaStream_t s) {
  count_launches(1);
  dim3 blk(32, 8);
  k_prolong_add<T><<<grid2(F.nq, F.nq, blk), blk, 0, s>>>(F, C, ec, xf);
}

template <typename TI, typename TO>
void launch_convert(const TI* in, TO* out, long long N, cudaStream_t s) {
  count_launches(1);
  long long blocks = (N + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_convert<TI, TO><<<static_cast<int>(blocks < 1 ? 1 : blocks), 256, 0, s>>>(in, out, N);
}

void launch_coarse(const double* G, int N0, const double* r, double* e, cudaStream_t s) {
  count_launches(1);
  k_coarse<<<1, 256, N0 * sizeof(double), s>>>(G, N0, r, e);
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
