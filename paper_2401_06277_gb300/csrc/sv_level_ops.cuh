// sv_level_ops.cuh -- per-vertex / per-element bodies of the operator, the
// residual and the grid transfers of one level (Section 2.2; Section 3,
// Algorithm 1), shared by the stand-alone kernels of sv_kernels.cu and the
// persistent coarse-level kernel (sv_vanka.cu), so both run the same arithmetic.
// Their pointer parameters carry no __restrict__: inside the persistent kernel the
// same buffers are written by one step and read by the next, so their loads must
// not take the read-only (non-coherent) path; the stand-alone kernels keep
// __restrict__ on their own parameters.
#pragma once

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace sv {
namespace ops {

__device__ __forceinline__ bool is_free(int I, int J, int nq) {
  return I > 0 && J > 0 && I < nq - 1 && J < nq - 1;
}

// ---------------------------------------------------------------------------
// Operator: y = A x (residual = 0) or y = b - A x (residual = 1).
// One thread per vertex (a, b): the four Q2 nodes (2a..2a+1) x (2b..2b+1) of
// both velocity components and the pressure row of (a, b).  Node parities
// are fixed per node, so every stencil coefficient is a compile-time constant.
// ---------------------------------------------------------------------------
// One vertex (a, bb): the 6 x 6 x neighbourhood of each component (Q2 nodes
// 2a-2..2a+3 x 2bb-2..2bb+3) and the 3 x 3 pressures around (a, bb) are read
// once into registers; the four velocity rows of the cell and the pressure row
// of the vertex are evaluated there with compile-time coefficients.  With MASK
// (vertices within two of the boundary) entries outside the grid or on
// Dirichlet nodes read as 0 (eliminated columns) and Dirichlet rows are the
// identity.
template <typename T, bool MASK>
__device__ __forceinline__ void apply_vertex_m(const LevelDev& L, const T* x,
                                             const T* b, T* y, int residual,
                                             int a, int bb) {
  const int nq = L.nq, np = L.np, n = L.n;
  const long long nv = L.nv;
  const int I0 = 2 * a, J0 = 2 * bb;
  const T cl = level_cl<T>(L), cb = level_cb<T>(L);
  const T* p = x + 2 * nv;
  T P[3][3];
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di) {
      const int pi = a + di - 1, pj = bb + dj - 1;
      const bool ok = !MASK || (pi >= 0 && pj >= 0 && pi <= n && pj <= n);
      P[dj][di] = ok ? p[static_cast<long long>(pj) * np + pi] : T(0);
    }
  T bu = T(0);
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T* xc = x + c * nv;
    T X[6][6];
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
      for (int q = 0; q < 6; ++q) {
        const int I = I0 - 2 + q, J = J0 - 2 + r;
        const bool ok = !MASK || is_free(I, J, nq);
        X[r][q] = ok ? xc[static_cast<long long>(J) * nq + I] : T(0);
      }
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ) {
#pragma unroll
      for (int PI = 0; PI < 2; ++PI) {
        const int I = I0 + PI, J = J0 + PJ;
        if (MASK && (I >= nq || J >= nq)) continue;
        const long long k = c * nv + static_cast<long long>(J) * nq + I;
        T v;
        if (MASK && !is_free(I, J, nq)) {
          v = xc[static_cast<long long>(J) * nq + I];   // Dirichlet row: identity
        } else {
          T sl = T(0), g = T(0);
#pragma unroll
          for (int dJ = -2; dJ <= 2; ++dJ)
#pragma unroll
            for (int dI = -2; dI <= 2; ++dI) {
              const T cf = T(k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ));
              if (cf != T(0)) sl = fma(cf, X[PJ + dJ + 2][PI + dI + 2], sl);
            }
#pragma unroll
          for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
              const T w = T(c == 0 ? ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj)
                                   : ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj));
              if (w != T(0)) g = fma(w, P[dj + 1][di + 1], g);
            }
          v = cl * sl + cb * g;
        }
        y[k] = residual ? b[k] - v : v;
      }
    }
    // pressure row of (a, bb): taps at Q2 nodes (2a + dI, 2bb + dJ)
#pragma unroll
    for (int dJ = -2; dJ <= 2; ++dJ)
#pragma unroll
      for (int dI = -2; dI <= 2; ++dI) {
        const T w = T(c == 0 ? crow(dI) * nrow(dJ) : nrow(dI) * crow(dJ));
        if (w != T(0)) bu = fma(w, X[dJ + 2][dI + 2], bu);
      }
  }
  const T ap = cb * bu;
  const long long k = 2 * nv + static_cast<long long>(bb) * np + a;
  y[k] = residual ? b[k] - ap : ap;
}

// y = A x or b - A x at vertex (a, bb): the masked variant within two of the boundary
template <typename T>
__device__ __forceinline__ void apply_vertex(const LevelDev& L, const T* x, const T* b,
                                             T* y, int residual, int a, int bb) {
  const int n = L.n;
  if (a >= 2 && a <= n - 2 && bb >= 2 && bb <= n - 2)
    apply_vertex_m<T, false>(L, x, b, y, residual, a, bb);
  else
    apply_vertex_m<T, true>(L, x, b, y, residual, a, bb);
}

// ---------------------------------------------------------------------------
// Restriction r_c = P^T r_f and prolongation x_f += P e_c (FE interpolation,
// Dirichlet rows of P (fine) and columns (coarse) zero).  In 1D a fine Q2
// node 2G coincides with coarse node G (weight 1); an odd fine node
// 4e+1 / 4e+3 inside coarse element e takes the coarse quadratic at t = 1/4 /
// 3/4: weights (3/8, 3/4, -1/8) / (-1/8, 3/4, 3/8) on coarse nodes 2e..2e+2.
// Q1: fine vertex 2g <- coarse g; 2g+1 <- (1/2, 1/2) on g, g+1.  The weights
// are compile-time constants of the element type; both passes are separable
// (x, then y) in registers.
// ---------------------------------------------------------------------------

// Per axis, fine Q2 nodes 4e..4e+3 of coarse element e take coarse nodes
// 2e..2e+2 with the weights PW[f][g] (rows f = 0..3); the transpose gives coarse
// nodes 2e, 2e+1 from fine nodes 4e-3..4e+3 with RW[g][k], k = F - (4e - 3).
// All weights are exact binary fractions.
__host__ __device__ constexpr double pw(int f, int g) {
  return f == 0 ? (g == 0 ? 1.0 : 0.0)
       : f == 1 ? (g == 0 ? 0.375 : g == 1 ? 0.75 : -0.125)
       : f == 2 ? (g == 1 ? 1.0 : 0.0)
                : (g == 0 ? -0.125 : g == 1 ? 0.75 : 0.375);
}
__host__ __device__ constexpr double rw(int g, int k) {
  // g = 0: fine 4e-3, 4e-1, 4e, 4e+1, 4e+3 -> k = 0, 2, 3, 4, 6 ; g = 1: fine 4e+1..4e+3 -> k = 4, 5, 6
  return g == 0 ? (k == 0 || k == 6 ? -0.125 : k == 2 || k == 4 ? 0.375 : k == 3 ? 1.0 : 0.0)
                : (k == 4 || k == 6 ? 0.75 : k == 5 ? 1.0 : 0.0);
}

// One thread per coarse element (ex, ey), ex, ey in 0..nc (the last one only
// reaches the far boundary nodes): coarse Q2 nodes (2ex + gx, 2ey + gy),
// g in {0, 1}, and coarse vertex (ex, ey).
template <typename T>
__device__ __forceinline__ void restrict_elem(const LevelDev& F, const LevelDev& C, const T* rf,
                                              T* rc, int ex, int ey) {
  const int fq = F.nq, cq = C.nq;
  const int F0x = 4 * ex - 3, F0y = 4 * ey - 3;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T* r = rf + c * F.nv;
    T H[7][2];
#pragma unroll
    for (int k2 = 0; k2 < 7; ++k2) {
      const int J = F0y + k2;
      T v[7];
#pragma unroll
      for (int k = 0; k < 7; ++k) {
        const int I = F0x + k;
        v[k] = (rw(0, k) != 0.0 || rw(1, k) != 0.0) && is_free(I, J, fq) ? r[static_cast<long long>(J) * fq + I]
                                                                        : T(0);
      }
#pragma unroll
      for (int g = 0; g < 2; ++g) {
        T acc = T(0);
#pragma unroll
        for (int k = 0; k < 7; ++k)
          if (rw(g, k) != 0.0) acc = fma(T(rw(g, k)), v[k], acc);
        H[k2][g] = acc;
      }
    }
#pragma unroll
    for (int gy = 0; gy < 2; ++gy) {
#pragma unroll
      for (int gx = 0; gx < 2; ++gx) {
        const int I = 2 * ex + gx, J = 2 * ey + gy;
        if (I >= cq || J >= cq) continue;
        T acc = T(0);
#pragma unroll
        for (int k2 = 0; k2 < 7; ++k2)
          if (rw(gy, k2) != 0.0) acc = fma(T(rw(gy, k2)), H[k2][gx], acc);
        rc[c * C.nv + static_cast<long long>(J) * cq + I] = is_free(I, J, cq) ? acc : T(0);
      }
    }
  }
  // Q1: coarse vertex (ex, ey) <- fine vertices 2e-1, 2e, 2e+1 per axis (1/2, 1, 1/2)
  const T* pf = rf + 2 * F.nv;
  T s = T(0);
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
    const int fj = 2 * ey + dj;
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const int fi = 2 * ex + di;
      if (fi < 0 || fj < 0 || fi >= F.np || fj >= F.np) continue;
      s = fma(T((di == 0 ? 1.0 : 0.5) * (dj == 0 ? 1.0 : 0.5)), pf[static_cast<long long>(fj) * F.np + fi], s);
    }
  }
  rc[2 * C.nv + static_cast<long long>(ey) * C.np + ex] = s;
}

// x_f += P e_c; one thread per coarse element (ex, ey), ex, ey in 0..nc: fine
// Q2 nodes (4ex + fx, 4ey + fy), f in 0..3, and fine vertices (2ex + fx, 2ey + fy),
// f in {0, 1}.  Coarse Dirichlet values read as 0; fine Dirichlet rows are untouched.
template <typename T>
__device__ __forceinline__ void prolong_elem(const LevelDev& F, const LevelDev& C, const T* ec,
                                             T* xf, int ex, int ey) {
  const int fq = F.nq, cq = C.nq;
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const T* e = ec + c * C.nv;
    T H[3][4];
#pragma unroll
    for (int gy = 0; gy < 3; ++gy) {
      const int J = 2 * ey + gy;
      T v[3];
#pragma unroll
      for (int gx = 0; gx < 3; ++gx) {
        const int I = 2 * ex + gx;
        v[gx] = is_free(I, J, cq) ? e[static_cast<long long>(J) * cq + I] : T(0);
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        T acc = T(0);
#pragma unroll
        for (int g = 0; g < 3; ++g)
          if (pw(f, g) != 0.0) acc = fma(T(pw(f, g)), v[g], acc);
        H[gy][f] = acc;
      }
    }
#pragma unroll
    for (int fy = 0; fy < 4; ++fy) {
#pragma unroll
      for (int fx = 0; fx < 4; ++fx) {
        const int I = 4 * ex + fx, J = 4 * ey + fy;
        if (!is_free(I, J, fq)) continue;
        T acc = T(0);
#pragma unroll
        for (int g = 0; g < 3; ++g)
          if (pw(fy, g) != 0.0) acc = fma(T(pw(fy, g)), H[g][fx], acc);
        xf[c * F.nv + static_cast<long long>(J) * fq + I] += acc;
      }
    }
  }
  // Q1: fine vertex 2e <- coarse e; 2e+1 <- (e + (e+1)) / 2, per axis
  const T* p = ec + 2 * C.nv;
  T P[2][2];
#pragma unroll
  for (int dj = 0; dj < 2; ++dj)
#pragma unroll
    for (int di = 0; di < 2; ++di) {
      const int i = ex + di, j = ey + dj;
      P[dj][di] = (i <= C.n && j <= C.n) ? p[static_cast<long long>(j) * C.np + i] : T(0);
    }
#pragma unroll
  for (int fy = 0; fy < 2; ++fy) {
#pragma unroll
    for (int fx = 0; fx < 2; ++fx) {
      const int I = 2 * ex + fx, J = 2 * ey + fy;
      if (I >= F.np || J >= F.np) continue;
      T v = P[0][0];
      if (fx == 1 && fy == 0) v = T(0.5) * (P[0][0] + P[0][1]);
      if (fx == 0 && fy == 1) v = T(0.5) * (P[0][0] + P[1][0]);
      if (fx == 1 && fy == 1) v = T(0.25) * ((P[0][0] + P[0][1]) + (P[1][0] + P[1][1]));
      xf[2 * F.nv + static_cast<long long>(J) * F.np + I] += v;
    }
  }
}

// e[row] = sum_k G[row][k] r[k] by one warp (lanes along the row, a fixed
// shuffle tree: deterministic); r converted to double on the fly
template <typename TR>
__device__ __forceinline__ double coarse_row(const double* G, int N0, const TR* r,
                                             int row, int lane) {
  const double* g = G + static_cast<long long>(row) * N0;
  double s = 0.0;
  for (int k = lane; k < N0; k += 32) s = fma(g[k], static_cast<double>(r[k]), s);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  return s;
}

}  // namespace ops
}  // namespace sv
