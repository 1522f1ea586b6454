// sv_vanka_common.cuh -- device pieces shared by the SIMT and the tensor-core
// Vanka sweep kernels: tile geometry, the residual of one 2x2 cell of Q2
// nodes with compile-time stencil coefficients, and the Vanka weights.
#pragma once

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace sv {
namespace vk {

__device__ __forceinline__ bool vfree(int I, int J, int nq) {
  return I > 0 && J > 0 && I < nq - 1 && J < nq - 1;
}

template <int TX, int TY>
struct VT {
  static constexpr int XW = 2 * TX + 12, XH = 2 * TY + 12;  // x, Q2 nodes, origin 2 i0 - 6
  static constexpr int PW = TX + 6, PH = TY + 6;            // x, vertices,  origin i0 - 3
  static constexpr int CW = TX + 4, CH = TY + 4;            // residual cells, origin 2 i0 - 4
  static constexpr int RW = 2 * CW, RH = 2 * CH;            // residual, Q2 nodes
  static constexpr int QW = TX + 2, QH = TY + 2;            // patches, origin i0 - 1
  static constexpr int NPATCH = QW * QH;
  static constexpr int SX = 2 * XW * XH, SP = PW * PH, SR = 2 * RW * RH, SRP = NPATCH;
  static constexpr int SD = NPATCH * 51;
  static constexpr int TOTAL = SX + SP + SR + SRP + SD;
};

// sum of nu (K (x) M + M (x) K) x / (nu/90) over the stencil of a node with
// parities (PI, PJ); xs points at the node in the x window.
template <typename T, int PI, int PJ, int XW>
__device__ __forceinline__ T lap(const T* xs) {
  T s = T(0);
#pragma unroll
  for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
    for (int dI = -2; dI <= 2; ++dI) {
      const T c = T(k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ));
      if (c != T(0)) s = fma(c, xs[dJ * XW + dI], s);
    }
  }
  return s;
}

// (B^T p) / (-h/18) for velocity component COMP at a node with parities
// (PI, PJ) of the cell whose vertex is (a, b); pc points at p(a, b).
template <typename T, int PI, int PJ, int COMP, int PW>
__device__ __forceinline__ T btp(const T* pc) {
  T g = T(0);
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const T w = T(COMP == 0 ? ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj)
                              : ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj));
      if (w != T(0)) g = fma(w, pc[dj * PW + di], g);
    }
  }
  return g;
}

// G: window geometry (XW, XH, PW, RW, RH), e.g. VT<TX, TY>
template <typename T, int PI, int PJ, typename G>
__device__ __forceinline__ void res_node(T* sr, const T* x0, const T* pc, int I, int J,
                                         const LevelDev& L, const T* x, T cl, T cb) {
  using V = G;
  const int nq = L.nq;
  if (I < 0 || J < 0 || I >= nq || J >= nq) return;  // outside: r stays 0
  if (!vfree(I, J, nq)) {                            // Dirichlet row: r = b - x
    const long long k = static_cast<long long>(J) * nq + I;
    sr[0] -= x[k];
    sr[V::RW * V::RH] -= x[L.nv + k];
    return;
  }
  const T* x1 = x0 + V::XW * V::XH;
  sr[0] -= cl * lap<T, PI, PJ, V::XW>(x0) + cb * btp<T, PI, PJ, 0, V::PW>(pc);
  sr[V::RW * V::RH] -= cl * lap<T, PI, PJ, V::XW>(x1) + cb * btp<T, PI, PJ, 1, V::PW>(pc);
}

// The global x of res_node / res_cell (read on Dirichlet rows) carries no
// __restrict__: in the persistent coarse-level kernel one step writes it and a later
// one reads it, so those loads must not take the read-only (non-coherent) path.
//
// Residual of the 2x2 cell of Q2 nodes (I0..I0+1) x (J0..J0+1) (I0, J0 even),
// both components.  When all four nodes are free, the 6x6 x neighbourhood of
// each component and the 3x3 pressures are loaded into registers once and the
// four stencils read them there; otherwise the per-node path handles the
// Dirichlet rows.  r0 / x0 point at (I0, J0) in the residual / x windows of
// component 0, pc at the pressure of vertex (I0/2, J0/2).
template <typename T, typename G>
__device__ __forceinline__ void res_cell(T* r0, const T* x0, const T* pc, int I0, int J0, const LevelDev& L,
                                         const T* x, T cl, T cb) {
  using V = G;
  const int nq = L.nq;
  if (I0 >= 1 && J0 >= 1 && I0 + 1 <= nq - 2 && J0 + 1 <= nq - 2) {
    T P[3][3];
#pragma unroll
    for (int dj = 0; dj < 3; ++dj)
#pragma unroll
      for (int di = 0; di < 3; ++di) P[dj][di] = pc[(dj - 1) * V::PW + (di - 1)];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const T* xc = x0 + c * V::XW * V::XH;
      T X[6][6];
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int bcol = 0; bcol < 6; ++bcol) X[a][bcol] = xc[(a - 2) * V::XW + (bcol - 2)];
#pragma unroll
      for (int PJ = 0; PJ < 2; ++PJ) {
#pragma unroll
        for (int PI = 0; PI < 2; ++PI) {
          T sl = T(0);
#pragma unroll
          for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
            for (int dI = -2; dI <= 2; ++dI) {
              const T cf = T(k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ));
              if (cf != T(0)) sl = fma(cf, X[PJ + dJ + 2][PI + dI + 2], sl);
            }
          }
          T g = T(0);
#pragma unroll
          for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
              const T w = T(c == 0 ? ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj)
                                   : ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj));
              if (w != T(0)) g = fma(w, P[dj + 1][di + 1], g);
            }
          }
          T& rr = r0[c * V::RW * V::RH + PJ * V::RW + PI];
          rr = fma(-cl, sl, fma(-cb, g, rr));   // r - (cl sl + cb g) as two multiply-adds
        }
      }
    }
    return;
  }
  res_node<T, 0, 0, G>(r0, x0, pc, I0, J0, L, x, cl, cb);
  res_node<T, 1, 0, G>(r0 + 1, x0 + 1, pc, I0 + 1, J0, L, x, cl, cb);
  res_node<T, 0, 1, G>(r0 + V::RW, x0 + V::XW, pc, I0, J0 + 1, L, x, cl, cb);
  res_node<T, 1, 1, G>(r0 + V::RW + 1, x0 + V::XW + 1, pc, I0 + 1, J0 + 1, L, x, cl, cb);
}

template <typename T>
__device__ __forceinline__ T inv_mult(int m) {
  switch (m) {
    case 1: return T(1.0);
    case 2: return T(0.5);
    case 3: return T(1.0 / 3.0);
    case 4: return T(0.25);
    case 6: return T(1.0 / 6.0);
    default: return T(1.0 / 9.0);
  }
}

}  // namespace vk
}  // namespace sv
