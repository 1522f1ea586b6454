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

template <typename T, int PI, int PJ, int TX, int TY>
__device__ __forceinline__ void res_node(T* sr, const T* x0, const T* pc, int I, int J,
                                         const LevelDev& L, const T* __restrict__ x, T cl, T cb) {
  using V = VT<TX, TY>;
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
