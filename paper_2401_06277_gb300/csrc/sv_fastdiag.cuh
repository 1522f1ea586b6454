// sv_fastdiag.cuh -- the interior patch solve of the Vanka sweeps by fast
// diagonalisation (Section 6.3: every interior patch has the same matrix, and its
// velocity block is a Kronecker sum, K = (nu/90)(k (x) m + m (x) k), so
// K^-1 = S (x) S diag(1/(l_a + l_b)) (S (x) S)^T with the generalised eigenvectors
// of (k, m)), shared by the SIMT sweep (sv_vanka.cu) and the FP32 strip sweep
// (sv_vanka_tc.cu).
#pragma once

#include "sv_internal.h"

namespace sv {
namespace fdm {

// Packed FP32 arithmetic on (u_x, u_y) pairs (sm_100 and later): both velocity
// components of a patch go through the same fast-diagonalisation transforms,
// so the FP32 sweep runs them as one pass of FFMA2 / FADD2 / FMUL2, each lane
// rounded exactly as the scalar operation (a - b as b * -1 + a).
__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a);
}
__device__ __forceinline__ float2 operator*(float2 a, float2 b) { return __fmul2_rn(a, b); }
using ::fma;   // keep the scalar overloads visible beside the pair one
__device__ __forceinline__ float2 fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// Forward transform of one 5-vector into the generalised eigenbasis S^T v
// (three symmetric, two antisymmetric eigenvectors, each scaled to 1 on the
// pair {0, 4}, so the first term needs no multiply: 4 add/sub + 8 FMA).  Also
// compiled for the host (T = double), which transforms constant windows with it.
template <typename T>
__host__ __device__ __forceinline__ void fd_fwd(const FastDiagT<T>& f, T v0, T v1, T v2, T v3, T v4, T* c) {
  const T e0 = v0 + v4, e1 = v1 + v3, o0 = v0 - v4, o1 = v1 - v3;
#pragma unroll
  for (int k = 0; k < 3; ++k) c[k] = fma(f.se[3 + k], e1, fma(f.se[6 + k], v2, e0));
#pragma unroll
  for (int k = 0; k < 2; ++k) c[3 + k] = fma(f.so[2 + k], o1, o0);
}

// Inverse transform S c of five eigen-coefficients (rows of the pair {0, 4}
// are all ones: 7 add/sub + 8 FMA/MUL).
template <typename T>
__device__ __forceinline__ void fd_inv(const FastDiagT<T>& f, const T* c, T* v) {
  T E[3], Od[2];
  E[0] = (c[0] + c[1]) + c[2];
#pragma unroll
  for (int m = 1; m < 3; ++m) E[m] = fma(f.se[m * 3], c[0], fma(f.se[m * 3 + 1], c[1], f.se[m * 3 + 2] * c[2]));
  Od[0] = c[3] + c[4];
  Od[1] = fma(f.so[2], c[3], f.so[3] * c[4]);
  v[0] = E[0] + Od[0];
  v[4] = E[0] - Od[0];
  v[1] = E[1] + Od[1];
  v[3] = E[1] - Od[1];
  v[2] = E[2];
}

// y = K^-1 r on an interior patch window (5 x 5, row-major [wj][wi]) by fast
// diagonalisation: transform both axes, divide by l_a + l_b, transform back.
// fd_rows is the first pass (along each window row), fd_finish the rest, which
// takes the row-transformed window Tm (overwritten) -- a sweep whose patches share
// their row transforms calls it alone.
template <typename T>
__device__ __forceinline__ void fd_rows(const FastDiagT<T>& f, const T* r, T* Tm) {
#pragma unroll
  for (int wj = 0; wj < 5; ++wj)
    fd_fwd(f, r[wj * 5], r[wj * 5 + 1], r[wj * 5 + 2], r[wj * 5 + 3], r[wj * 5 + 4], Tm + wj * 5);
}

// The column pass (fd_cols) -- forward transform along y, division by l_a + l_b,
// inverse transform along y -- is one operator per window column that keeps the
// parity split (f.gs, f.ga): 4 add/sub, a 3 x 3 and a 2 x 2 product, 4 add/sub (21
// operations instead of 12 + 5 + 15).  Tm holds row coefficients before and after.
template <typename T>
__device__ __forceinline__ void fd_cols(const FastDiagT<T>& f, T* Tm) {
#pragma unroll
  for (int k = 0; k < 5; ++k) {
    const T v0 = Tm[k], v1 = Tm[5 + k], v2 = Tm[10 + k], v3 = Tm[15 + k], v4 = Tm[20 + k];
    const T e0 = v0 + v4, e1 = v1 + v3, o0 = v0 - v4, o1 = v1 - v3;
    const T* G = f.gs + 9 * k;
    const T* H = f.ga + 4 * k;
    T E[3];
#pragma unroll
    for (int m = 0; m < 3; ++m) E[m] = fma(G[3 * m], e0, fma(G[3 * m + 1], e1, G[3 * m + 2] * v2));
    const T O0 = fma(H[0], o0, H[1] * o1), O1 = fma(H[2], o0, H[3] * o1);
    Tm[k] = E[0] + O0;
    Tm[20 + k] = E[0] - O0;
    Tm[5 + k] = E[1] + O1;
    Tm[15 + k] = E[1] - O1;
    Tm[10 + k] = E[2];
  }
}

// fd_cols, then the inverse transform along each window row
template <typename T>
__device__ __forceinline__ void fd_finish(const FastDiagT<T>& f, T* Tm, T* y) {
  fd_cols(f, Tm);
#pragma unroll
  for (int wj = 0; wj < 5; ++wj) fd_inv(f, Tm + wj * 5, y + wj * 5);
}

template <typename T>
__device__ __forceinline__ void fd_solve(const FastDiagT<T>& f, const T* r, T* y) {
  T Tm[25];
  fd_rows(f, r, Tm);
  fd_finish(f, Tm, y);
}

}  // namespace fdm
}  // namespace sv
