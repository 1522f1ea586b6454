// sv_bs.cu -- Braess-Sarazin relaxation (Section 3.1, Algorithm 2: the inexact
// variant) and Schur-Uzawa relaxation (Section 3.3, Algorithm 4), matrix-free,
// templated on the V-cycle's element type.  With
// D = diag(L) and S = -(1/t) B D^-1 B^T one sweep is
//
//   r = b - A x                                              (k_apply)
//   g = r_p - (1/t) B D^-1 r_u,  diag(S),  dp = w_J g / diag(S)   (k_bs_rhs)
//   repeat jacobi_iters - 1 times:
//     dp += w_J (g - S dp) / diag(S)                         (k_bs_jacobi_s: S dp
//       from dp directly, a 5 x 5 vertex stencil away from the boundary)
//   du = (1/t) D^-1 (r_u - B^T dp);  x_out = x + omega_BS (du, dp)   (k_bs_update)
//
// Schur-Uzawa solves the block lower-triangular system [[tD, 0], [B, S]]: its
// Schur right-hand side r_p - B du with du = (1/t) D^-1 r_u is the same g, and
// its velocity update drops the B^T dp term.
//
// On a uniform grid diag(L) depends only on the parities of a node's indices:
// nu/90 times 224 (vertex), 352 (edge midpoints) or 512 (cell centre), so D^-1
// is a compile-time constant per stencil tap, as are all B and B^T weights.
// Dirichlet nodes have identity rows in L and zero columns in B: their D is 1,
// they carry no B coupling, and du = r_u / t there.
#include <cuda_runtime.h>

#include "sv_internal.h"
#include "sv_stencil.cuh"

namespace sv {
namespace {

__device__ __forceinline__ bool bs_free(int I, int J, int nq) { return I > 0 && J > 0 && I < nq - 1 && J < nq - 1; }

// Level constants in the element type, formed once on the host (no FP64
// arithmetic in the FP32 kernels): B weight, 1 / (nu/90), 1/t, Jacobi weight, omega.
template <typename T>
struct BSC {
  T cb, icl, inv_t, wj, om;
};

// diag(L) / (nu/90) at a free node of parities (PI, PJ)
__host__ __device__ constexpr double dcoef(int PI, int PJ) { return k1(PI, 0) * m1(PJ, 0) + m1(PI, 0) * k1(PJ, 0); }

// Pressure rows: g, diag(S) and the first Jacobi step.  One thread per vertex
// (a, b); taps at Q2 nodes (2a + dI, 2b + dJ), parities (dI & 1, dJ & 1).
template <typename T, bool MASK>
__device__ __forceinline__ void bs_rhs_vertex(const LevelDev& L, const T* __restrict__ r, T* __restrict__ g,
                                              T* __restrict__ ds, T* __restrict__ dp, BSC<T> k, int a, int b) {
  const int nq = L.nq;
  const long long nv = L.nv;
  const T cb = k.cb, icl = k.icl, inv_t = k.inv_t, wj = k.wj;
  T s = T(0), d = T(0);
#pragma unroll
  for (int dJ = -2; dJ <= 2; ++dJ)
#pragma unroll
    for (int dI = -2; dI <= 2; ++dI) {
      const double wx = crow(dI) * nrow(dJ), wy = nrow(dI) * crow(dJ);
      if (wx == 0.0 && wy == 0.0) continue;
      const int I = 2 * a + dI, J = 2 * b + dJ;
      if (MASK && !bs_free(I, J, nq)) continue;
      const T id = T(1.0 / dcoef(dI & 1, dJ & 1));
      const long long k = static_cast<long long>(J) * nq + I;
      if (wx != 0.0) s = fma(T(wx) * id, r[k], s);
      if (wy != 0.0) s = fma(T(wy) * id, r[nv + k], s);
      d = fma(T(wx * wx + wy * wy), id, d);
    }
  const int p = b * L.np + a;
  const T gv = r[2 * nv + p] - inv_t * cb * icl * s;
  const T dsv = -inv_t * cb * cb * icl * d;
  g[p] = gv;
  ds[p] = dsv;
  dp[p] = wj * gv / dsv;
}

template <typename T>
__global__ void k_bs_rhs(LevelDev L, const T* __restrict__ r, T* __restrict__ g, T* __restrict__ ds,
                         T* __restrict__ dp, BSC<T> k) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = L.n;
  if (a > n || b > n) return;
  if (a >= 2 && a <= n - 2 && b >= 2 && b <= n - 2)
    bs_rhs_vertex<T, false>(L, r, g, ds, dp, k, a, b);
  else
    bs_rhs_vertex<T, true>(L, r, g, ds, dp, k, a, b);
}

// (B^T p) / (cb) at node (2a + PI, 2b + PJ), component C, from the 3 x 3 pressures P around (a, b)
template <typename T, int PI, int PJ, int C>
__device__ __forceinline__ T btp3(const T (&P)[3][3]) {
  T s = T(0);
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj)
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const double w = C == 0 ? ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj) : ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj);
      if (w != 0.0) s = fma(T(w), P[dj + 1][di + 1], s);
    }
  return s;
}

template <typename T>
__device__ __forceinline__ void load_p3(const LevelDev& L, const T* __restrict__ p, int a, int b, T (&P)[3][3]) {
#pragma unroll
  for (int dj = 0; dj < 3; ++dj)
#pragma unroll
    for (int di = 0; di < 3; ++di) {
      const int i = a + di - 1, j = b + dj - 1;
      P[dj][di] = (i >= 0 && j >= 0 && i <= L.n && j <= L.n) ? p[static_cast<long long>(j) * L.np + i] : T(0);
    }
}

// Entry (v, v + o) of S / (-(1/t) cb^2 / cl) for a vertex v whose 5 x 5 node
// window is free: sum over the window's nodes n (offset from node 2v) of
// (w_x(n) w_x(n - 2o) + w_y(n) w_y(n - 2o)) / dcoef(parities of n), with
// w_x = C (x) N and w_y = N (x) C the integer B weights.  o = 0 gives diag(S).
__host__ __device__ constexpr double s_coef(int ox, int oy) {
  double s = 0.0;
  for (int nJ = -2; nJ <= 2; ++nJ)
    for (int nI = -2; nI <= 2; ++nI) {
      const int mI = nI - 2 * ox, mJ = nJ - 2 * oy;
      if (mI < -2 || mI > 2 || mJ < -2 || mJ > 2) continue;
      const double id = 1.0 / dcoef(nI & 1, nJ & 1);
      s += (crow(nI) * nrow(nJ) * crow(mI) * nrow(mJ) + nrow(nI) * crow(nJ) * nrow(mI) * crow(mJ)) * id;
    }
  return s;
}

// One Jacobi step on S with S dp formed directly from dp: dp_out = dp_in + w_J (g -
// S dp_in) / diag(S).  Vertices 2..n-2 apply the 5 x 5 vertex stencil s_coef
// (compile-time); the others compose S = -(1/t) B D^-1 B^T over their free
// nodes.  Replaces q = D^-1 B^T dp through HBM (two velocity components) and a
// second pass; dp_out must not alias dp_in.
template <typename T>
__global__ void k_bs_jacobi_s(LevelDev L, const T* __restrict__ dpi, const T* __restrict__ g,
                              const T* __restrict__ ds, T* __restrict__ dpo, BSC<T> kc) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
  const int n = L.n, nq = L.nq, np = L.np;
  if (a > n || b > n) return;
  T s = T(0);
  if (a >= 2 && a <= n - 2 && b >= 2 && b <= n - 2) {
    const T* d0 = dpi + static_cast<long long>(b) * np + a;
#pragma unroll
    for (int oy = -2; oy <= 2; ++oy)
#pragma unroll
      for (int ox = -2; ox <= 2; ++ox) {
        const double c = s_coef(ox, oy);
        if (c != 0.0) s = fma(T(c), d0[oy * np + ox], s);
      }
  } else {
#pragma unroll
    for (int dJ = -2; dJ <= 2; ++dJ)
#pragma unroll
      for (int dI = -2; dI <= 2; ++dI) {
        const double wx = crow(dI) * nrow(dJ), wy = nrow(dI) * crow(dJ);
        if (wx == 0.0 && wy == 0.0) continue;
        const int I = 2 * a + dI, J = 2 * b + dJ;
        if (!bs_free(I, J, nq)) continue;   // D^-1 B^T dp is 0 on Dirichlet nodes
        T qx = T(0), qy = T(0);
#pragma unroll
        for (int oy = -2; oy <= 2; ++oy)
#pragma unroll
          for (int ox = -2; ox <= 2; ++ox) {
            const int mI = dI - 2 * ox, mJ = dJ - 2 * oy;
            if (mI < -2 || mI > 2 || mJ < -2 || mJ > 2) continue;
            const double vx = crow(mI) * nrow(mJ), vy = nrow(mI) * crow(mJ);
            if (vx == 0.0 && vy == 0.0) continue;
            const int i = a + ox, j = b + oy;
            if (i < 0 || j < 0 || i > n || j > n) continue;
            const T pv = dpi[static_cast<long long>(j) * np + i];
            if (vx != 0.0) qx = fma(T(vx), pv, qx);
            if (vy != 0.0) qy = fma(T(vy), pv, qy);
          }
        s = fma(T(1.0 / dcoef(dI & 1, dJ & 1)), T(wx) * qx + T(wy) * qy, s);
      }
  }
  const int p = b * np + a;
  const T sdp = -kc.inv_t * kc.cb * kc.cb * kc.icl * s;
  dpo[p] = fma(kc.wj, (g[p] - sdp) / ds[p], dpi[p]);
}

// du = (1/t) D^-1 (r_u - B^T dp) (Braess-Sarazin) or (1/t) D^-1 r_u (Schur-Uzawa, UZ);
// x_out = x + omega (du, dp)
template <typename T, int PI, int PJ, bool UZ>
__device__ __forceinline__ void bs_update_node(const LevelDev& L, const T (&P)[3][3], const T* __restrict__ r,
                                               const T* __restrict__ x, T* __restrict__ xo, const BSC<T>& kc,
                                               int a, int b) {
  const int I = 2 * a + PI, J = 2 * b + PJ, nq = L.nq;
  if (I >= nq || J >= nq) return;
  const long long k = static_cast<long long>(J) * nq + I;
  const bool fr = bs_free(I, J, nq);
  const T inv_t = kc.inv_t, om = kc.om, cb = kc.cb;
  const T sc = inv_t * kc.icl * T(1.0 / dcoef(PI, PJ));
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    const long long kc = c * L.nv + k;
    T du;
    if (fr) {
      if (UZ) {
        du = sc * r[kc];
      } else {
        const T bt = c == 0 ? btp3<T, PI, PJ, 0>(P) : btp3<T, PI, PJ, 1>(P);
        du = sc * (r[kc] - cb * bt);
      }
    } else {
      du = inv_t * r[kc];
    }
    xo[kc] = fma(om, du, x != nullptr ? x[kc] : T(0));
  }
}

template <typename T, bool UZ>
__global__ void k_bs_update(LevelDev L, const T* __restrict__ r, const T* __restrict__ dp, const T* __restrict__ x,
                            T* __restrict__ xo, BSC<T> kc) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x, b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > L.n || b > L.n) return;
  T P[3][3];
  load_p3(L, dp, a, b, P);
  bs_update_node<T, 0, 0, UZ>(L, P, r, x, xo, kc, a, b);
  bs_update_node<T, 1, 0, UZ>(L, P, r, x, xo, kc, a, b);
  bs_update_node<T, 0, 1, UZ>(L, P, r, x, xo, kc, a, b);
  bs_update_node<T, 1, 1, UZ>(L, P, r, x, xo, kc, a, b);
  const long long kp = 2 * L.nv + static_cast<long long>(b) * L.np + a;
  xo[kp] = fma(kc.om, P[1][1], x != nullptr ? x[kp] : T(0));
}

}  // namespace

size_t bs_scratch_elems(const LevelDev& L) {
  return static_cast<size_t>(2 * L.nv) + 3 * static_cast<size_t>(L.np) * L.np;
}

template <typename T>
void launch_bs_sweep(const LevelDev& L, const BSParams& prm, T* scratch, T* rbuf, const T* x, const T* b, T* xo,
                     cudaStream_t s) {
  const long long np2 = static_cast<long long>(L.np) * L.np;
  T* q = scratch;                 // 2 nv: the second dp buffer of the Jacobi steps
  T* g = q + 2 * L.nv;            // np^2 each
  T* ds = g + np2;
  T* dp = ds + np2;
  const T* r = b;
  if (x != nullptr) {
    launch_apply<T>(L, x, b, rbuf, 1, s);
    r = rbuf;
  }
  const BSC<T> k{T(L.cb), T(1.0 / L.cl), T(1.0 / prm.t), T(prm.jacobi_weight), T(prm.omega)};
  dim3 blk(32, 8), grid((L.np + 31) / 32, (L.np + 7) / 8);
  count_launches(2 + (prm.jacobi_iters - 1));
  launch_pdl(k_bs_rhs<T>, dim3(grid), dim3(blk), 0, s, L, r, g, ds, dp, k);
  T* dp_other = q;
  for (int it = 1; it < prm.jacobi_iters; ++it) {
    launch_pdl(k_bs_jacobi_s<T>, dim3(grid), dim3(blk), 0, s, L, static_cast<const T*>(dp), static_cast<const T*>(g),
               static_cast<const T*>(ds), dp_other, k);
    T* t = dp;
    dp = dp_other;
    dp_other = t;
  }
  if (prm.uzawa)
    launch_pdl(k_bs_update<T, true>, dim3(grid), dim3(blk), 0, s, L, r, dp, x, xo, k);
  else
    launch_pdl(k_bs_update<T, false>, dim3(grid), dim3(blk), 0, s, L, r, dp, x, xo, k);
}

template void launch_bs_sweep<double>(const LevelDev&, const BSParams&, double*, double*, const double*,
                                      const double*, double*, cudaStream_t);
template void launch_bs_sweep<float>(const LevelDev&, const BSParams&, float*, float*, const float*, const float*,
                                     float*, cudaStream_t);

}  // namespace sv
