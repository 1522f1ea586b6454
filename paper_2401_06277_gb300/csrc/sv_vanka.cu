// sv_vanka.cu -- fused additive Vanka sweep (Section 3.2, Algorithm 3; the
// shared patch inverses of Section 6.3), templated on the element type:
// double for the FP64 form, float inside the mixed-precision preconditioner.
//
//   x_out = x + sum_i V_i^T W_i A_i^-1 V_i (b - A x),  W_i = omega diag(1/m_j)
//
// A CTA owns TX x TY vertices.  It loads x and b for the windows of the
// patches of those vertices plus a one-vertex halo, computes the residual
// there (every stencil coefficient is a compile-time constant: a thread
// handles one 2x2 cell of Q2 nodes, whose four node parities are fixed),
// solves every patch of the (TX+2) x (TY+2) region exactly with its class's
// Schur factors (K^-1 by fast diagonalisation of its tensor-product
// structure: the interior factors, or per-axis factors for boundary classes,
// whose free nodes form a sub-rectangle of the window), keeps the
// corrections in shared memory, and writes
// x + W (sum of corrections) for the dofs it owns: Q2 nodes
// (2i-1..2i) x (2j-1..2j) of both components and p(i, j) for each owned
// vertex (i, j).  The sum over patches runs in a fixed order (no atomics), so
// the result is deterministic.
//
// In FP64 the kernel is bound by the FP64 pipe on GB300 (2 DFMA / clk / SM).
// The tile shape trades halo recomputation against shared memory per CTA and
// is chosen per level by a timing autotuner at hierarchy creation.
//
// Issue-slot economies: window rows load one warp per row with compile-time
// extents; on tiles whose owned vertices lie in 1..n-1 the update sums each
// node's patch corrections at compile-time slot offsets; in FP32 the interior
// patch solves of u_x and u_y run as one packed pass (FFMA2 on component
// pairs) and the interior Schur vector is read from constant memory.
//
// The split sweep below (the operator kernel's residual, k_vanka_own, then
// k_colsum_update) solves only a tile's own patches and passes sums of their
// corrections through HBM: the better trade where the FP64 pipe is the bound.
#include <cuda_runtime.h>

#include <cmath>
#include <utility>

#include "sv_fastdiag.cuh"
#include "sv_internal.h"
#include "sv_level_ops.cuh"
#include "sv_stencil.cuh"
#include "sv_vanka_common.cuh"

namespace sv {
namespace {

using fdm::fd_fwd;
using fdm::fd_inv;
using fdm::fd_solve;
using fdm::fd_finish;
using fdm::fd_cols;
using fdm::operator+;
using fdm::operator-;
using fdm::operator*;
using ::fma;
using fdm::fma;

using vk::VT;
using vk::vfree;
using vk::res_node;
using vk::inv_mult;

// z_u of the interior patches (interior_unit_schur), in each precision: indexed
// by compile-time slots, it is read as a constant-bank operand of the FMAs.
__constant__ double c_zu[50];
__constant__ float c_zu_f[50];
template <typename R>
__device__ __forceinline__ R zu(int k);
template <>
__device__ __forceinline__ double zu<double>(int k) { return c_zu[k]; }
template <>
__device__ __forceinline__ float zu<float>(int k) { return c_zu_f[k]; }

// dp of a patch (Schur step, Section 6.3): (z . r_u - r_p) / s.  In FP32 a warp
// whose patches are all interior takes z = zs z_u from constant memory (50 fewer
// loads per patch); otherwise, and in FP64 (where the loads run beside the busy
// FP64 pipe and the constant path measured slower), z and 1 / s come from the
// patch's class data.
template <typename R>
__device__ __forceinline__ R schur_dp(bool warp_interior, const LevelDev& L, const R* __restrict__ C,
                                      const R (&ru)[50], R rp) {
  R zr = R(0);
  if (sizeof(R) == 4 && warp_interior) {
#pragma unroll
    for (int k = 0; k < 50; ++k) zr = fma(zu<R>(k), ru[k], zr);
    return (level_zs<R>(L) * zr - rp) * level_zsinv<R>(L);
  }
#pragma unroll
  for (int k = 0; k < 50; ++k) zr = fma(__ldg(C + CD_Z + k), ru[k], zr);
  return (zr - rp) * __ldg(C + CD_SINV);
}

// y = K^-1 r on the window of a patch of any class (ax, ay) by fast
// diagonalisation with the padded per-axis factors (sx, sy: [slot * 5 + mode]),
// dv = (90/nu) / (l_x + l_y) per mode pair (0 for padded modes); window slots
// off the free rectangle (fmask bit wj * 5 + wi clear) keep identity rows
// (y = r there).  r is read from the shared residual window (row stride rs);
// y, 25 values, is built in place in shared memory (rows, columns, columns,
// rows), which keeps few values live in registers.
template <typename T>
__device__ __forceinline__ void fd_solve_edge(const T* __restrict__ sx, const T* __restrict__ sy,
                                              const T* __restrict__ dv, int fmask, const T* r, int rs,
                                              T* y_, long long ys = 1) {
  struct Y {   // y[i] at stride ys (1: a shared-memory row; the split sweep's global delta: P)
    T* p;
    long long s;
    __device__ T& operator[](int i) const { return p[i * s]; }
  } y{y_, ys};
#pragma unroll 1
  for (int wj = 0; wj < 5; ++wj) {
    T v[5];
#pragma unroll
    for (int wi = 0; wi < 5; ++wi) v[wi] = r[wj * rs + wi];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      T a = T(0);
#pragma unroll
      for (int wi = 0; wi < 5; ++wi) a = fma(v[wi], sx[wi * 5 + k], a);
      y[wj * 5 + k] = a;
    }
  }
#pragma unroll 1
  for (int k = 0; k < 5; ++k) {
    T v[5], u[5];
#pragma unroll
    for (int wj = 0; wj < 5; ++wj) v[wj] = y[wj * 5 + k];
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) {
      T a = T(0);
#pragma unroll
      for (int wj = 0; wj < 5; ++wj) a = fma(sy[wj * 5 + k2], v[wj], a);
      u[k2] = a * dv[k2 * 5 + k];
    }
#pragma unroll
    for (int wj = 0; wj < 5; ++wj) {
      T a = T(0);
#pragma unroll
      for (int k2 = 0; k2 < 5; ++k2) a = fma(sy[wj * 5 + k2], u[k2], a);
      y[wj * 5 + k] = a;
    }
  }
#pragma unroll 1
  for (int wj = 0; wj < 5; ++wj) {
    T v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = y[wj * 5 + k];
#pragma unroll
    for (int wi = 0; wi < 5; ++wi) {
      T a = T(0);
#pragma unroll
      for (int k = 0; k < 5; ++k) a = fma(sx[wi * 5 + k], v[k], a);
      y[wj * 5 + wi] = ((fmask >> (wj * 5 + wi)) & 1) ? a : r[wj * rs + wi];
    }
  }
}

// FP32: fd_solve_edge for both velocity components at once.  The two components
// of a patch see the same scalar block K, so the per-axis factors are shared and
// each step is one packed multiply-add on the (u_x, u_y) pair, term by term the
// scalar pass: the values are those of two fd_solve_edge calls, in half the
// dependent steps.  r0, r1: the components' residual windows; y0, y1: their 25
// outputs (shared memory, also the scratch between the passes).
__device__ __forceinline__ void fd_solve_edge2(const float* __restrict__ sx, const float* __restrict__ sy,
                                               const float* __restrict__ dv, int fmask, const float* r0,
                                               const float* r1, int rs, float* y0, float* y1) {
  const auto pair = [](float s) { return make_float2(s, s); };
#pragma unroll 1
  for (int wj = 0; wj < 5; ++wj) {
    float2 v[5];
#pragma unroll
    for (int wi = 0; wi < 5; ++wi) v[wi] = make_float2(r0[wj * rs + wi], r1[wj * rs + wi]);
#pragma unroll
    for (int k = 0; k < 5; ++k) {
      float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int wi = 0; wi < 5; ++wi) a = __ffma2_rn(v[wi], pair(sx[wi * 5 + k]), a);
      y0[wj * 5 + k] = a.x;
      y1[wj * 5 + k] = a.y;
    }
  }
#pragma unroll 1
  for (int k = 0; k < 5; ++k) {
    float2 v[5], u[5];
#pragma unroll
    for (int wj = 0; wj < 5; ++wj) v[wj] = make_float2(y0[wj * 5 + k], y1[wj * 5 + k]);
#pragma unroll
    for (int k2 = 0; k2 < 5; ++k2) {
      float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int wj = 0; wj < 5; ++wj) a = __ffma2_rn(pair(sy[wj * 5 + k2]), v[wj], a);
      u[k2] = __fmul2_rn(a, pair(dv[k2 * 5 + k]));
    }
#pragma unroll
    for (int wj = 0; wj < 5; ++wj) {
      float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k2 = 0; k2 < 5; ++k2) a = __ffma2_rn(pair(sy[wj * 5 + k2]), u[k2], a);
      y0[wj * 5 + k] = a.x;
      y1[wj * 5 + k] = a.y;
    }
  }
#pragma unroll 1
  for (int wj = 0; wj < 5; ++wj) {
    float2 v[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) v[k] = make_float2(y0[wj * 5 + k], y1[wj * 5 + k]);
#pragma unroll
    for (int wi = 0; wi < 5; ++wi) {
      float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int k = 0; k < 5; ++k) a = __ffma2_rn(pair(sx[wi * 5 + k]), v[k], a);
      const bool keep = (fmask >> (wj * 5 + wi)) & 1;
      y0[wj * 5 + wi] = keep ? a.x : r0[wj * rs + wi];
      y1[wj * 5 + wi] = keep ? a.y : r1[wj * rs + wi];
    }
  }
}

// Load a ROWS x WIDTH window (row-major, pitch WIDTH) of src (row stride ld):
// element (jj, ii) is src[(J0 + jj) ld + I0 + ii] where ok(I, J), else 0.  Warp w
// takes rows w, w + NW, ...; lane k columns k, k + 32: the row's validity and
// address are formed once, and with compile-time extents every load is issued
// before the stores.
template <typename R, int ROWS, int WIDTH, int NW, typename OK>
__device__ __forceinline__ void load_window(R* __restrict__ dst, const R* src, long long ld, int I0,
                                            int J0, int warp, int lane, OK ok) {
  constexpr int RPW = (ROWS + NW - 1) / NW, CPL = (WIDTH + 31) / 32;
  R v[RPW][CPL];
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int jj = warp + k * NW, J = J0 + jj;
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
      const int ii = lane + 32 * h, I = I0 + ii;
      v[k][h] = (jj < ROWS && ii < WIDTH && ok(I, J)) ? src[static_cast<long long>(J) * ld + I] : R(0);
    }
  }
#pragma unroll
  for (int k = 0; k < RPW; ++k) {
    const int jj = warp + k * NW;
#pragma unroll
    for (int h = 0; h < CPL; ++h) {
      const int ii = lane + 32 * h;
      if (jj < ROWS && ii < WIDTH) dst[jj * WIDTH + ii] = v[k][h];
    }
  }
}

// One fused sweep of tile (bx, by) by the calling CTA (NT threads); smem_raw holds
// (VT<TX, TY>::TOTAL + EDGE_TAB) elements.  Shared by the stand-alone kernel
// below and the persistent coarse-level kernel, which loops over tiles.  x, b and
// xo carry no __restrict__ (see sv_level_ops.cuh): in the persistent kernel they
// are written by other steps of the same launch.
template <typename R, int TX, int TY, int NT>
__device__ __forceinline__ void vanka_tile(const LevelDev& L, const R* __restrict__ cd, const FastDiagT<R>& fdg,
                                           const FastDiagT<float2>& fdp, const R* x, const R* b, R* xo, R omega,
                                           int bx, int by, unsigned char* smem_raw) {
  using T = VT<TX, TY>;
  R* sx = reinterpret_cast<R*>(smem_raw);
  R* sp = sx + T::SX;
  R* sr = sp + T::SP;
  R* srp = sr + T::SR;
  R* sd = srp + T::SRP;
  R* se = sd + T::SD;   // fast-diagonalisation table of all classes (boundary tiles only)
  const int n = L.n, nq = L.nq, np = L.np;
  const long long nv = L.nv;
  const int i0 = bx * TX, j0 = by * TY;
  const int tid = threadIdx.x;
  const int XI0 = 2 * i0 - 6, XJ0 = 2 * j0 - 6;
  const int RI0 = 2 * i0 - 4, RJ0 = 2 * j0 - 4;

  // 0. tiles with patches of vertices 0, 1, n-1 or n stage the per-class factors
  const bool edge_tile = (i0 <= 2) || (j0 <= 2) || (i0 + TX >= n - 1) || (j0 + TY >= n - 1);
  if (edge_tile)
    for (int t = tid; t < EDGE_TAB; t += NT) se[t] = cd[CD_EDGE + t];

  // 1. x windows (Dirichlet / outside entries read as 0: their columns are
  //    dropped), b on the residual windows (0 outside).
  constexpr int NW = NT / 32;
  static_assert(NT % 32 == 0, "whole warps");
  const int warp = tid >> 5, lane = tid & 31;
  const auto free_node = [nq](int I, int J) { return vfree(I, J, nq); };
  const auto in_grid = [nq](int I, int J) { return I >= 0 && J >= 0 && I < nq && J < nq; };
  if (x != nullptr) {
#pragma unroll
    for (int c = 0; c < 2; ++c)
      load_window<R, T::XH, T::XW, NW>(sx + c * T::XW * T::XH, x + c * nv, nq, XI0, XJ0, warp, lane, free_node);
#pragma unroll
    for (int t = tid; t < T::SP; t += NT) {
      const int jj = t / T::PW, ii = t - jj * T::PW;
      const int i = i0 - 3 + ii, j = j0 - 3 + jj;
      sp[t] = (i >= 0 && j >= 0 && i <= n && j <= n) ? x[2 * nv + static_cast<long long>(j) * np + i] : R(0);
    }
  }
#pragma unroll
  for (int c = 0; c < 2; ++c)
    load_window<R, T::RH, T::RW, NW>(sr + c * T::RW * T::RH, b + c * nv, nq, RI0, RJ0, warp, lane, in_grid);
#pragma unroll
  for (int t = tid; t < T::SRP; t += NT) {
    const int jj = t / T::QW, ii = t - jj * T::QW;
    const int i = i0 - 1 + ii, j = j0 - 1 + jj;
    srp[t] = (i >= 0 && j >= 0 && i <= n && j <= n) ? b[2 * nv + static_cast<long long>(j) * np + i] : R(0);
  }
  __syncthreads();

  // 2. residual r = b - A x (skipped for a zero initial guess: r = b)
  const R cl = level_cl<R>(L), cb = level_cb<R>(L);
  if (x != nullptr) {
    for (int t = tid; t < T::CW * T::CH; t += NT) {
      const int cy = t / T::CW, cx = t - cy * T::CW;
      const int I0 = RI0 + 2 * cx, J0 = RJ0 + 2 * cy;
      const R* x0 = sx + (2 * cy + 2) * T::XW + (2 * cx + 2);
      const R* pc = sp + (cy + 1) * T::PW + (cx + 1);  // vertex (I0/2, J0/2)
      R* r0 = sr + (2 * cy) * T::RW + 2 * cx;
      vk::res_cell<R, T>(r0, x0, pc, I0, J0, L, x, cl, cb);
    }
    for (int t = tid; t < T::SRP; t += NT) {
      const int jj = t / T::QW, ii = t - jj * T::QW;
      const int i = i0 - 1 + ii, j = j0 - 1 + jj;
      if (i < 0 || j < 0 || i > n || j > n) continue;
      // window of vertex (i, j): Q2 (2i + dI) - XI0 = 2 ii + 4 + dI
      const R* xs0 = sx + (2 * jj + 4) * T::XW + (2 * ii + 4);
      const R* xs1 = xs0 + T::XW * T::XH;
      R s = R(0);
#pragma unroll
      for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
        for (int dI = -2; dI <= 2; ++dI) {
          const R wx = R(crow(dI) * nrow(dJ)), wy = R(nrow(dI) * crow(dJ));
          if (wx != R(0)) s = fma(wx, xs0[dJ * T::XW + dI], s);
          if (wy != R(0)) s = fma(wy, xs1[dJ * T::XW + dI], s);
        }
      }
      srp[t] -= cb * s;
    }
  }
  __syncthreads();

  // 3. exact patch solves, one thread per patch (Schur-factored class inverse)
  for (int t0 = 0; t0 < T::NPATCH; t0 += NT) {
    const int t = t0 + tid;
    const int qj = t / T::QW, qi = t - qj * T::QW;
    const int pi = i0 - 1 + qi, pj = j0 - 1 + qj;
    const bool valid = t < T::NPATCH && pi >= 0 && pj >= 0 && pi <= n && pj <= n;
    const int ax = valid ? axis_class(pi, n) : 2, ay = valid ? axis_class(pj, n) : 2;
    const int cls = 5 * ay + ax;
    // the interior path for a warp whose patches are all interior: a vote of all 32
    // lanes (lanes without a patch count as interior), so the choice depends on the
    // tile alone, not on how the compiler converged the loop
    const bool warp_interior = __all_sync(0xffffffffu, cls == INTERIOR_CLASS);
    if (!valid) continue;
    const R* C = cd + cls * CD_STRIDE;
    R ru[50];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int wj = 0; wj < 5; ++wj)
#pragma unroll
        for (int wi = 0; wi < 5; ++wi)
          ru[c * 25 + wj * 5 + wi] = sr[c * T::RW * T::RH + (2 * qj + wj) * T::RW + 2 * qi + wi];
    const R dp = schur_dp<R>(warp_interior, L, C, ru, srp[t]);
    R* D = sd + t * 51;
    // K^-1 r_u by fast diagonalisation (exact up to rounding): warps whose
    // patches are all interior use the symmetric/antisymmetric split of the
    // interior factors; a warp with any boundary-class patch takes the
    // per-axis factors for all of its patches (one path per warp)
    if (warp_interior) {
      // du = K^-1 r_u - z dp = K^-1 (r_u - b^T dp): the coupling b^T of an interior
      // patch is the compile-time stencil cb (C (x) N) / cb (N (x) C), 12 entries per component
      const R q = cb * dp;
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int w = 0; w < 25; ++w) {
          const int dI = w % 5 - 2, dJ = w / 5 - 2;
          const R bw = R(c == 0 ? crow(dI) * nrow(dJ) : nrow(dI) * crow(dJ));
          if (bw != R(0)) ru[c * 25 + w] = fma(-bw, q, ru[c * 25 + w]);
        }
      if constexpr (sizeof(R) == 4) {   // FP32: both components in one packed pass
        float2 r2[25], y2[25];
#pragma unroll
        for (int w = 0; w < 25; ++w) r2[w] = make_float2(ru[w], ru[25 + w]);
        fd_solve<float2>(fdp, r2, y2);
#pragma unroll
        for (int o = 0; o < 25; ++o) {
          D[o] = y2[o].x;
          D[25 + o] = y2[o].y;
        }
      } else {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          R y[25];
          fd_solve<R>(fdg, ru + c * 25, y);
#pragma unroll
          for (int o = 0; o < 25; ++o) D[c * 25 + o] = y[o];
        }
      }
    } else {
      const int fx = axis_free_mask(ax), fy = axis_free_mask(ay);
      int fmask = 0;
#pragma unroll
      for (int wj = 0; wj < 5; ++wj)
        if ((fy >> wj) & 1) fmask |= fx << (5 * wj);
      if constexpr (sizeof(R) == 4) {   // FP32: both components in one packed pass
        const R* r0 = sr + (2 * qj) * T::RW + 2 * qi;
        fd_solve_edge2(se + EDGE_S + ax * 25, se + EDGE_S + ay * 25, se + EDGE_DINV + cls * 25, fmask, r0,
                       r0 + T::RW * T::RH, T::RW, D, D + 25);
#pragma unroll 5
        for (int o = 0; o < 50; ++o) D[o] = fma(-__ldg(C + CD_Z + o), dp, D[o]);
      } else {
#pragma unroll 1
        for (int c = 0; c < 2; ++c) {
          R* y = D + c * 25;
          fd_solve_edge<R>(se + EDGE_S + ax * 25, se + EDGE_S + ay * 25, se + EDGE_DINV + cls * 25, fmask,
                           sr + c * T::RW * T::RH + (2 * qj) * T::RW + 2 * qi, T::RW, y);
#pragma unroll 5
          for (int o = 0; o < 25; ++o) y[o] = fma(-__ldg(C + CD_Z + c * 25 + o), dp, y[o]);
        }
      }
    }
    D[50] = dp;
  }
  __syncthreads();

  // 4. weighted additive update of the owned dofs, W = omega / m_j.  In a tile
  //    whose owned vertices all lie in 1..n-1 every owned node is free and is
  //    held by all 9 / 6 / 6 / 4 patches around it: one thread per owned vertex
  //    sums them at compile-time slot offsets (patch q + (dj, di), slot of the
  //    node), in the order of the general loop below, which serves the others.
  if (i0 >= 1 && j0 >= 1 && i0 + TX <= n && j0 + TY <= n) {
    static_assert(NT >= TX * TY, "one thread per owned vertex");
    if (tid < TX * TY) {
      const int vj = tid / TX, vi = tid - vj * TX;
      const int i = i0 + vi, j = j0 + vj;
      const R* dq = sd + ((vj + 1) * T::QW + (vi + 1)) * 51;   // the vertex's own patch
      const int xj = 2 * j - XJ0, xi = 2 * i - XI0;              // x window at node (2i, 2j)
      const long long base = static_cast<long long>(2 * j) * nq + 2 * i;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int nj = 0; nj < 2; ++nj) {      // node J = 2j - nj
#pragma unroll
          for (int ni = 0; ni < 2; ++ni) {    // node I = 2i - ni
            R acc = R(0);
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
              for (int di = -1; di <= 1; ++di) {
                if ((ni == 1 && di == 1) || (nj == 1 && dj == 1)) continue;
                const int wi = 2 - ni - 2 * di, wj = 2 - nj - 2 * dj;   // window offsets of the node
                acc += dq[(dj * T::QW + di) * 51 + c * 25 + wj * 5 + wi];
              }
            }
            const R w = omega * inv_mult<R>((ni ? 2 : 3) * (nj ? 2 : 3));
            const R xold = x != nullptr ? sx[c * T::XW * T::XH + (xj - nj) * T::XW + (xi - ni)] : R(0);
            xo[c * nv + base - static_cast<long long>(nj) * nq - ni] = fma(w, acc, xold);
          }
        }
      }
      const R xoldp = x != nullptr ? sp[(j - (j0 - 3)) * T::PW + (i - (i0 - 3))] : R(0);
      xo[2 * nv + static_cast<long long>(j) * np + i] = fma(omega, dq[50], xoldp);
    }
    return;
  }
  constexpr int OW = 2 * TX, OH = 2 * TY;
  for (int t = tid; t < 2 * OW * OH + TX * TY; t += NT) {
    if (t < 2 * OW * OH) {
      const int c = t / (OW * OH);
      const int rem = t - c * OW * OH;
      const int oj = rem / OW, oi = rem - oj * OW;
      const int I = 2 * i0 - 1 + oi, J = 2 * j0 - 1 + oj;
      if (I < 0 || J < 0 || I >= nq || J >= nq) continue;
      const int pil = I < 2 ? 0 : (I - 1) / 2, pih = min(n, (I + 2) / 2);
      const int pjl = J < 2 ? 0 : (J - 1) / 2, pjh = min(n, (J + 2) / 2);
      R acc = R(0);
      for (int pj = pjl; pj <= pjh; ++pj) {
        for (int pi = pil; pi <= pih; ++pi) {
          const int q = (pj - (j0 - 1)) * T::QW + (pi - (i0 - 1));
          acc += sd[q * 51 + c * 25 + (J - 2 * pj + 2) * 5 + (I - 2 * pi + 2)];
        }
      }
      const R w = omega * inv_mult<R>((pih - pil + 1) * (pjh - pjl + 1));
      const long long k = c * nv + static_cast<long long>(J) * nq + I;
      // x of free nodes is in the shared window; Dirichlet values come from global
      R xold = R(0);
      if (x != nullptr)
        xold = vfree(I, J, nq) ? sx[c * T::XW * T::XH + (J - XJ0) * T::XW + (I - XI0)] : x[k];
      xo[k] = fma(w, acc, xold);
    } else {
      const int u = t - 2 * OW * OH;
      const int vj = u / TX, vi = u - vj * TX;
      const int i = i0 + vi, j = j0 + vj;
      if (i > n || j > n) continue;
      const int q = (vj + 1) * T::QW + (vi + 1);
      const long long k = 2 * nv + static_cast<long long>(j) * np + i;
      const R xold = x != nullptr ? sp[(j - (j0 - 3)) * T::PW + (i - (i0 - 3))] : R(0);
      xo[k] = fma(omega, sd[q * 51 + 50], xold);
    }
  }
}

template <typename R, int TX, int TY, int NT>
__global__ void __launch_bounds__(NT, (sizeof(R) == 4 && NT == 256) ? 3 : 1) k_vanka(LevelDev L, const R* __restrict__ cd,
                                              const FastDiagT<R> fdg, const FastDiagT<float2> fdp,
                                              const R* __restrict__ x,
                                              const R* __restrict__ b, R* __restrict__ xo, R omega,
                                              int skip_lo, int skip_hi) {
  pdl_begin();
  // With a non-empty [skip_lo, skip_hi] the tensor-core kernel sweeps the tiles
  // in that square and this launch enumerates the ring of tiles around it
  // (1-D grid: rows below, the left/right parts of the middle rows, rows above).
  int bx = blockIdx.x, by = blockIdx.y;
  if (skip_hi >= skip_lo) {
    const int gx = (L.np + TX - 1) / TX;
    const int w = skip_hi - skip_lo + 1, mid_row = gx - w;
    const int idx = blockIdx.x, n_bottom = skip_lo * gx, n_mid = w * mid_row;
    if (idx < n_bottom) {
      by = idx / gx;
      bx = idx - by * gx;
    } else if (idx < n_bottom + n_mid) {
      const int k = idx - n_bottom, row = k / mid_row, c = k - row * mid_row;
      by = skip_lo + row;
      bx = c < skip_lo ? c : c + w;
    } else {
      const int k = idx - n_bottom - n_mid;
      by = skip_hi + 1 + k / gx;
      bx = k - (k / gx) * gx;
    }
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  vanka_tile<R, TX, TY, NT>(L, cd, fdg, fdp, x, b, xo, omega, bx, by, smem_raw);
}

// ---------------------------------------------------------------------------
// Split sweep: a CTA solves only the TX x TY patches of the vertices it owns (no
// halo patches) from the residual on a one-vertex halo -- formed by the operator
// kernel beforehand when the caller passes a scratch vector, else in the tile --
// and writes, per patch column, the sums of its patches' corrections (SplitOut);
// k_colsum_update then forms x + W sum of the corrections.  Against the fused
// kernel this trades 1.27x halo patch solves and 1.56x halo residuals for one
// write and one read of the sums: the better trade where the FP64 pipe, not HBM,
// is the bound.
//
// In a tile whose patches are all interior, the first pass of the fast
// diagonalisation (the transform along each window row) is shared: patches
// (qi, qj) and (qi, qj + 1) overlap in 3 node rows, so the transform of node row
// J over the window columns of patch column qi serves 2 or 3 patches.  It is
// computed once per (component, row, patch column) into shared memory, and each
// patch applies its Schur coupling to it by linearity:
//   T_rows(r_u - b^T q) = T_rows(r_u) - q T_rows(b^T),
// with T_rows(b^T) a constant table (BRows) whose zero entries are known at
// compile time (b^T rows are antisymmetric in x for u_x, symmetric for u_y).
// ---------------------------------------------------------------------------
template <int TX, int TY>
struct VO {
  static constexpr int XW = 2 * TX + 8, XH = 2 * TY + 8;   // x, Q2 nodes, origin 2 i0 - 4
  static constexpr int PW = TX + 4, PH = TY + 4;           // x, vertices,  origin i0 - 2
  static constexpr int CW = TX + 2, CH = TY + 2;           // residual cells, origin 2 i0 - 2
  static constexpr int RW = 2 * CW, RH = 2 * CH;           // residual, Q2 nodes
  static constexpr int NPATCH = TX * TY;                   // own patches, origin i0
  static constexpr int SX = 2 * XW * XH, SP = PW * PH, SR = 2 * RW * RH, SRP = NPATCH;
  static constexpr int TR = 2 * TY + 3;                    // node rows the patch windows use
  static constexpr int ST = 2 * TR * 5 * TX;               // shared row transforms [c][J][mode][qi]
  // layout: residual, pressure residual, then x, p and the edge tables, which the
  // row transforms of an interior tile overwrite once the residual is formed
  static constexpr int TAIL = (SX + SP + EDGE_TAB > ST) ? SX + SP + EDGE_TAB : ST;
  static constexpr int SA = TR * 5 * TX;                   // summed row coefficients [J][mode][qi]
  static constexpr int SMEM = SR + SRP + TAIL + SA;        // elements
};

// Output of the split sweep: per (component, tile row ty, node row lr of the tile's
// windows, window column w, patch column pi) the sum of the corrections of the
// tile's patches in patch column pi at node (2 pi - 2 + w, 32 ty - 2 + lr); the
// update adds the 2 or 3 patch columns and the 1 or 2 tile rows around a node.
// delta holds, in this order: 51 x P per-patch corrections (scratch of the edge
// tiles), the column sums [c][ty][lr][w][pi] with pi pitch ncol, then the
// pressure corrections [vertex].
struct SplitOut {
  int P;      // per-patch stride of the scratch
  int ncol;   // patch-column pitch of the column sums (tiles x TX)
  int nty;    // tile rows
  long long col_off, dp_off;
};
inline SplitOut split_out(const LevelDev& L) {
  SplitOut o;
  o.P = patch_stride(L);
  o.ncol = ((L.np + 15) / 16) * 16;
  o.nty = (L.np + 15) / 16;
  o.col_off = 51LL * o.P;
  o.dp_off = o.col_off + 2LL * o.nty * VO<16, 16>::TR * 5 * o.ncol;
  return o;
}


// Constant tables of an interior patch in the row-transformed basis (u_x window
// at 0, u_y window at 25; [wj * 5 + mode]):
//   t:  T_rows(b^T), the row transforms of its coupling windows, in the patch's
//       units (q = cb dp multiplies them);
//   zh: the unit Schur vector z_u seen through the row transform, zh = M^-T z_u
//       per row (M the 5 x 5 forward transform), so that z_u . r_u = zh . T_rows(r_u):
//       the Schur step reads the shared row transforms instead of r_u and z.
template <typename R>
struct BRows {
  R t[50];
  R zh[50];
};

// Compile-time zero patterns.  b^T: u_x rows wj = 1..3 are antisymmetric in x
// (crow), so only the antisymmetric modes 3, 4 survive the row transform; u_y rows
// wj != 2 are symmetric in x (nrow): only the symmetric modes 0..2.  z_u = K^-1 b^T
// inherits the parities (K commutes with the reflection x -> -x): zh keeps modes 3, 4
// of u_x and 0..2 of u_y in every row.
__host__ __device__ constexpr bool brows_nonzero(int c, int wj, int k) {
  return c == 0 ? (nrow(wj - 2) != 0.0 && k >= 3) : (crow(wj - 2) != 0.0 && k < 3);
}
__host__ __device__ constexpr bool zh_nonzero(int c, int k) { return c == 0 ? k >= 3 : k < 3; }

double g_zu_host[50];   // z_u as uploaded by set_interior_unit_z

template <typename R>
BRows<R> coupling_row_transforms(const FastDiagT<R>& f) {
  FastDiagT<double> fd{};
  for (int k = 0; k < 9; ++k) fd.se[k] = static_cast<double>(f.se[k]);
  for (int k = 0; k < 4; ++k) fd.so[k] = static_cast<double>(f.so[k]);
  BRows<R> o{};
  for (int c = 0; c < 2; ++c)
    for (int wj = 0; wj < 5; ++wj) {
      double v[5], cc[5];
      for (int wi = 0; wi < 5; ++wi)
        v[wi] = c == 0 ? crow(wi - 2) * nrow(wj - 2) : nrow(wi - 2) * crow(wj - 2);
      fd_fwd<double>(fd, v[0], v[1], v[2], v[3], v[4], cc);
      for (int k = 0; k < 5; ++k) o.t[c * 25 + wj * 5 + k] = brows_nonzero(c, wj, k) ? static_cast<R>(cc[k]) : R(0);
    }
  // M (row k = the transform's weights of v_0..v_4), then M^T zh_row = z_row by
  // Gaussian elimination with partial pivoting, row by row of each window
  double M[5][5];
  for (int k = 0; k < 5; ++k) {
    double e[5] = {0, 0, 0, 0, 0}, cc[5];
    e[k] = 1.0;
    fd_fwd<double>(fd, e[0], e[1], e[2], e[3], e[4], cc);   // column k of M
    for (int i = 0; i < 5; ++i) M[i][k] = cc[i];
  }
  for (int c = 0; c < 2; ++c)
    for (int wj = 0; wj < 5; ++wj) {
      double a[5][6];
      for (int i = 0; i < 5; ++i) {
        for (int j = 0; j < 5; ++j) a[i][j] = M[j][i];   // M^T
        a[i][5] = g_zu_host[c * 25 + wj * 5 + i];
      }
      for (int col = 0; col < 5; ++col) {
        int piv = col;
        for (int i = col + 1; i < 5; ++i)
          if (std::fabs(a[i][col]) > std::fabs(a[piv][col])) piv = i;
        for (int j = 0; j < 6; ++j) std::swap(a[col][j], a[piv][j]);
        for (int i = 0; i < 5; ++i) {
          if (i == col) continue;
          const double m = a[i][col] / a[col][col];
          for (int j = col; j < 6; ++j) a[i][j] -= m * a[col][j];
        }
      }
      for (int k = 0; k < 5; ++k)
        o.zh[c * 25 + wj * 5 + k] = zh_nonzero(c, k) ? static_cast<R>(a[k][5] / a[k][k]) : R(0);
    }
  return o;
}

template <typename R, int TX, int TY, int NT, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_vanka_own(LevelDev L, const R* __restrict__ cd,
                                                  const FastDiagT<R> fdg, const BRows<R> xb,
                                                  const R* __restrict__ x, const R* __restrict__ b,
                                                  R* delta, const SplitOut so) {
  pdl_begin();
  using T = VO<TX, TY>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  R* sr = reinterpret_cast<R*>(smem_raw);
  R* srp = sr + T::SR;
  R* sx = srp + T::SRP;
  R* sp = sx + T::SX;
  R* se = sp + T::SP;
  R* sT = sx;   // interior tiles: the shared row transforms, once x and p are dead
  R* sA = se + (T::TAIL - T::SX - T::SP);   // summed row coefficients of one component
  const int n = L.n, nq = L.nq, np = L.np;
  const long long nv = L.nv;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int tid = threadIdx.x;
  const int XI0 = 2 * i0 - 4, XJ0 = 2 * j0 - 4;
  const int RI0 = 2 * i0 - 2, RJ0 = 2 * j0 - 2;
  const int P = so.P;
  R* colsum = delta + so.col_off;
  R* dpo = delta + so.dp_off;
  // column sum (c, lr, w) of patch column i0 + qi
  auto col_at = [&](int c, int lr, int w, int qi) -> R& {
    return colsum[((static_cast<long long>(c) * so.nty + blockIdx.y) * T::TR + lr) * 5 * so.ncol +
                  static_cast<long long>(w) * so.ncol + i0 + qi];
  };

  const bool edge_tile = (i0 <= 1) || (j0 <= 1) || (i0 + TX - 1 >= n - 1) || (j0 + TY - 1 >= n - 1);
  if (edge_tile)
    for (int t = tid; t < EDGE_TAB; t += NT) se[t] = cd[CD_EDGE + t];
  if (x != nullptr) {
#pragma unroll
    for (int t = tid; t < T::SX; t += NT) {
      const int c = t / (T::XW * T::XH);
      const int rem = t - c * T::XW * T::XH;
      const int jj = rem / T::XW, ii = rem - jj * T::XW;
      const int I = XI0 + ii, J = XJ0 + jj;
      sx[t] = vfree(I, J, nq) ? x[c * nv + static_cast<long long>(J) * nq + I] : R(0);
    }
#pragma unroll
    for (int t = tid; t < T::SP; t += NT) {
      const int jj = t / T::PW, ii = t - jj * T::PW;
      const int i = i0 - 2 + ii, j = j0 - 2 + jj;
      sp[t] = (i >= 0 && j >= 0 && i <= n && j <= n) ? x[2 * nv + static_cast<long long>(j) * np + i] : R(0);
    }
  }
#pragma unroll
  for (int t = tid; t < T::SR; t += NT) {
    const int c = t / (T::RW * T::RH);
    const int rem = t - c * T::RW * T::RH;
    const int jj = rem / T::RW, ii = rem - jj * T::RW;
    const int I = RI0 + ii, J = RJ0 + jj;
    sr[t] = (I >= 0 && J >= 0 && I < nq && J < nq) ? b[c * nv + static_cast<long long>(J) * nq + I] : R(0);
  }
#pragma unroll
  for (int t = tid; t < T::SRP; t += NT) {
    const int jj = t / TX, ii = t - jj * TX;
    const int i = i0 + ii, j = j0 + jj;
    srp[t] = (i <= n && j <= n) ? b[2 * nv + static_cast<long long>(j) * np + i] : R(0);
  }
  __syncthreads();

  const R cl = level_cl<R>(L), cb = level_cb<R>(L);
  if (x != nullptr) {
    for (int t = tid; t < T::CW * T::CH; t += NT) {
      const int cy = t / T::CW, cx = t - cy * T::CW;
      const int I0 = RI0 + 2 * cx, J0 = RJ0 + 2 * cy;
      const R* x0 = sx + (2 * cy + 2) * T::XW + (2 * cx + 2);
      const R* pc = sp + (cy + 1) * T::PW + (cx + 1);
      R* r0 = sr + (2 * cy) * T::RW + 2 * cx;
      vk::res_cell<R, T>(r0, x0, pc, I0, J0, L, x, cl, cb);
    }
    for (int t = tid; t < T::SRP; t += NT) {
      const int jj = t / TX, ii = t - jj * TX;
      if (i0 + ii > n || j0 + jj > n) continue;
      const R* xs0 = sx + (2 * jj + 4) * T::XW + (2 * ii + 4);
      const R* xs1 = xs0 + T::XW * T::XH;
      R s = R(0);
#pragma unroll
      for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
        for (int dI = -2; dI <= 2; ++dI) {
          const R wx = R(crow(dI) * nrow(dJ)), wy = R(nrow(dI) * crow(dJ));
          if (wx != R(0)) s = fma(wx, xs0[dJ * T::XW + dI], s);
          if (wy != R(0)) s = fma(wy, xs1[dJ * T::XW + dI], s);
        }
      }
      srp[t] -= cb * s;
    }
  }
  __syncthreads();

  // interior tile: the row transforms of every (component, node row, patch column),
  // over x and p, which no thread reads any more
  const bool shared_rows = !edge_tile;
  if (shared_rows) {
    for (int t = tid; t < T::ST / 5; t += NT) {
      const int qi = t % TX, rest = t / TX;
      const int J = rest % T::TR, c = rest / T::TR;
      const R* src = sr + c * T::RW * T::RH + J * T::RW + 2 * qi;
      R cc[5];
      fd_fwd<R>(fdg, src[0], src[1], src[2], src[3], src[4], cc);
      R* dst = sT + (c * T::TR + J) * 5 * TX + qi;
#pragma unroll
      for (int k = 0; k < 5; ++k) dst[k * TX] = cc[k];
    }
    __syncthreads();
  }

  static_assert(T::NPATCH == NT, "one patch per thread");
  if (shared_rows) {
    // every patch of the tile is interior and valid: thread t owns patch (qi, qj)
    const int qj = tid / TX, qi = tid - qj * TX;
    const int pi = i0 + qi, pj = j0 + qj;
    // Schur step from the shared row transforms: z . r_u = zs (zh . T_rows(r_u)),
    // the two components summed separately
    R zr[2] = {R(0), R(0)};
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const R* src = sT + (c * T::TR + 2 * qj) * 5 * TX + qi;
#pragma unroll
      for (int wj = 0; wj < 5; ++wj)
#pragma unroll
        for (int k = 0; k < 5; ++k)
          if (zh_nonzero(c, k)) zr[c] = fma(xb.zh[c * 25 + wj * 5 + k], src[(wj * 5 + k) * TX], zr[c]);
    }
    const R dp = (level_zs<R>(L) * (zr[0] + zr[1]) - srp[tid]) * level_zsinv<R>(L);
    dpo[static_cast<long long>(pj) * np + pi] = dp;
    const R q = cb * dp;
    // first patch row (in the order of the phases below) whose window holds tile row lr
    auto first_phase = [&](int lr) {
      const int lo = max(0, (lr - 3) / 2), hi = min(TY - 1, lr / 2);
      int f = 3;
      for (int qq = lo; qq <= hi; ++qq) f = min(f, qq % 3);
      return f;
    };
#pragma unroll 1
    for (int c = 0; c < 2; ++c) {
      // K^-1 (r_u - b^T q) up to its last pass: row transforms minus the coupling,
      // then the column pass
      R Tm[25];
      const R* src = sT + (c * T::TR + 2 * qj) * 5 * TX + qi;
#pragma unroll
      for (int wj = 0; wj < 5; ++wj)
#pragma unroll
        for (int k = 0; k < 5; ++k) {
          const R v = src[(wj * 5 + k) * TX];
          Tm[wj * 5 + k] = brows_nonzero(c, wj, k) ? fma(-q, xb.t[c * 25 + wj * 5 + k], v) : v;
        }
      fd_cols<R>(fdg, Tm);
      // sum the row coefficients of the patches sharing a node row: patch rows qj of
      // one residue mod 3 have disjoint windows, so three phases add without races,
      // in a fixed order; the first contributor of a row stores
#pragma unroll 1
      for (int ph = 0; ph < 3; ++ph) {
        if (qj % 3 == ph) {
#pragma unroll
          for (int wj = 0; wj < 5; ++wj) {
            const int lr = 2 * qj + wj;
            R* dst = sA + lr * 5 * TX + qi;
            if (first_phase(lr) == ph) {
#pragma unroll
              for (int k = 0; k < 5; ++k) dst[k * TX] = Tm[wj * 5 + k];
            } else {
#pragma unroll
              for (int k = 0; k < 5; ++k) dst[k * TX] += Tm[wj * 5 + k];
            }
          }
        }
        __syncthreads();
      }
      // the last pass once per (node row, patch column): the inverse row transform of
      // the summed coefficients is the sum of the patches' corrections there
      for (int it = tid; it < T::TR * TX; it += NT) {
        const int lr = it / TX, q2 = it - lr * TX;
        R cc[5], v[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) cc[k] = sA[(lr * 5 + k) * TX + q2];
        fd_inv<R>(fdg, cc, v);
        if (i0 + q2 <= n) {
#pragma unroll
          for (int w = 0; w < 5; ++w) col_at(c, lr, w, q2) = v[w];
        }
      }
      __syncthreads();
    }
    return;
  }

  // edge tile: per-patch corrections into the scratch, then their column sums
  {
    const int t = tid;
    const int qj = t / TX, qi = t - qj * TX;
    const int pi = i0 + qi, pj = j0 + qj;
    const bool valid = pi <= n && pj <= n;
    const int ax = valid ? axis_class(pi, n) : 2, ay = valid ? axis_class(pj, n) : 2;
    const int cls = 5 * ay + ax;
    const bool warp_interior = __all_sync(0xffffffffu, cls == INTERIOR_CLASS);   // as in vanka_tile
    if (valid) {
      const R* C = cd + cls * CD_STRIDE;
      const int p = pj * np + pi;
      R* D = delta + p;
      R ru[50];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int wj = 0; wj < 5; ++wj)
#pragma unroll
          for (int wi = 0; wi < 5; ++wi)
            ru[c * 25 + wj * 5 + wi] = sr[c * T::RW * T::RH + (2 * qj + wj) * T::RW + 2 * qi + wi];
      const R dp = schur_dp<R>(warp_interior, L, C, ru, srp[t]);
      const int fx = axis_free_mask(ax), fy = axis_free_mask(ay);
      int fmask = 0;
#pragma unroll
      for (int wj = 0; wj < 5; ++wj)
        if ((fy >> wj) & 1) fmask |= fx << (5 * wj);
#pragma unroll 1
      for (int c = 0; c < 2; ++c) {
        R* y = D + static_cast<long long>(c * 25) * P;
        fd_solve_edge<R>(se + EDGE_S + ax * 25, se + EDGE_S + ay * 25, se + EDGE_DINV + cls * 25, fmask,
                            sr + c * T::RW * T::RH + (2 * qj) * T::RW + 2 * qi, T::RW, y, P);
#pragma unroll 5
        for (int o = 0; o < 25; ++o)
          y[static_cast<long long>(o) * P] = fma(-__ldg(C + CD_Z + c * 25 + o), dp, y[static_cast<long long>(o) * P]);
      }
      dpo[p] = dp;
    }
  }
  __syncthreads();   // the tile's corrections in the scratch are visible to the whole CTA
  for (int it = tid; it < 2 * T::TR * TX; it += NT) {
    const int qi = it % TX, rest = it / TX;
    const int lr = rest % T::TR, c = rest / T::TR;
    const int pi = i0 + qi;
    if (pi > n) continue;
    const int lo = max(0, (lr - 3) / 2), hi = min(min(TY - 1, lr / 2), n - j0);
#pragma unroll
    for (int w = 0; w < 5; ++w) {
      R acc = R(0);
      for (int qq = lo; qq <= hi; ++qq)   // patch rows in ascending order
        acc += __ldcg(delta + static_cast<long long>(c * 25 + (lr - 2 * qq) * 5 + w) * P +
                      static_cast<long long>(j0 + qq) * np + pi);
      col_at(c, lr, w, qi) = acc;
    }
  }
}

// x_out = x + (omega / m_j) (sum of the corrections at dof j) from the split
// sweep's column sums: for a Q2 node the 2 or 3 patch columns and the 1 or 2 tile
// rows whose windows hold it, summed in ascending order; the pressure from the
// dof's own patch.  One thread per vertex (a, b): its four Q2 nodes and p(a, b).
template <typename T, int PI, int PJ>
__device__ __forceinline__ void colsum_node(const LevelDev& L, const SplitOut& so, const T* __restrict__ cs,
                                            const T* __restrict__ x, T* __restrict__ xo, T omega, int a, int b) {
  using V = VO<16, 16>;
  const int I = 2 * a + PI, J = 2 * b + PJ, nq = L.nq, n = L.n;
  if (I >= nq || J >= nq) return;
  const int pil = max(0, a - (PI ? 0 : 1)), pih = min(n, a + 1);
  const int pjl = max(0, b - (PJ ? 0 : 1)), pjh = min(n, b + 1);
  const T w = omega * vk::inv_mult<T>((pih - pil + 1) * (pjh - pjl + 1));
  const int tyh = min(so.nty - 1, (J + 2) / 32);   // tile rows hold node rows 32 ty - 2 .. 32 ty + 32
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    T acc = T(0);
    for (int ty = max(0, tyh - 1); ty <= tyh; ++ty) {
      const int lr = J - 32 * ty + 2;
      if (lr < 0 || lr >= V::TR) continue;
      const T* row = cs + ((static_cast<long long>(c) * so.nty + ty) * V::TR + lr) * 5 * so.ncol;
      for (int pi = pil; pi <= pih; ++pi) acc += row[static_cast<long long>(I - 2 * pi + 2) * so.ncol + pi];
    }
    const long long k = c * L.nv + static_cast<long long>(J) * nq + I;
    xo[k] = fma(w, acc, x != nullptr ? x[k] : T(0));
  }
}

template <typename T>
__global__ void k_colsum_update(LevelDev L, const SplitOut so, const T* __restrict__ delta, const T* __restrict__ x,
                                T* __restrict__ xo, T omega) {
  pdl_begin();
  const int a = blockIdx.x * blockDim.x + threadIdx.x;
  const int b = blockIdx.y * blockDim.y + threadIdx.y;
  if (a > L.n || b > L.n) return;
  const T* cs = delta + so.col_off;
  colsum_node<T, 0, 0>(L, so, cs, x, xo, omega, a, b);
  colsum_node<T, 1, 0>(L, so, cs, x, xo, omega, a, b);
  colsum_node<T, 0, 1>(L, so, cs, x, xo, omega, a, b);
  colsum_node<T, 1, 1>(L, so, cs, x, xo, omega, a, b);
  const int p = b * L.np + a;
  const long long k = 2 * L.nv + p;
  xo[k] = fma(omega, delta[so.dp_off + p], x != nullptr ? x[k] : T(0));
}

template <typename R, int TX, int TY, int NT>
void launch_t(const LevelDev& L, const R* cd, const FastDiagT<R>& fd, const R* x, const R* b, R* xo,
              R omega, int skip_lo, int skip_hi, cudaStream_t s) {
  const int gx = (L.np + TX - 1) / TX, gy = (L.np + TY - 1) / TY;
  dim3 grid(gx, gy);
  if (skip_hi >= skip_lo) {  // ring of tiles around the tensor-core square only
    const int w = skip_hi - skip_lo + 1;
    grid = dim3(gx * gy - w * w, 1);
  }
  FastDiagT<float2> fp{};   // (v, v) pairs of the FP32 table for the packed interior solves
  if constexpr (sizeof(R) == 4)
    fp = fd_cast<float2>(fd, [](R v) { return make_float2(static_cast<float>(v), static_cast<float>(v)); });
  launch_pdl(k_vanka<R, TX, TY, NT>, dim3(grid), dim3(NT), (VT<TX, TY>::TOTAL + EDGE_TAB) * sizeof(R), s, L, cd, fd, fp, x, b, xo,
                                                                                    omega, skip_lo, skip_hi);
}

// ---------------------------------------------------------------------------
// Persistent coarse-level kernel.  The coarse levels of a V-cycle are small: a
// level of n <= 128 has at most 289 sweep tiles, and launched kernel by kernel
// every step costs its launch and drain latency rather than its work (about 65 us
// per level in the FP32 forms).  Here one cooperative launch runs all steps of
// the cycle below and at the tail's top level -- sweeps, residuals, transfers and
// the coarse solve, each with the same device code as the stand-alone kernels --
// separated by grid barriers.  Work items of a step (sweep tiles, vertices,
// coarse elements, matrix rows) are spread over the CTAs.
// ---------------------------------------------------------------------------
struct TailArgs {
  const TailOp* ops;
  int nops;
  const TailLevel* levels;
  const double* G;
  int N0;
  FastDiagT<float> fdg;
  FastDiagT<float2> fdp;
  float omega;
  unsigned* bar;     // [0] arrivals, [1] generation
  int* err;
  int spin_limit;
  int skip_arrival;  // test hook: CTA that withholds its first arrival (-1: none)
};

// Grid-wide barrier of a cooperative launch: arrivals counted with an acquire-
// release atomic, the last arrival resets the count and advances the generation
// with a release, the others poll it with acquire loads (bounded: after
// spin_limit polls the CTA sets *err and the kernel returns).  With the CTA
// barriers around it this orders every CTA's writes of a step before any read of
// the next step.
__device__ bool grid_barrier(const TailArgs& A, bool withhold) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned* cnt = A.bar;
    unsigned* gen = A.bar + 1;
    unsigned g;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(gen) : "memory");
    if (withhold) {
      ok = 0;
    } else {
      unsigned old;
      asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(cnt), "r"(1u) : "memory");
      if (old == gridDim.x - 1) {
        asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(cnt), "r"(0u) : "memory");
        asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(gen), "r"(1u) : "memory");
        ok = 1;
      } else {
        int it = 0;
        unsigned cur = g;
        while (it < A.spin_limit) {
          asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(gen) : "memory");
          if (cur != g) break;
          __nanosleep(64);
          ++it;
        }
        ok = (cur != g) ? 1 : 0;
        if (!ok) atomicExch(A.err, 1);
      }
    }
  }
  __syncthreads();
  return ok != 0;
}

__global__ void __launch_bounds__(TAIL_NT) k_tail(TailArgs A) {
  pdl_begin();
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int G = gridDim.x, cta = blockIdx.x, tid = threadIdx.x;
  const long long gtid = static_cast<long long>(cta) * TAIL_NT + tid, gstride = static_cast<long long>(G) * TAIL_NT;
  for (int o = 0; o < A.nops; ++o) {
    const TailOp op = A.ops[o];
    const TailLevel T = A.levels[op.level];
    const LevelDev& L = T.d;
    switch (op.kind) {
      case TAIL_SWEEP: {
        const int gx = (L.np + 7) / 8, nt = gx * ((L.np + 7) / 8);
        for (int t = cta; t < nt; t += G) {
          const int by = t / gx, bx = t - by * gx;
          vanka_tile<float, 8, 8, TAIL_NT>(L, T.cd, A.fdg, A.fdp, op.a, op.b, op.c, A.omega, bx, by, smem_raw);
          __syncthreads();
        }
        break;
      }
      case TAIL_ZERO:
        for (long long i = gtid; i < L.N; i += gstride) op.c[i] = 0.0f;
        break;
      case TAIL_COPY:
        for (long long i = gtid; i < L.N; i += gstride) op.c[i] = op.a[i];
        break;
      case TAIL_RESID: {
        const long long nvx = static_cast<long long>(L.np) * L.np;
        for (long long i = gtid; i < nvx; i += gstride) {
          const int bb = static_cast<int>(i / L.np), a = static_cast<int>(i - static_cast<long long>(bb) * L.np);
          ops::apply_vertex<float>(L, op.a, op.b, op.c, 1, a, bb);
        }
        break;
      }
      case TAIL_RESTRICT:
      case TAIL_PROLONG: {
        const LevelDev C = A.levels[op.level - 1].d;
        const long long ne = static_cast<long long>(C.n + 1) * (C.n + 1);
        for (long long i = gtid; i < ne; i += gstride) {
          const int ey = static_cast<int>(i / (C.n + 1)), ex = static_cast<int>(i - static_cast<long long>(ey) * (C.n + 1));
          if (op.kind == TAIL_RESTRICT)
            ops::restrict_elem<float>(L, C, op.a, op.c, ex, ey);
          else
            ops::prolong_elem<float>(L, C, op.a, op.c, ex, ey);
        }
        break;
      }
      case TAIL_COARSE: {
        const long long w0 = gtid >> 5, ws = gstride >> 5;
        const int lane = tid & 31;
        for (long long row = w0; row < A.N0; row += ws) {
          const double v = ops::coarse_row<float>(A.G, A.N0, op.a, static_cast<int>(row), lane);
          if (lane == 0) op.c[row] = static_cast<float>(v);
        }
        break;
      }
      default:
        break;
    }
    if (o + 1 < A.nops && !grid_barrier(A, o == 0 && cta == A.skip_arrival)) return;
  }
}

template <typename R, int TX, int TY, int NT>
cudaError_t prepare_t() {
  return cudaFuncSetAttribute(k_vanka<R, TX, TY, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              static_cast<int>((VT<TX, TY>::TOTAL + EDGE_TAB) * sizeof(R)));
}

template <typename R>
cudaError_t prepare_all() {
  cudaError_t e;
  if ((e = prepare_t<R, 8, 8, 128>()) != cudaSuccess) return e;
  if ((e = prepare_t<R, 16, 8, 192>()) != cudaSuccess) return e;
  if ((e = prepare_t<R, 16, 16, 352>()) != cudaSuccess) return e;
  if ((e = prepare_t<R, 4, 4, 64>()) != cudaSuccess) return e;
  return prepare_t<R, 14, 14, 256>();
}

}  // namespace

cudaError_t set_interior_unit_z(const double* z50) {
  for (int k = 0; k < 50; ++k) g_zu_host[k] = z50[k];
  float zf[50];
  for (int k = 0; k < 50; ++k) zf[k] = static_cast<float>(z50[k]);
  cudaError_t e = cudaMemcpyToSymbol(c_zu, z50, 50 * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(c_zu_f, zf, 50 * sizeof(float));
  return e;
}

constexpr size_t TAIL_SMEM = (VT<8, 8>::TOTAL + EDGE_TAB) * sizeof(float);

cudaError_t tail_prepare(int* max_ctas) {
  cudaError_t e = cudaFuncSetAttribute(k_tail, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(TAIL_SMEM));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tail, TAIL_NT, TAIL_SMEM)) != cudaSuccess)
    return e;
  *max_ctas = per_sm * sms;
  return cudaSuccess;
}

void launch_tail(const TailOp* ops, int nops, const TailLevel* levels, const double* G, int N0,
                 const FastDiagT<float>& fd, double omega, unsigned* bar, int* err, int spin_limit,
                 int skip_arrival, int grid, cudaStream_t s) {
  count_launches(1);
  TailArgs A;
  A.ops = ops;
  A.nops = nops;
  A.levels = levels;
  A.G = G;
  A.N0 = N0;
  A.fdg = fd;
  A.fdp = fd_cast<float2>(fd, [](float v) { return make_float2(v, v); });
  A.omega = static_cast<float>(omega);
  A.bar = bar;
  A.err = err;
  A.spin_limit = spin_limit;
  A.skip_arrival = skip_arrival;
  // the grid barrier needs every CTA resident at once: a cooperative launch
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(TAIL_NT);
  cfg.dynamicSmemBytes = TAIL_SMEM;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k_tail, A);
}

cudaError_t vanka_prepare() {
  const int smem_own = static_cast<int>(VO<16, 16>::SMEM * sizeof(double));
  cudaError_t e = cudaFuncSetAttribute(k_vanka_own<double, 16, 16, 256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       smem_own);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vanka_own<double, 16, 16, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_own);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vanka_own<float, 16, 16, 256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_own / 2);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vanka_own<float, 16, 16, 256, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             smem_own / 2);
  if (e == cudaSuccess) e = prepare_all<double>();
  if (e != cudaSuccess) return e;
  return prepare_all<float>();
}

template <typename R>
void launch_vanka(const LevelDev& L, const R* cd, const FastDiagT<R>& fd, const R* x, const R* b, R* xo,
                  double omega, int cfg, cudaStream_t s, int skip_lo, int skip_hi) {
  count_launches(1);
  const R w = R(omega);
  switch (cfg) {
    case 1: launch_t<R, 16, 8, 192>(L, cd, fd, x, b, xo, w, skip_lo, skip_hi, s); break;
    case 2: launch_t<R, 16, 16, 352>(L, cd, fd, x, b, xo, w, skip_lo, skip_hi, s); break;
    case 3: launch_t<R, 14, 14, 256>(L, cd, fd, x, b, xo, w, skip_lo, skip_hi, s); break;
    case VANKA_CFG_4: launch_t<R, 4, 4, 64>(L, cd, fd, x, b, xo, w, skip_lo, skip_hi, s); break;
    default: launch_t<R, 8, 8, 128>(L, cd, fd, x, b, xo, w, skip_lo, skip_hi, s); break;
  }
}

template <typename R>
void launch_vanka_split(const LevelDev& L, const R* cd, const FastDiagT<R>& fd, const R* x, const R* b, R* xo,
                        double omega, R* delta, int two_per_sm, cudaStream_t s, R* rscratch) {
  // with a scratch vector the residual is formed once per cell by the operator kernel
  // (instead of on the tiles' one-vertex halo), and the own-patch kernel takes it as
  // the right-hand side of a zero guess
  const R* xs = x;
  const R* bs = b;
  if (rscratch != nullptr && x != nullptr) {
    launch_apply<R>(L, x, b, rscratch, 1, s);
    xs = nullptr;
    bs = rscratch;
  }
  count_launches(1);
  const SplitOut so = split_out(L);
  dim3 grid((L.np + 15) / 16, (L.np + 15) / 16);
  constexpr size_t smem = VO<16, 16>::SMEM * sizeof(R);
  const BRows<R> xb = coupling_row_transforms<R>(fd);
  if (two_per_sm)
    launch_pdl(k_vanka_own<R, 16, 16, 256, 2>, dim3(grid), dim3(256), smem, s, L, cd, fd, xb, xs, bs, delta, so);
  else
    launch_pdl(k_vanka_own<R, 16, 16, 256, 1>, dim3(grid), dim3(256), smem, s, L, cd, fd, xb, xs, bs, delta, so);
  count_launches(1);
  launch_pdl(k_colsum_update<R>, dim3((L.np + 31) / 32, (L.np + 7) / 8), dim3(32, 8), 0, s, L, so,
             static_cast<const R*>(delta), x, xo, static_cast<R>(omega));
}
size_t split_delta_doubles(const LevelDev& L) {
  const SplitOut so = split_out(L);
  return static_cast<size_t>(so.dp_off) + static_cast<size_t>(L.np) * L.np;
}

template void launch_vanka_split<double>(const LevelDev&, const double*, const FastDiag&, const double*,
                                         const double*, double*, double, double*, int, cudaStream_t, double*);
template void launch_vanka_split<float>(const LevelDev&, const float*, const FastDiagT<float>&, const float*,
                                        const float*, float*, double, float*, int, cudaStream_t, float*);

template void launch_vanka<double>(const LevelDev&, const double*, const FastDiagT<double>&, const double*,
                                   const double*, double*, double, int, cudaStream_t, int, int);
template void launch_vanka<float>(const LevelDev&, const float*, const FastDiagT<float>&, const float*,
                                  const float*, float*, double, int, cudaStream_t, int, int);

const char* vanka_cfg_name(int cfg) {
  static const char* names[VANKA_NCFG] = {"8x8", "16x8", "16x16", "14x14"};
  return (cfg >= 0 && cfg < VANKA_NCFG) ? names[cfg] : "?";
}

}  // namespace sv
