// sv_vanka_tc.cu -- additive Vanka sweep with the interior patch solves as one
// BF16 GEMM per tile on the 5th-generation tensor cores (tcgen05), for the
// mixed-precision preconditioner (FP32 vectors, FP32 accumulation).
//
// Section 6.3 of the paper observes that on a uniform grid all interior patches
// share one patch matrix A_int.  The solves delta_i = A_int^-1 r_i of a tile's
// 256 patches are therefore the product D = R A_int^-T with R the 256 x 51
// matrix of gathered patch residuals (Algorithm 3, Section 3.2): M = 256
// (two M=128 MMAs), N = K = 51, padded to 64.
//
// One CTA per 14 x 14 vertex tile (256 threads, one per patch of the 16 x 16
// patch region including the one-vertex halo):
//   1. warp 0 allocates 128 TMEM columns; thread 0 starts a bulk (TMA) copy of
//      the 8 KB BF16 inverse, already in the UMMA core-matrix layout, into
//      shared memory, completing on an mbarrier;
//   2. the x and p windows are loaded; one thread per 2x2 cell of Q2 nodes
//      reads b from global memory and forms the FP32 residual of its four
//      nodes (compile-time stencils) and, from the same registers, the
//      pressure residual of the cell's vertex;
//   3. each thread writes its patch row of R, converted to BF16, into the
//      K-major no-swizzle core-matrix layout (8 rows x 16 bytes per core
//      matrix, LBO = 128 B along K, SBO = 1024 B along M);
//   4. thread 0 issues 2 x 4 tcgen05.mma (kind::f16, M=128, N=64, K=16) into
//      TMEM and commits them to an mbarrier;
//   5. after the wait, each thread reads its patch row of D with tcgen05.ld and
//      stores the 51 corrections in shared memory (over the dead R, B and
//      residual buffers);
//   6. x_out = x + (omega / m_j) * sum of the corrections of the patches that
//      hold the dof, summed in a fixed order (deterministic, no atomics).
// The x and residual windows hold (u_x, u_y) pairs (float2), so a stencil tap
// of both components is one 64-bit load and one packed FP32 FMA (FFMA2; the
// two components share the Laplacian stencil), and are stored column-parity
// split (the even nodes of a row, then the odd ones) with row pitches for which
// the stencil, patch-gather and update loads are free of bank conflicts.
// Every wait is bounded; on expiry the kernel sets *err, waits (bounded, with
// the full limit) for its bulk copy and MMAs, frees its TMEM and returns.  The
// limit of the first wait (the inverse's bulk copy) is a launch argument, so a
// test can make it expire (0 polls) without faulting or hanging anything.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "sv_internal.h"
#include "sv_stencil.cuh"
#include "sv_vanka_common.cuh"

namespace sv {
namespace {

using vk::inv_mult;
using vk::VT;
using vk::vfree;

constexpr int TC_NT = 256;
using TT = VT<TC_TILE, TC_TILE>;
static_assert(TT::NPATCH == TC_NT, "one thread per patch");
static_assert(TC_TILE % 2 == 0 && TC_TILE / 2 <= TC_NT / 32 && 2 * TC_TILE <= 32, "update: two vertex rows per warp");

// Windows (origins as in the SIMT sweep: x at Q2 node 2 i0 - 6, residual at
// 2 i0 - 4, p at vertex i0 - 3).  A row of the x window holds the (u_x, u_y)
// pairs of its 20 even nodes, then of its 20 odd ones; a residual row those of
// its 18 even, then 18 odd nodes.  A half-warp's 64-bit accesses are free of
// bank conflicts when its 16 addresses differ modulo 16 pairs.  The residual
// cells are taken row-major, 18 per row (item t = 18 cy + cx); x rows two apart
// (one cell row) are 2 XP = 82 = 18 = 2 (mod 16) pairs apart, so the pair index
// of every stencil load is t + const (mod 16), and the same holds for the cell
// stores into the residual window (RP = 41); the patch gather reads one row of
// 16 patches per half-warp.  p (scalar) rows have pitch 50 = 18 (mod 32): the
// bank of a p load is t + const (mod 32).
constexpr int XP = 41, XHALF = 20;                         // x: 40 rows of 40 pairs (+1 pad)
constexpr int RP = 41, RHALF = 18;                         // residual: 36 rows of 36 pairs (+5 pad)
constexpr int PP = 50;                                     // p: 20 rows of 20
static_assert(TT::XW == 2 * XHALF && TT::XW <= XP && TT::RW == 2 * RHALF && TT::RW <= RP && TT::PW <= PP,
              "window widths");
static_assert((2 * XP) % 16 == TT::CW % 16 && (2 * RP) % 16 == TT::CW % 16 && PP % 32 == TT::CW,
              "bank schedule");
__device__ __forceinline__ int xcol(int ii) { return (ii & 1) * XHALF + (ii >> 1); }

// shared-memory layout (bytes).  The correction array D (256 x 51 FP32,
// 52,224 B) overlays A, B, the residual and the pressure residual, which are
// all dead once the MMAs have completed; the x windows stay live for x_old.
constexpr int OFF_A = 0;                                   // 256 x 64 BF16 = 32 KB
constexpr int OFF_B = OFF_A + 256 * 64 * 2;                // 64 x 64 BF16 = 8 KB
constexpr int OFF_R = OFF_B + 64 * 64 * 2;                 // residual pairs (FP32)
constexpr int OFF_RP = OFF_R + TT::RH * RP * 8;            // pressure residual
constexpr int OFF_X = OFF_RP + TT::SRP * 4;                // x window pairs
constexpr int OFF_P = OFF_X + TT::XH * XP * 8;             // p window
constexpr int OFF_BAR = OFF_P + TT::PH * PP * 4;           // two mbarriers
constexpr int OFF_TMEM = OFF_BAR + 16;                     // TMEM base address
constexpr int SMEM_BYTES = OFF_TMEM + 16;
constexpr int OFF_D = 0;                                   // corrections, after the MMAs
static_assert(OFF_D + TT::NPATCH * 51 * 4 <= OFF_X, "corrections overlay only dead buffers");
static_assert(OFF_BAR % 8 == 0 && OFF_R % 8 == 0 && OFF_X % 8 == 0, "mbarrier and float2 alignment");

constexpr uint32_t TMEM_COLS = 128;
constexpr int WAIT_LIMIT = TC_WAIT_LIMIT;

__device__ __forceinline__ uint32_t su32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// UMMA shared-memory descriptor: K-major, no swizzle (layout type 0), version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= static_cast<uint64_t>((saddr >> 4) & 0x3FFF);
  d |= static_cast<uint64_t>((128u >> 4) & 0x3FFF) << 16;   // LBO: next core matrix along K
  d |= static_cast<uint64_t>((1024u >> 4) & 0x3FFF) << 32;  // SBO: next 8-row group along M/N
  d |= static_cast<uint64_t>(1) << 46;
  return d;
}

// instruction descriptor: D FP32, A/B BF16, both K-major, N = 64, M = 128
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase, int limit = WAIT_LIMIT) {
  for (int it = 0; it < limit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(TC_NT) k_vanka_tc(LevelDev L, const uint4* __restrict__ Bg,
                                                     const float* __restrict__ x,
                                                     const float* __restrict__ b, float* __restrict__ xo,
                                                     float omega, int tile0, int* __restrict__ err,
                                                     int first_wait_limit) {
  pdl_begin();
  extern __shared__ __align__(1024) unsigned char sm[];
  float2* sx = reinterpret_cast<float2*>(sm + OFF_X);
  float* sp = reinterpret_cast<float*>(sm + OFF_P);
  float2* sr = reinterpret_cast<float2*>(sm + OFF_R);
  float* srp = reinterpret_cast<float*>(sm + OFF_RP);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_TMEM);
  const uint32_t bar_b = su32(bars), bar_mma = su32(bars + 1);
  const int nq = L.nq, np = L.np;
  const long long nv = L.nv;
  const int i0 = (tile0 + static_cast<int>(blockIdx.x)) * TC_TILE;
  const int j0 = (tile0 + static_cast<int>(blockIdx.y)) * TC_TILE;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int XI0 = 2 * i0 - 6, XJ0 = 2 * j0 - 6;
  const int RI0 = 2 * i0 - 4, RJ0 = 2 * j0 - 4;

  // 1. barriers, TMEM, bulk copy of the BF16 inverse
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_b), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_mma), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  if (tid == 0) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_b), "r"(64 * 64 * 2)
                 : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            su32(sm + OFF_B)),
        "l"(Bg), "r"(64 * 64 * 2), "r"(bar_b)
        : "memory");
  }

  // 2. x and p windows (x of Dirichlet or outside nodes reads as 0: those
  //    columns are eliminated); residual of every cell (all cells of an
  //    interior tile are free), b read from global memory
  if (x != nullptr) {
    // warp w fills window rows w, w + 8, ..., lane k pair k of a row (even
    // nodes first, then odd): row validity and address once per row, all loads
    // issued before the stores (fully unrolled)
    constexpr int XROWS = TT::XH / (TC_NT / 32);
    static_assert(TT::XH % (TC_NT / 32) == 0 && TT::XW > 32 && TT::XW <= 64, "x window rows per warp");
    float2 xv[XROWS][2];
#pragma unroll
    for (int k = 0; k < XROWS; ++k) {
      const int jj = warp + k * (TC_NT / 32);
      const int J = XJ0 + jj;
      const bool jfree = J > 0 && J < nq - 1;
      const float* xr = x + static_cast<long long>(jfree ? J : 0) * nq;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int pos = lane + 32 * h;
        const int I = XI0 + (pos < XHALF ? 2 * pos : 2 * (pos - XHALF) + 1);
        const bool ok = jfree && pos < TT::XW && I > 0 && I < nq - 1;
        xv[k][h] = ok ? make_float2(xr[I], xr[nv + I]) : make_float2(0.0f, 0.0f);
      }
    }
#pragma unroll
    for (int k = 0; k < XROWS; ++k) {
      float2* dst = sx + (warp + k * (TC_NT / 32)) * XP;
      dst[lane] = xv[k][0];
      if (lane + 32 < TT::XW) dst[lane + 32] = xv[k][1];
    }
    // p window: 20 x 20 vertices, flat over the CTA
#pragma unroll
    for (int t = tid; t < TT::SP; t += TC_NT) {
      const int jj = t / TT::PW, ii = t - jj * TT::PW;
      const int i = i0 - 3 + ii, j = j0 - 3 + jj;
      sp[jj * PP + ii] = (i >= 0 && j >= 0 && i < np && j < np) ? x[2 * nv + static_cast<long long>(j) * np + i] : 0.0f;
    }
  }
  __syncthreads();
  const float cl = L.clf, cb = L.cbf;
  // cell (cx, cy) of the 18 x 18 residual cells: nodes (RI0 + 2 cx + PI, RJ0 + 2 cy + PJ),
  // taken row-major (t = 18 cy + cx)
  for (int t = tid; t < TT::CW * TT::CH; t += TC_NT) {
    const int cy = t / TT::CW, cx = t - cy * TT::CW;
    const int I0 = RI0 + 2 * cx, J0 = RJ0 + 2 * cy;
    const bool own_p = cx >= 1 && cy >= 1 && cx <= TT::QW && cy <= TT::QH;   // the vertex carries a patch
    float rp = own_p ? b[2 * nv + static_cast<long long>(J0 >> 1) * np + (I0 >> 1)] : 0.0f;
    float2 r[2][2];   // [PJ][PI]: (u_x, u_y) residual of node (I0 + PI, J0 + PJ)
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
      for (int PI = 0; PI < 2; ++PI) {
        const long long k = static_cast<long long>(J0 + PJ) * nq + I0 + PI;
        r[PJ][PI] = make_float2(b[k], b[nv + k]);
      }
    if (x != nullptr) {
      float P[3][3];
#pragma unroll
      for (int dj = 0; dj < 3; ++dj)
#pragma unroll
        for (int di = 0; di < 3; ++di) P[dj][di] = sp[(cy + dj) * PP + cx + di];
      // rows a = 0..5 of the 6 x 6 pair neighbourhood (node (I0 - 2 + bb, J0 - 2 + a))
      // stream through registers: each feeds the Laplacian of the nodes it reaches
      // and, for a <= 4, the divergence row of the vertex (node (I0, J0))
      const float2* xc = sx + 2 * cy * XP + cx;
      float2 sl[2][2];
#pragma unroll
      for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
        for (int PI = 0; PI < 2; ++PI) sl[PJ][PI] = make_float2(0.0f, 0.0f);
      float2 sdiv = make_float2(0.0f, 0.0f);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        float2 Xa[6];
#pragma unroll
        for (int bb = 0; bb < 6; ++bb) Xa[bb] = xc[a * XP + (bb & 1) * XHALF + (bb >> 1)];
#pragma unroll
        for (int PJ = 0; PJ < 2; ++PJ) {
#pragma unroll
          for (int PI = 0; PI < 2; ++PI) {
#pragma unroll
            for (int bb = 0; bb < 6; ++bb) {
              const int dJ = a - 2 - PJ, dI = bb - 2 - PI;
              const float cf = (dJ < -2 || dJ > 2 || dI < -2 || dI > 2)
                                   ? 0.0f
                                   : static_cast<float>(k1(PI, dI) * m1(PJ, dJ) + m1(PI, dI) * k1(PJ, dJ));
              if (cf != 0.0f) sl[PJ][PI] = __ffma2_rn(make_float2(cf, cf), Xa[bb], sl[PJ][PI]);
            }
          }
        }
        if (a <= 4) {   // -int p div u of the vertex: C (x) N on u_x, N (x) C on u_y
#pragma unroll
          for (int bb = 0; bb < 5; ++bb) {
            const float wx = static_cast<float>(crow(bb - 2) * nrow(a - 2));
            const float wy = static_cast<float>(nrow(bb - 2) * crow(a - 2));
            if (wx != 0.0f || wy != 0.0f) sdiv = __ffma2_rn(make_float2(wx, wy), Xa[bb], sdiv);
          }
        }
      }
#pragma unroll
      for (int PJ = 0; PJ < 2; ++PJ) {
#pragma unroll
        for (int PI = 0; PI < 2; ++PI) {
          float g0 = 0.0f, g1 = 0.0f;   // (B^T p) / (-h/18) for u_x, u_y
#pragma unroll
          for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
            for (int di = -1; di <= 1; ++di) {
              const float w0 = static_cast<float>(ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj));
              const float w1 = static_cast<float>(ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj));
              if (w0 != 0.0f) g0 = fmaf(w0, P[dj + 1][di + 1], g0);
              if (w1 != 0.0f) g1 = fmaf(w1, P[dj + 1][di + 1], g1);
            }
          }
          r[PJ][PI].x -= cl * sl[PJ][PI].x + cb * g0;
          r[PJ][PI].y -= cl * sl[PJ][PI].y + cb * g1;
        }
      }
      rp -= cb * (sdiv.x + sdiv.y);
    }
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
      for (int PI = 0; PI < 2; ++PI) sr[(2 * cy + PJ) * RP + PI * RHALF + cx] = r[PJ][PI];
    if (own_p) srp[(cy - 1) * TT::QW + (cx - 1)] = rp;
  }
  __syncthreads();

  // 3. this thread's patch row of R (BF16, core-matrix layout)
  const int qj = tid / TT::QW, qi = tid - qj * TT::QW;
  {
    float row[64];
#pragma unroll
    for (int wj = 0; wj < 5; ++wj)
#pragma unroll
      for (int wi = 0; wi < 5; ++wi) {
        const float2 v = sr[(2 * qj + wj) * RP + (wi & 1) * RHALF + qi + (wi >> 1)];
        row[wj * 5 + wi] = v.x;
        row[25 + wj * 5 + wi] = v.y;
      }
    row[50] = srp[tid];
#pragma unroll
    for (int k = 51; k < 64; ++k) row[k] = 0.0f;
    unsigned char* arow = sm + OFF_A + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll
    for (int kg = 0; kg < 8; ++kg) {
      uint4 v;
      __nv_bfloat162 h0 = __floats2bfloat162_rn(row[8 * kg + 0], row[8 * kg + 1]);
      __nv_bfloat162 h1 = __floats2bfloat162_rn(row[8 * kg + 2], row[8 * kg + 3]);
      __nv_bfloat162 h2 = __floats2bfloat162_rn(row[8 * kg + 4], row[8 * kg + 5]);
      __nv_bfloat162 h3 = __floats2bfloat162_rn(row[8 * kg + 6], row[8 * kg + 7]);
      memcpy(&v.x, &h0, 4);
      memcpy(&v.y, &h1, 4);
      memcpy(&v.z, &h2, 4);
      memcpy(&v.w, &h3, 4);
      *reinterpret_cast<uint4*>(arow + kg * 128) = v;
    }
  }
  // make the generic-proxy writes of R visible to the tensor cores
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  // 4. the GEMM: D[t] (128 x 64, FP32, TMEM columns 64 t) = R[t] B^T
  __shared__ int ok_s;
  if (tid == 0) {
    int ok = mbar_wait(bar_b, 0, first_wait_limit) ? 1 : 0;
    if (ok) {
      const uint32_t a0 = su32(sm + OFF_A), b0 = su32(sm + OFF_B);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint64_t da = umma_desc(a0 + t * 16384 + s * 256);
          const uint64_t db = umma_desc(b0 + s * 256);
          const uint32_t acc = s > 0 ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem + t * 64),
              "l"(da), "l"(db), "r"(IDESC), "r"(acc));
        }
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                   : "memory");
    }
    ok_s = ok;
  }
  __syncthreads();
  bool ok = ok_s != 0 && mbar_wait(bar_mma, 0);
  if (!ok && tid == 0) atomicExch(err, 1);
  ok = __syncthreads_and(ok);
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok) {
    // 5. this thread's row of D -> shared corrections (thread = patch)
    float* sd = reinterpret_cast<float*>(sm + OFF_D);
    const uint32_t taddr = tmem + (static_cast<uint32_t>(32 * (warp & 3)) << 16) + 64 * (warp >> 2);
    float d[64];
#pragma unroll
    for (int ch = 0; ch < 4; ++ch) tmem_ld16(taddr + 16 * ch, d + 16 * ch);
    __syncthreads();  // every thread is done with R, B and the residual before they are overwritten
#pragma unroll
    for (int k = 0; k < 51; ++k) sd[tid * 51 + k] = d[k];
    __syncthreads();
    // 6. weighted update of the owned dofs: one thread per owned vertex (vi, vj);
    //    its Q2 nodes (2i-1..2i) x (2j-1..2j) take the corrections of the 9 / 6 /
    //    6 / 4 patches around them at compile-time offsets (patch q + dq, slot s).
    //    Warp w takes vertex rows 2w and 2w + 1 (lanes 0..27): their patches q
    //    lie in two rows of 16, distinct modulo 32, so the reads of D (pitch 51,
    //    odd) are free of bank conflicts.
    const int uw = tid >> 5, ul = tid & 31;
    if (uw < TC_TILE / 2 && ul < 2 * TC_TILE) {
      const int vj = 2 * uw + (ul >= TC_TILE ? 1 : 0), vi = ul - (ul >= TC_TILE ? TC_TILE : 0);
      const int i = i0 + vi, j = j0 + vj;
      const float* dq = sd + ((vj + 1) * TT::QW + (vi + 1)) * 51;  // the vertex's own patch
      const int xj = 2 * j - XJ0, xi = 2 * i - XI0;                  // x window at node (2i, 2j)
      const long long base = static_cast<long long>(2 * j) * nq + 2 * i;
#pragma unroll
      for (int nj = 0; nj < 2; ++nj) {        // node J = 2j - nj
#pragma unroll
        for (int ni = 0; ni < 2; ++ni) {      // node I = 2i - ni
          const float2 xold = x != nullptr ? sx[(xj - nj) * XP + xcol(xi - ni)] : make_float2(0.0f, 0.0f);
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            float acc = 0.0f;
            // patches (i + di, j + dj): di in {-1, 0, +1} for an even node, {-1, 0} for an odd one
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
              for (int di = -1; di <= 1; ++di) {
                if ((ni == 1 && di == 1) || (nj == 1 && dj == 1)) continue;
                const int wi = 2 - ni - 2 * di, wj = 2 - nj - 2 * dj;  // window offsets of the node
                acc += dq[(dj * TT::QW + di) * 51 + c * 25 + wj * 5 + wi];
              }
            }
            const float w = omega * (ni ? 0.5f : (1.0f / 3.0f)) * (nj ? 0.5f : (1.0f / 3.0f));
            xo[c * nv + base - static_cast<long long>(nj) * nq - ni] = fmaf(w, acc, c == 0 ? xold.x : xold.y);
          }
        }
      }
      const float xoldp = x != nullptr ? sp[(j - (j0 - 3)) * PP + (i - (i0 - 3))] : 0.0f;
      xo[2 * nv + static_cast<long long>(j) * np + i] = fmaf(omega, dq[50], xoldp);
    }
  } else if (tid == 0) {
    // the bulk copy and the MMAs may still be in flight: wait (bounded) before leaving
    mbar_wait(bar_b, 0);
    if (ok_s) mbar_wait(bar_mma, 0);
  }

  // teardown: free TMEM
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
}

}  // namespace

// Interior 14 x 14 tiles: origin i0 = 14 bx with 3 <= i0 and i0 + 14 <= n - 2,
// so every patch (vertex i0-1 .. i0+14) is of the interior class.
void tc_interior_range(int n, int* lo, int* hi) {
  *lo = 1;
  *hi = (n - 2 - TC_TILE) / TC_TILE;
  if (n < 2 + 2 * TC_TILE) *hi = 0;  // no interior tile
}

cudaError_t vanka_tc_prepare() {
  return cudaFuncSetAttribute(k_vanka_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_BYTES);
}

void launch_vanka_tc(const LevelDev& L, const void* Bcanon, const float* x, const float* b, float* xo,
                     double omega, int lo, int hi, int* err, cudaStream_t s, int first_wait_limit) {
  if (hi < lo) return;
  count_launches(1);
  g_tc_launches.fetch_add(1, std::memory_order_relaxed);
  const int g = hi - lo + 1;
  launch_pdl(k_vanka_tc, dim3(dim3(g, g)), dim3(TC_NT), SMEM_BYTES, s, L, static_cast<const uint4*>(Bcanon), x, b, xo,
                                                   static_cast<float>(omega), lo, err, first_wait_limit);
}

void tc_pack_inverse(const double* inv51, unsigned short* out) {
  // B[n][k] = A_int^-1[n][k] (N = output slot, K = input slot), zero padded to 64 x 64,
  // stored K-major in 8 x 8 core matrices: byte offset (n/8)*1024 + (k/8)*128 + (n%8)*16 + (k%8)*2
  for (int i = 0; i < 64 * 64; ++i) out[i] = 0;
  for (int nn = 0; nn < 51; ++nn) {
    for (int k = 0; k < 51; ++k) {
      const float v = static_cast<float>(inv51[nn * 51 + k]);
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      unsigned short bits;
      memcpy(&bits, &h, 2);
      const int off = (nn / 8) * 1024 + (k / 8) * 128 + (nn % 8) * 16 + (k % 8) * 2;
      out[off / 2] = bits;
    }
  }
}

}  // namespace sv
