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
//   2. x and b windows are loaded and the FP32 residual is computed with
//      compile-time stencils (shared code with the SIMT sweep);
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
// Every wait is bounded; on expiry the kernel sets *err, waits (bounded) for
// its bulk copy, frees its TMEM and returns.
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
using vk::res_cell;
using vk::VT;
using vk::vfree;

constexpr int TC_NT = 256;
using TT = VT<TC_TILE, TC_TILE>;
static_assert(TT::NPATCH == TC_NT, "one thread per patch");

// shared-memory layout (bytes).  The correction array D (256 x 51 FP32,
// 52,224 B) overlays A, B, the residual and the pressure residual, which are
// all dead once the MMAs have completed; the x windows stay live for x_old.
constexpr int OFF_A = 0;                                   // 256 x 64 BF16 = 32 KB
constexpr int OFF_B = OFF_A + 256 * 64 * 2;                // 64 x 64 BF16 = 8 KB
constexpr int OFF_R = OFF_B + 64 * 64 * 2;                 // residual (FP32)
constexpr int OFF_RP = OFF_R + TT::SR * 4;                 // pressure residual
constexpr int OFF_X = OFF_RP + TT::SRP * 4;                // x window
constexpr int OFF_P = OFF_X + TT::SX * 4;                  // p window
constexpr int OFF_BAR = OFF_P + TT::SP * 4;                // two mbarriers
constexpr int OFF_TMEM = OFF_BAR + 16;                     // TMEM base address
constexpr int SMEM_BYTES = OFF_TMEM + 16;
constexpr int OFF_D = 0;                                   // corrections, after the MMAs
static_assert(OFF_D + TT::NPATCH * 51 * 4 <= OFF_X, "corrections overlay only dead buffers");
static_assert(OFF_BAR % 8 == 0, "mbarrier alignment");

constexpr uint32_t TMEM_COLS = 128;
constexpr int WAIT_LIMIT = 1 << 22;

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

__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t phase) {
  for (int it = 0; it < WAIT_LIMIT; ++it) {
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
                                                     float omega, int tile0, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char sm[];
  float* sx = reinterpret_cast<float*>(sm + OFF_X);
  float* sp = reinterpret_cast<float*>(sm + OFF_P);
  float* sr = reinterpret_cast<float*>(sm + OFF_R);
  float* srp = reinterpret_cast<float*>(sm + OFF_RP);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + OFF_BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + OFF_TMEM);
  const uint32_t bar_b = su32(bars), bar_mma = su32(bars + 1);
  const int nq = L.nq, np = L.np;
  const long long nv = L.nv;
  const int i0 = (tile0 + static_cast<int>(blockIdx.x)) * TC_TILE;
  const int j0 = (tile0 + static_cast<int>(blockIdx.y)) * TC_TILE;
  const int tid = threadIdx.x, warp = tid >> 5;
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

  // 2. windows and FP32 residual (all windows lie in the free interior here)
  if (x != nullptr) {
#pragma unroll
    for (int t = tid; t < TT::SX; t += TC_NT) {
      const int c = t / (TT::XW * TT::XH);
      const int rem = t - c * TT::XW * TT::XH;
      const int jj = rem / TT::XW, ii = rem - jj * TT::XW;
      const int I = XI0 + ii, J = XJ0 + jj;
      sx[t] = vfree(I, J, nq) ? x[c * nv + static_cast<long long>(J) * nq + I] : 0.0f;
    }
#pragma unroll
    for (int t = tid; t < TT::SP; t += TC_NT) {
      const int jj = t / TT::PW, ii = t - jj * TT::PW;
      const int i = i0 - 3 + ii, j = j0 - 3 + jj;
      sp[t] = (i >= 0 && j >= 0 && i < np && j < np) ? x[2 * nv + static_cast<long long>(j) * np + i] : 0.0f;
    }
  }
#pragma unroll
  for (int t = tid; t < TT::SR; t += TC_NT) {
    const int c = t / (TT::RW * TT::RH);
    const int rem = t - c * TT::RW * TT::RH;
    const int jj = rem / TT::RW, ii = rem - jj * TT::RW;
    const int I = RI0 + ii, J = RJ0 + jj;
    sr[t] = (I >= 0 && J >= 0 && I < nq && J < nq) ? b[c * nv + static_cast<long long>(J) * nq + I] : 0.0f;
  }
  {
    const int jj = tid / TT::QW, ii = tid - jj * TT::QW;
    const int i = i0 - 1 + ii, j = j0 - 1 + jj;
    srp[tid] = b[2 * nv + static_cast<long long>(j) * np + i];
  }
  __syncthreads();
  const float cl = L.clf, cb = L.cbf;
  if (x != nullptr) {
    for (int t = tid; t < TT::CW * TT::CH; t += TC_NT) {
      const int cy = t / TT::CW, cx = t - cy * TT::CW;
      const int I0 = RI0 + 2 * cx, J0 = RJ0 + 2 * cy;
      const float* x0 = sx + (2 * cy + 2) * TT::XW + (2 * cx + 2);
      const float* pc = sp + (cy + 1) * TT::PW + (cx + 1);
      float* r0 = sr + (2 * cy) * TT::RW + 2 * cx;
      res_cell<float, TT>(r0, x0, pc, I0, J0, L, x, cl, cb);
    }
    {
      const int jj = tid / TT::QW, ii = tid - jj * TT::QW;
      const float* xs0 = sx + (2 * jj + 4) * TT::XW + (2 * ii + 4);
      const float* xs1 = xs0 + TT::XW * TT::XH;
      float s = 0.0f;
#pragma unroll
      for (int dJ = -2; dJ <= 2; ++dJ) {
#pragma unroll
        for (int dI = -2; dI <= 2; ++dI) {
          const float wx = static_cast<float>(crow(dI) * nrow(dJ)), wy = static_cast<float>(nrow(dI) * crow(dJ));
          if (wx != 0.0f) s = fmaf(wx, xs0[dJ * TT::XW + dI], s);
          if (wy != 0.0f) s = fmaf(wy, xs1[dJ * TT::XW + dI], s);
        }
      }
      srp[tid] -= cb * s;
    }
  }
  __syncthreads();

  // 3. this thread's patch row of R (BF16, core-matrix layout)
  const int qj = tid / TT::QW, qi = tid - qj * TT::QW;
  {
    float row[64];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int wj = 0; wj < 5; ++wj)
#pragma unroll
        for (int wi = 0; wi < 5; ++wi)
          row[c * 25 + wj * 5 + wi] = sr[c * TT::RW * TT::RH + (2 * qj + wj) * TT::RW + 2 * qi + wi];
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
    int ok = mbar_wait(bar_b, 0) ? 1 : 0;
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
    if (tid < TC_TILE * TC_TILE) {
      const int vj = tid / TC_TILE, vi = tid - vj * TC_TILE;
      const int i = i0 + vi, j = j0 + vj;
      const float* dq = sd + ((vj + 1) * TT::QW + (vi + 1)) * 51;  // the vertex's own patch
      const float* xs = sx + (2 * j - XJ0) * TT::XW + (2 * i - XI0);  // x window at node (2i, 2j)
      const long long base = static_cast<long long>(2 * j) * nq + 2 * i;
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int nj = 0; nj < 2; ++nj) {      // node J = 2j - nj
#pragma unroll
          for (int ni = 0; ni < 2; ++ni) {    // node I = 2i - ni
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
            const float xold = x != nullptr ? xs[c * TT::XW * TT::XH - nj * TT::XW - ni] : 0.0f;
            xo[c * nv + base - static_cast<long long>(nj) * nq - ni] = fmaf(w, acc, xold);
          }
        }
      }
      const float xoldp = x != nullptr ? sp[(j - (j0 - 3)) * TT::PW + (i - (i0 - 3))] : 0.0f;
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
                     double omega, int lo, int hi, int* err, cudaStream_t s) {
  if (hi < lo) return;
  count_launches(1);
  const int g = hi - lo + 1;
  k_vanka_tc<<<dim3(g, g), TC_NT, SMEM_BYTES, s>>>(L, static_cast<const uint4*>(Bcanon), x, b, xo,
                                                   static_cast<float>(omega), lo, err);
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
