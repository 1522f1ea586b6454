// sv_vanka_tc.cu -- additive Vanka sweep with the interior patch solves as BF16
// GEMMs on the 5th-generation tensor cores (tcgen05), for the mixed-precision
// preconditioner (FP32 vectors, FP32 accumulation).
//
// Section 6.3 of the paper observes that on a uniform grid all interior patches
// share one patch matrix A_int.  The solves delta_i = A_int^-1 r_i of a group of
// patches are therefore one product D = R A_int^-T, with R the matrix of gathered
// patch residuals (Algorithm 3, Section 3.2): one tcgen05.mma (kind::f16,
// BF16 x BF16 -> FP32 in tensor memory) of M = 128 patches, N = K = 51 padded
// to 64.
//
// Work decomposition.  A CTA (128 threads, warp r <-> row r of a step) sweeps a
// segment of a strip: 28 owned vertex columns [i0, i0 + 28) and S owned vertex
// rows [j0, j0 + S), S a multiple of 4.  It walks up the segment in steps of 4
// rows, keeping the rows it still needs in shared-memory rings, so a residual
// cell or a patch is computed once per strip instead of once per square tile
// (halo overhead 32/28 in cells and 30/28 in patches, against 18^2/14^2 and
// 16^2/14^2 for a 14 x 14 tile).  Step t, three phases separated by barriers:
//   A. the residual b - A x of cell row group t (32 x 4 cells: one 2x2 cell of
//      Q2 nodes and its vertex per thread, compile-time stencils, (u_x, u_y)
//      pairs with packed FP32 FMAs) into the residual ring; the weighted
//      update of vertex rows j0 + 4t - 12 .. j0 + 4t - 9 from the partial-sum
//      ring; the loads of x, p and b for step t + 1 are issued here and
//      stored in phase C, so their latency overlaps the step's work;
//   B. the patch rows of group t (30 x 4 patches: one per thread, lanes 30 and
//      31 of each warp padding) gathered from the residual ring into the
//      K-major BF16 operand (core matrices of 8 rows x 16 bytes);
//   C. one thread issues the MMA of group t into one of two tensor-memory
//      buffers; every warp reads its patch row of group t - 1 from the other
//      buffer (tcgen05.ld: lane = patch), adds the corrections of the patches
//      that share a Q2 node column with warp shuffles, and stores per-node
//      partial sums (one float4 per node-pair and window row) in the
//      partial-sum ring; the prefetched rows are stored.
// Update: x_out = x + (omega / m_j) * (sum of the corrections of the patches
// that hold dof j): the 3 (or 2) partial sums of a node's row, added in a fixed
// order (deterministic, no atomics).
//
// Slot order of a patch row (the K dimension of R and both dimensions of the
// inverse image): the (u_x, u_y) pair of window node s = 5 wj + wi at 2s, 2s + 1
// (so that one BF16x2 conversion packs one node), the pressure at 50.
//
// Every wait is bounded; on expiry the kernel sets *err, waits (bounded, with
// the full limit) for its bulk copy and the last MMA it issued, frees its tensor
// memory and returns.  The limit of the first wait (the inverse's bulk copy) is
// a launch argument, so a test can make it expire (0 polls) without faulting or
// hanging anything.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>

#include "sv_fastdiag.cuh"
#include "sv_internal.h"
#include "sv_stencil.cuh"
#include "sv_vanka_common.cuh"

namespace sv {
namespace {

constexpr int SW = 2 * TC_TILE;     // owned vertex columns of a strip (28)
constexpr int NPC = SW + 2;         // patches per row of a step (30)
constexpr int NCC = SW + 4;         // residual cells per row (32)
constexpr int XN = 2 * SW + 12;     // x window nodes per row (68)
constexpr int NPW = SW + 6;         // p window vertices per row (34)
constexpr int GR = 4;               // vertex rows per step
constexpr int NT = 128;             // threads
// resident CTAs per SM: 4 in the GEMM form (tensor memory, shared memory), 5 in the
// FP32 form (registers)
__host__ __device__ constexpr int ctas_per_sm(bool tc) { return tc ? 4 : 5; }
static_assert(NCC == 32 && NPC <= 32 && GR * 32 == NT, "warp r <-> row r, lane <-> column");

// Rings (row index taken modulo the ring size; each holds exactly the rows that are
// alive across a phase boundary).  x: node rows, (u_x, u_y) pairs, column-parity
// split (even nodes at pair c/2, odd nodes at XHO + c/2): the stencil loads of a
// warp read 32 consecutive pairs; the prefetch stores of a half-warp (8 even, 8
// odd nodes) hit disjoint banks since XHO = 40 = 8 (mod 16).  The GEMM form stores
// the next step's x and p rows after phase B, over rows read in phase A (12 and 6
// rows); the FP32 form stores them at the end of phase A, beside the rows still
// being read (20 and 10 rows), so that no prefetched value is held in registers
// across its patch solves.
__host__ __device__ constexpr int xr_rows(bool tc) { return tc ? 12 : 20; }
__host__ __device__ constexpr int prr_rows(bool tc) { return tc ? 6 : 10; }
constexpr int XHO = 40, XPP = XHO + XN / 2;                 // node rows of 74 pairs
constexpr int RR = 12, RHO = 32, RPP = 64;                  // residual: 12 node rows of 64 pairs
constexpr int CRR = 8;                                      // cell rows (pressure residual)
constexpr int PPW = 36;                                     // p: vertex rows of 34 (+2)
constexpr int SRR = 6;                                      // partial sums: 6 patch rows
static_assert(XN / 2 <= XHO && (2 * XHO) % 32 == 16, "x ring layout");

// Shared-memory layout (bytes).  The FP32 strip sweep (TC = false) has no GEMM
// operands, so its rings start at 0; it keeps the next step's b of each thread's
// cell in BS ([value][thread], 9 values) instead of registers.
template <bool TC>
struct SL {
  static constexpr int A = 0;                               // 128 x 64 BF16 = 16 KB (TC)
  static constexpr int B = A + 128 * 64 * 2;                // 64 x 64 BF16 = 8 KB (TC)
  static constexpr int X = TC ? B + 64 * 64 * 2 : 0;
  static constexpr int R = X + xr_rows(TC) * XPP * 8;
  static constexpr int RPR = R + RR * RPP * 8;
  static constexpr int P = RPR + CRR * NCC * 4;
  static constexpr int PS = P + prr_rows(TC) * PPW * 4;      // [row][wj][lane] float4
  static constexpr int PSP = PS + SRR * 5 * 32 * 16;         // [row][lane] pressure corrections
  static constexpr int BS = PSP + SRR * 32 * 4;
  static constexpr int BAR = BS + (TC ? 0 : 9 * NT * 4);     // bulk-copy and MMA mbarriers
  static constexpr int TMEM = BAR + 16;
  static constexpr int FLAG = TMEM + 4;
  static constexpr int BYTES = FLAG + 12;
  static_assert(X % 16 == 0 && PS % 16 == 0 && BAR % 8 == 0, "alignment");
  static_assert(ctas_per_sm(TC) * (BYTES + 1024) <= 228 * 1024, "resident CTAs per SM");
};

constexpr uint32_t TMEM_COLS = 128;   // two 64-column accumulators (4 CTAs per SM: all 512 columns)
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

// this lane's 52 accumulator columns (32 + 16 + 4) from tensor memory
__device__ __forceinline__ void tmem_ld52(uint32_t taddr, float* v) {
  uint32_t r[52];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47])
      : "r"(taddr + 32));
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51])
               : "r"(taddr + 48));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 52; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
  uint32_t u;
  memcpy(&u, &h, 4);
  return u;
}

// A global load issued where it is written: the memory clobber keeps the compiler
// from sinking it towards its first use (the prefetches of a step are issued at the
// top of phase A and consumed a phase or a step later, which hides their latency).
__device__ __forceinline__ float ldg_early(const float* p) {
  float v;
  asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
  return v;
}

// z_u of the interior patches (the Schur vector K^-1 b^T at unit viscosity and
// spacing, u_x window then u_y window) for the FP32 strip sweep; a level scales it
// by zs.  Compile-time slot indices make it a constant-bank operand.
__constant__ float c_zu_strip[50];

// TC: the BF16 tensor-core sweep; !TC: the FP32 strip sweep, each thread solving
// its interior patch by fast diagonalisation (fdp: the (v, v) pairs of the FP32
// factors; z_u from constant memory) in the same strip walk.
template <bool TC>
__global__ void __launch_bounds__(NT, ctas_per_sm(TC)) k_vanka_strip(LevelDev L, const uint4* __restrict__ Bg,
                                                       const FastDiagT<float2> fdp, const float* __restrict__ x,
                                                       const float* __restrict__ b, float* __restrict__ xo,
                                                       float omega, int lo, int hi, int seg_rows,
                                                       int* __restrict__ err, int first_wait_limit) {
  pdl_begin();
  using Y = SL<TC>;
  constexpr int XR = xr_rows(TC), PRR = prr_rows(TC);
  extern __shared__ __align__(1024) unsigned char sm[];
  float2* sx = reinterpret_cast<float2*>(sm + Y::X);
  float2* sr = reinterpret_cast<float2*>(sm + Y::R);
  float* srp = reinterpret_cast<float*>(sm + Y::RPR);
  float* sp = reinterpret_cast<float*>(sm + Y::P);
  float4* sps = reinterpret_cast<float4*>(sm + Y::PS);
  float* spp = reinterpret_cast<float*>(sm + Y::PSP);
  float* sbs = reinterpret_cast<float*>(sm + Y::BS);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + Y::BAR);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + Y::TMEM);
  volatile int* s_fail = reinterpret_cast<volatile int*>(sm + Y::FLAG);
  const uint32_t bar_b = su32(bars), bar_mma = su32(bars + 1);
  const int nq = L.nq, np = L.np;
  const long long nv = L.nv;
  const int tid = threadIdx.x, r = tid >> 5, l = tid & 31;
  const int i0 = TC_TILE * (lo + 2 * static_cast<int>(blockIdx.x));
  const int j0 = TC_TILE * lo + seg_rows * static_cast<int>(blockIdx.y);
  const int S = min(seg_rows, TC_TILE * (hi + 1) - j0);   // owned rows, a multiple of 4
  const int T = S / GR;                                     // steps with cells / patches
  const int XI0 = 2 * i0 - 6;                               // x window origin (Q2 column)
  const bool has_x = x != nullptr;
  const float cl = L.clf, cb = L.cbf;

  // ---- set-up: barriers, tensor memory, bulk copy of the BF16 inverse, zero pad rows ----
  if (tid == 0) {
    if constexpr (TC) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_b), "r"(1));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar_mma), "r"(1));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    *s_fail = 0;
  }
  __syncwarp();
  uint32_t tmem = 0;
  if constexpr (TC) {
    if (r == 0) {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)),
                   "r"(TMEM_COLS));
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    // A: lanes 30, 31 of every 32-row group are padding patches (zero rows); the K
    // chunk 7 (slots 56..63) of every row is zero
    unsigned char* arow = sm + Y::A + (tid >> 3) * 1024 + (tid & 7) * 16;
    const uint4 z = make_uint4(0u, 0u, 0u, 0u);
    if (l >= NPC) {
#pragma unroll
      for (int kg = 0; kg < 8; ++kg) *reinterpret_cast<uint4*>(arow + kg * 128) = z;
    } else {
      *reinterpret_cast<uint4*>(arow + 7 * 128) = z;
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if constexpr (TC) {
    tmem = *tslot;
    if (tid == 0) {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar_b), "r"(64 * 64 * 2)
                   : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
              su32(sm + Y::B)),
          "l"(Bg), "r"(64 * 64 * 2), "r"(bar_b)
          : "memory");
    }
  }

  // ---- loaders (warp r takes rows r, r + 4, ...) ----
  // x node row J: lane l takes the window-column pairs (2 q, 2 q + 1), q = l and l + 32
  // (< 34), i.e. nodes XI0 + 2 q (even half, pair q) and XI0 + 2 q + 1 (odd half, pair
  // q): [k] = (u_x, u_y) of node XI0 + 2 q + k; 0 on Dirichlet / outside nodes
  struct XPair {
    float2 v[2];
  };
  auto x_pair = [&](int J, int q) -> XPair {
    XPair o;
    const bool jok = J > 0 && J < nq - 1;
    const float* xr = x + static_cast<long long>(jok ? J : 1) * nq + XI0 + 2 * q;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int I = XI0 + 2 * q + k;
      o.v[k] = (jok && I > 0 && I < nq - 1) ? make_float2(ldg_early(xr + k), ldg_early(xr + nv + k))
                                            : make_float2(0.0f, 0.0f);
    }
    return o;
  };
  auto x_pair_store = [&](int J, int q, const XPair& v) {
    float2* row = sx + (J % XR) * XPP;
    row[q] = v.v[0];
    row[XHO + q] = v.v[1];
  };
  // p vertex row j (vertices i0 - 3 .. i0 + 30), window column c
  auto p_item = [&](int j, int c) -> float {
    const int i = i0 - 3 + c;
    return (i >= 0 && j >= 0 && i < np && j < np) ? ldg_early(x + 2 * nv + static_cast<long long>(j) * np + i) : 0.0f;
  };
  // b of this thread's cell (column l, row cy): [PJ][PI] pairs and the vertex's pressure row
  struct BCell {
    float2 v[2][2];
    float p;
  };
  auto b_load = [&](int cy) -> BCell {
    BCell o;
    const int cx = i0 - 2 + l;
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
      for (int PI = 0; PI < 2; ++PI) {
        const long long k = static_cast<long long>(2 * cy + PJ) * nq + 2 * cx + PI;
        o.v[PJ][PI] = make_float2(ldg_early(b + k), ldg_early(b + nv + k));
      }
    o.p = ldg_early(b + 2 * nv + static_cast<long long>(cy) * np + cx);
    return o;
  };
  // FP32 form: the next step's b of this thread's cell, kept in shared memory
  auto b_stash = [&](const BCell& v) {
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
      for (int PI = 0; PI < 2; ++PI) {
        sbs[(4 * PJ + 2 * PI) * NT + tid] = v.v[PJ][PI].x;
        sbs[(4 * PJ + 2 * PI + 1) * NT + tid] = v.v[PJ][PI].y;
      }
    sbs[8 * NT + tid] = v.p;
  };
  auto b_unstash = [&]() -> BCell {
    BCell o;
#pragma unroll
    for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
      for (int PI = 0; PI < 2; ++PI)
        o.v[PJ][PI] = make_float2(sbs[(4 * PJ + 2 * PI) * NT + tid], sbs[(4 * PJ + 2 * PI + 1) * NT + tid]);
    o.p = sbs[8 * NT + tid];
    return o;
  };

  // prologue: x rows 2 j0 - 6 .. 2 j0 + 5, p rows j0 - 3 .. j0 + 2, b of step 0
  if (has_x) {
    for (int rr = r; rr < 12; rr += GR) {
      const int J = 2 * j0 - 6 + rr;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int q = l + 32 * k;
        if (q < XN / 2) x_pair_store(J, q, x_pair(J, q));
      }
    }
    for (int rr = r; rr < 6; rr += GR) {
      const int j = j0 - 3 + rr;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const int c = l + 32 * k;
        if (c < NPW) sp[(j % PRR) * PPW + c] = p_item(j, c);
      }
    }
  }
  // b of this step's cells (bc) and of the next step's (bn), loaded two steps ahead
  // (GEMM form); the FP32 form stashes step 0's and loads one step ahead
  BCell bc, bn;
  if constexpr (TC) {
    bc = b_load(j0 - 2 + r);
    bn = b_load(j0 + 2 + r);
  } else {
    b_stash(b_load(j0 - 2 + r));
  }
  __syncthreads();

  // prefetch registers (step t + 1): x rows 2 j0 + 8 t + 6 + {r, r + 4} x 2 column-pair
  // chunks, p row j0 + 4 t + 3 + r x 2 chunks
  XPair xpf[2][2];
  float ppf[2];
  // x at the dofs of this step's update (0 for a zero guess): loaded a step earlier in
  // the GEMM form, at the top of phase A in the FP32 form
  float xold[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) xold[k] = 0.0f;
  uint32_t mma_phase = 0;

  // the update trails the residual by 3 steps with the GEMM (its corrections are read
  // a step after their MMA), by 2 with the FP32 solve
  constexpr int LAG = TC ? 12 : 8;
  for (int t = 0; t <= T + (TC ? 2 : 1); ++t) {
    // ================= phase A: residual of cell rows t, update, prefetch =================
    const bool pf = (t + 1 <= T);
    // the update of this step (vertex row vb) and its x_old (9 values per vertex; in
    // L2: its rows were loaded into the window)
    const int vb = j0 + 4 * t - LAG + r;
    const bool upd = vb >= j0 && vb < j0 + S && l >= 1 && l <= SW;
    const int vi = i0 + l - 1;
    const long long ke = static_cast<long long>(2 * vb) * nq + 2 * vi;   // node (2 vi, 2 vb)
    const long long ko = ke - nq;                                         // node (2 vi, 2 vb - 1)
    const long long kp = 2 * nv + static_cast<long long>(vb) * np + vi;
    auto load_xold = [&](int dv, float* o) {   // vertex row vb + dv
      const int vr = vb + dv;
      if (has_x && vr >= j0 && vr < j0 + S && l >= 1 && l <= SW) {
        const long long kk = ke + 2LL * dv * nq, kq = kk - nq, kpp = kp + static_cast<long long>(dv) * np;
        o[0] = ldg_early(x + kk);
        o[1] = ldg_early(x + nv + kk);
        o[2] = ldg_early(x + kk - 1);
        o[3] = ldg_early(x + nv + kk - 1);
        o[4] = ldg_early(x + kq);
        o[5] = ldg_early(x + nv + kq);
        o[6] = ldg_early(x + kq - 1);
        o[7] = ldg_early(x + nv + kq - 1);
        o[8] = ldg_early(x + kpp);
      } else {
#pragma unroll
        for (int k = 0; k < 9; ++k) o[k] = 0.0f;
      }
    };
    float xold_n[TC ? 9 : 1];
    BCell bn2;   // b two steps ahead (GEMM form), one step ahead (FP32 form)
    if constexpr (TC) {
      load_xold(GR, xold_n);
      if (t + 2 <= T) bn2 = b_load(j0 + 4 * t + 6 + r);
    } else {
      load_xold(0, xold);
      if (t + 1 <= T) bn2 = b_load(j0 + 4 * t + 2 + r);
    }
    if (pf) {
      if (has_x) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int J = 2 * j0 + 8 * t + 6 + r + 4 * h;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int q = l + 32 * k;
            if (q < XN / 2) xpf[h][k] = x_pair(J, q);
          }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = l + 32 * k;
          if (c < NPW) ppf[k] = p_item(j0 + 4 * t + 3 + r, c);
        }
      }
    }
    if (t <= T) {
      // cell (cx, cy) = (i0 - 2 + l, j0 - 2 + 4 t + r): Q2 nodes (2 cx + PI, 2 cy + PJ)
      const int cy = j0 - 2 + 4 * t + r;
      if constexpr (!TC) bc = b_unstash();
      float2 res[2][2];
#pragma unroll
      for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
        for (int PI = 0; PI < 2; ++PI) res[PJ][PI] = bc.v[PJ][PI];
      float rp = bc.p;
      if (has_x) {
        float P[3][3];
#pragma unroll
        for (int dj = 0; dj < 3; ++dj)
#pragma unroll
          for (int di = 0; di < 3; ++di) P[dj][di] = sp[((cy - 1 + dj) % PRR) * PPW + l + di];
        float2 slap[2][2];
#pragma unroll
        for (int PJ = 0; PJ < 2; ++PJ)
#pragma unroll
          for (int PI = 0; PI < 2; ++PI) slap[PJ][PI] = make_float2(0.0f, 0.0f);
        float2 sdiv = make_float2(0.0f, 0.0f);
        // rows a = 0..5 of the 6 x 6 pair neighbourhood (node (2 cx - 2 + bb, 2 cy - 2 + a))
#pragma unroll
        for (int a = 0; a < 6; ++a) {
          const float2* xrow = sx + ((2 * cy - 2 + a) % XR) * XPP + l;
          float2 Xa[6];
#pragma unroll
          for (int bb = 0; bb < 6; ++bb) Xa[bb] = xrow[(bb & 1) * XHO + (bb >> 1)];
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
                if (cf != 0.0f) slap[PJ][PI] = __ffma2_rn(make_float2(cf, cf), Xa[bb], slap[PJ][PI]);
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
            float2 g = make_float2(0.0f, 0.0f);   // (B^T p) / (-h/18) for (u_x, u_y)
#pragma unroll
            for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
              for (int di = -1; di <= 1; ++di) {
                const float w0 = static_cast<float>(ccol(2 + PI, 1 + di) * ncol(2 + PJ, 1 + dj));
                const float w1 = static_cast<float>(ncol(2 + PI, 1 + di) * ccol(2 + PJ, 1 + dj));
                const float pv = P[dj + 1][di + 1];
                if (w0 != 0.0f || w1 != 0.0f) g = __ffma2_rn(make_float2(w0, w1), make_float2(pv, pv), g);
              }
            }
            // r - (cl slap + cb g) as two packed multiply-adds
            res[PJ][PI] = __ffma2_rn(make_float2(-cl, -cl), slap[PJ][PI],
                                     __ffma2_rn(make_float2(-cb, -cb), g, res[PJ][PI]));
          }
        }
        rp -= cb * (sdiv.x + sdiv.y);
      }
#pragma unroll
      for (int PJ = 0; PJ < 2; ++PJ) {
        float2* rrow = sr + ((2 * cy + PJ) % RR) * RPP;
        rrow[l] = res[PJ][0];
        rrow[RHO + l] = res[PJ][1];
      }
      srp[(cy & (CRR - 1)) * NCC + l] = rp;
    }
    // weighted update of vertex row vb (partial sums of patch rows vb - 1 .. vb + 1)
    if (upd) {
      const float4* pm = sps + ((vb - 1) % SRR) * 160 + l;
      const float4* p0 = sps + (vb % SRR) * 160 + l;
      const float4* pp = sps + ((vb + 1) % SRR) * 160 + l;
      const float4 e4 = pm[4 * 32], e2 = p0[2 * 32], e0 = pp[0];   // node row 2 vb
      const float4 o3 = pm[3 * 32], o1 = p0[1 * 32];               // node row 2 vb - 1
      const float dp = spp[(vb % SRR) * 32 + l];
      // (odd column 2 vi - 1, even column 2 vi) x (even row, odd row)
      const float2 s_oe = __fadd2_rn(__fadd2_rn(make_float2(e4.x, e4.y), make_float2(e2.x, e2.y)),
                                     make_float2(e0.x, e0.y));
      const float2 s_ee = __fadd2_rn(__fadd2_rn(make_float2(e4.z, e4.w), make_float2(e2.z, e2.w)),
                                     make_float2(e0.z, e0.w));
      const float2 s_oo = __fadd2_rn(make_float2(o3.x, o3.y), make_float2(o1.x, o1.y));
      const float2 s_eo = __fadd2_rn(make_float2(o3.z, o3.w), make_float2(o1.z, o1.w));
      const float w9 = omega * (1.0f / 9.0f), w6 = omega * (1.0f / 6.0f), w4 = omega * 0.25f;
      xo[ke] = fmaf(w9, s_ee.x, xold[0]);
      xo[nv + ke] = fmaf(w9, s_ee.y, xold[1]);
      xo[ke - 1] = fmaf(w6, s_oe.x, xold[2]);
      xo[nv + ke - 1] = fmaf(w6, s_oe.y, xold[3]);
      xo[ko] = fmaf(w6, s_eo.x, xold[4]);
      xo[nv + ko] = fmaf(w6, s_eo.y, xold[5]);
      xo[ko - 1] = fmaf(w4, s_oo.x, xold[6]);
      xo[nv + ko - 1] = fmaf(w4, s_oo.y, xold[7]);
      xo[kp] = fmaf(omega, dp, xold[8]);
    }
    // the next step's x and p rows into their rings, b into its stash
    auto store_prefetch = [&]() {
      if (pf && has_x) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int J = 2 * j0 + 8 * t + 6 + r + 4 * h;
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const int q = l + 32 * k;
            if (q < XN / 2) x_pair_store(J, q, xpf[h][k]);
          }
        }
#pragma unroll
        for (int k = 0; k < 2; ++k) {
          const int c = l + 32 * k;
          if (c < NPW) sp[((j0 + 4 * t + 3 + r) % PRR) * PPW + c] = ppf[k];
        }
      }
    };
    if constexpr (!TC) {
      // FP32 form: rows no warp reads in this step (the rings hold both)
      store_prefetch();
      if (pf) b_stash(bn2);
    }
    // the MMA of step t - 1 must be complete before its operand is overwritten and
    // its accumulator read (issued a whole phase A earlier); the inverse's bulk copy
    // before the first MMA
    if constexpr (TC) {
      if (tid == 0) {
        bool ok = true;
        if (t == 0) ok = mbar_wait(bar_b, 0, first_wait_limit);
        if (ok && t >= 1 && t - 1 <= T) {
          ok = mbar_wait(bar_mma, mma_phase);
          mma_phase ^= 1u;
        }
        if (!ok) *s_fail = t == 0 ? 1 : 2;
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (*s_fail) break;

    // corrections of patch row pj to per-node partial sums (phase C with the GEMM, in
    // phase B with the FP32 solve, whose corrections are per thread, not in tensor memory).
    // patch row pj, lane l = patch pi = i0 - 1 + l; the node columns 2 pi - 1 (odd) and
    // 2 pi (even) of window row wj take
    //   odd:  D[pi - 1](wi = 3) + D[pi](wi = 1)
    //   even: D[pi - 1](wi = 4) + D[pi](wi = 2) + D[pi + 1](wi = 0)
    auto store_partials = [&](int pj, const float* d) {
      float4* dst = sps + (pj % SRR) * 160 + l;
#pragma unroll
      for (int wj = 0; wj < 5; ++wj) {
        const float* dw = d + 10 * wj;
        const float u3x = __shfl_up_sync(0xffffffffu, dw[6], 1), u3y = __shfl_up_sync(0xffffffffu, dw[7], 1);
        const float u4x = __shfl_up_sync(0xffffffffu, dw[8], 1), u4y = __shfl_up_sync(0xffffffffu, dw[9], 1);
        const float d0x = __shfl_down_sync(0xffffffffu, dw[0], 1), d0y = __shfl_down_sync(0xffffffffu, dw[1], 1);
        const float2 odd = __fadd2_rn(make_float2(u3x, u3y), make_float2(dw[2], dw[3]));
        const float2 even = __fadd2_rn(__fadd2_rn(make_float2(u4x, u4y), make_float2(dw[4], dw[5])),
                                       make_float2(d0x, d0y));
        dst[wj * 32] = make_float4(odd.x, odd.y, even.x, even.y);
      }
      spp[(pj % SRR) * 32 + l] = d[50];
    };
    // ================= phase B: the patch rows of group t =================
    // patch (pi, pj) = (i0 - 1 + l, j0 + 4 t - 3 + r); window node (2 pi - 2 + wi, 2 pj - 2 + wj)
    // sits at residual column 2 l + wi (even: pair l + wi/2, odd: RHO + l + (wi-1)/2)
    if constexpr (TC) {
      if (t <= T && l < NPC) {
        const int pj = j0 + 4 * t - 3 + r;
        uint32_t w[26];
#pragma unroll
        for (int wj = 0; wj < 5; ++wj) {
          const float2* rrow = sr + ((2 * pj - 2 + wj) % RR) * RPP + l;
#pragma unroll
          for (int wi = 0; wi < 5; ++wi) {
            const float2 v = rrow[(wi & 1) * RHO + (wi >> 1)];
            w[wj * 5 + wi] = pack_bf16x2(v.x, v.y);
          }
        }
        w[25] = pack_bf16x2(srp[(pj & (CRR - 1)) * NCC + l + 1], 0.0f);
        unsigned char* arow = sm + Y::A + (tid >> 3) * 1024 + (tid & 7) * 16;
#pragma unroll
        for (int kg = 0; kg < 7; ++kg) {
          const uint32_t a0 = 4 * kg < 26 ? w[4 * kg] : 0u;
          const uint32_t a1 = 4 * kg + 1 < 26 ? w[4 * kg + 1] : 0u;
          const uint32_t a2 = 4 * kg + 2 < 26 ? w[4 * kg + 2] : 0u;
          const uint32_t a3 = 4 * kg + 3 < 26 ? w[4 * kg + 3] : 0u;
          *reinterpret_cast<uint4*>(arow + kg * 128) = make_uint4(a0, a1, a2, a3);
        }
      }
      // make the generic-proxy writes of R visible to the tensor cores
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    } else if (t <= T) {
      // every lane takes part in the shuffles of the partial sums; lanes 30, 31 add zeros
      float d[52];
#pragma unroll
      for (int k = 0; k < 52; ++k) d[k] = 0.0f;
      const int pj = j0 + 4 * t - 3 + r;
      if (l < NPC) {
        // the exact interior patch solve (Section 6.3) in FP32, both velocity components
        // packed: dp = (z . r_u - r_p) / s with z = zs z_u, then K^-1 (r_u - b^T dp) by
        // fast diagonalisation; corrections in the kernel's slot order
        float2 r2[25];
#pragma unroll
        for (int wj = 0; wj < 5; ++wj) {
          const float2* rrow = sr + ((2 * pj - 2 + wj) % RR) * RPP + l;
#pragma unroll
          for (int wi = 0; wi < 5; ++wi) r2[wj * 5 + wi] = rrow[(wi & 1) * RHO + (wi >> 1)];
        }
        const float rp = srp[(pj & (CRR - 1)) * NCC + l + 1];
        float zr = 0.0f;
#pragma unroll
        for (int k = 0; k < 25; ++k) zr = fmaf(c_zu_strip[k], r2[k].x, zr);
#pragma unroll
        for (int k = 0; k < 25; ++k) zr = fmaf(c_zu_strip[25 + k], r2[k].y, zr);
        const float dp = (L.zsf * zr - rp) * L.zsinvf;
        const float q = cb * dp;
#pragma unroll
        for (int w = 0; w < 25; ++w) {
          const int dI = w % 5 - 2, dJ = w / 5 - 2;
          const float bx = static_cast<float>(crow(dI) * nrow(dJ)), by = static_cast<float>(nrow(dI) * crow(dJ));
          if (bx != 0.0f || by != 0.0f) r2[w] = __ffma2_rn(make_float2(-bx, -by), make_float2(q, q), r2[w]);
        }
        float2 y2[25];
        fdm::fd_solve<float2>(fdp, r2, y2);
#pragma unroll
        for (int w = 0; w < 25; ++w) {
          d[2 * w] = y2[w].x;
          d[2 * w + 1] = y2[w].y;
        }
        d[50] = dp;
      }
      store_partials(pj, d);
    }
    if constexpr (TC) {
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the MMA of group t, then the corrections of group t - 1 from the other buffer
      if (tid == 0 && t <= T) {
        const uint32_t a0 = su32(sm + Y::A), b0 = su32(sm + Y::B), acc = tmem + 64 * (t & 1);
#pragma unroll
        for (int s = 0; s < 4; ++s) {
          const uint64_t da = umma_desc(a0 + s * 256);
          const uint64_t db = umma_desc(b0 + s * 256);
          const uint32_t accum = s > 0 ? 1u : 0u;
          asm volatile(
              "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
              " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(acc),
              "l"(da), "l"(db), "r"(IDESC), "r"(accum));
        }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_mma)
                     : "memory");
      }
      __syncwarp();
      if (t >= 1 && t - 1 <= T) {
        float d[52];
        tmem_ld52(tmem + (static_cast<uint32_t>(32 * r) << 16) + 64 * ((t - 1) & 1), d);
        store_partials(j0 + 4 * (t - 1) - 3 + r, d);
      }
    }
    if constexpr (TC) {
      // GEMM form: over the rows phase A read
      store_prefetch();
      if (pf) {
        bc = bn;
        bn = bn2;
      }
#pragma unroll
      for (int k = 0; k < 9; ++k) xold[k] = xold_n[k];
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }

  if constexpr (TC) {
    const int fail = *s_fail;
    if (fail && tid == 0) {
      atomicExch(err, 1);
      // the bulk copy, and an MMA issued before the failed wait, may still be in flight
      mbar_wait(bar_b, 0);
      if (fail == 2) mbar_wait(bar_mma, mma_phase ^ 1u);
    }
    // teardown: free tensor memory
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (r == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

}  // namespace

// Interior 14 x 14 tiles [lo, hi]^2 (both axes): origin i0 = 14 bx with 3 <= i0
// and i0 + 14 <= n - 2, so every patch (vertex i0-1 .. i0+14) is of the interior
// class.  Strips are two tiles wide, so the range holds an even number of tiles
// (a last odd tile goes to the SIMT ring); no range below two tiles.
void tc_interior_range(int n, int* lo, int* hi) {
  *lo = 1;
  int h = (n - 2 - TC_TILE) / TC_TILE;
  if (n < 2 + 2 * TC_TILE) h = 0;
  const int cnt = h - *lo + 1;
  *hi = (cnt >= 2) ? *lo + (cnt & ~1) - 1 : 0;
}

cudaError_t vanka_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_vanka_strip<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, SL<true>::BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_vanka_strip<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, SL<false>::BYTES);
  return e;
}

cudaError_t set_strip_unit_z(const double* z50) {
  float zf[50];
  for (int k = 0; k < 50; ++k) zf[k] = static_cast<float>(z50[k]);
  return cudaMemcpyToSymbol(c_zu_strip, zf, 50 * sizeof(float));
}

namespace {
// Segments of a strip: a whole number of 4-row steps each.  A segment of s steps
// runs s + 3 loop iterations (the first computes residual rows below it, the last
// ones finish its updates), and the CTAs run in waves of ctas_per_sm per SM, so
// the time is about waves x (s + 3) step times: the count of segments per strip
// minimises that (ties: fewer CTAs).  At 2048^2 (72 strips of 504 steps, 152 SMs)
// that is 8 segments of 63 steps, 576 CTAs, in the GEMM form (4 per SM) and 10
// segments of 51 steps, 720 CTAs, in the FP32 form (5 per SM): one wave.
int strip_segment_steps(int strips, int steps, int slots) {
  long long best = -1;
  int best_s = steps;
  for (int nseg = 1; nseg <= steps; ++nseg) {
    const int s = (steps + nseg - 1) / nseg;
    const int used = (steps + s - 1) / s;   // segments actually launched
    const long long waves = (static_cast<long long>(strips) * used + slots - 1) / slots;
    const long long cost = waves * (s + 3);
    if (best < 0 || cost < best) {
      best = cost;
      best_s = s;
    }
  }
  return best_s;
}

dim3 strip_grid(int cnt, int* seg_rows, bool tc) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int steps = TC_TILE * cnt / GR;   // cnt is even: 28-row pairs of tiles
  const int s = strip_segment_steps(cnt / 2, steps, ctas_per_sm(tc) * sms);
  *seg_rows = GR * s;
  return dim3(cnt / 2, (steps + s - 1) / s);
}
}  // namespace

void launch_vanka_tc(const LevelDev& L, const void* Bcanon, const float* x, const float* b, float* xo,
                     double omega, int lo, int hi, int* err, cudaStream_t s, int first_wait_limit) {
  const int cnt = hi - lo + 1;
  if (cnt < 2 || (cnt & 1)) return;
  count_launches(1);
  g_tc_launches.fetch_add(1, std::memory_order_relaxed);
  int seg = GR;
  const dim3 grid = strip_grid(cnt, &seg, true);
  launch_pdl(k_vanka_strip<true>, grid, dim3(NT), SL<true>::BYTES, s, L, static_cast<const uint4*>(Bcanon),
             FastDiagT<float2>{}, x, b, xo, static_cast<float>(omega), lo, hi, seg, err, first_wait_limit);
}

void launch_vanka_strip_f32(const LevelDev& L, const FastDiagT<float>& fd, const float* x, const float* b,
                            float* xo, double omega, int lo, int hi, cudaStream_t s) {
  const int cnt = hi - lo + 1;
  if (cnt < 2 || (cnt & 1)) return;
  count_launches(1);
  // (v, v) pairs: both velocity components in one packed pass
  const FastDiagT<float2> fp = fd_cast<float2>(fd, [](float v) { return make_float2(v, v); });
  int seg = GR;
  const dim3 grid = strip_grid(cnt, &seg, false);
  launch_pdl(k_vanka_strip<false>, grid, dim3(NT), SL<false>::BYTES, s, L, static_cast<const uint4*>(nullptr), fp,
             x, b, xo, static_cast<float>(omega), lo, hi, seg, static_cast<int*>(nullptr), 0);
}

// slot of the dense 51 x 51 inverse (u_x window 0..24, u_y window 25..49, p 50)
// at position k of the kernel's patch row: (u_x, u_y) of window node s at 2 s, 2 s + 1
static int tc_slot(int k) { return k == 50 ? 50 : (k & 1) * 25 + (k >> 1); }

void tc_pack_inverse(const double* inv51, unsigned short* out) {
  // B[n][k] = A_int^-1[slot(n)][slot(k)] (N = output position, K = input position),
  // zero padded to 64 x 64, stored K-major in 8 x 8 core matrices: byte offset
  // (n/8)*1024 + (k/8)*128 + (n%8)*16 + (k%8)*2
  for (int i = 0; i < 64 * 64; ++i) out[i] = 0;
  for (int nn = 0; nn < 51; ++nn) {
    for (int k = 0; k < 51; ++k) {
      const float v = static_cast<float>(inv51[tc_slot(nn) * 51 + tc_slot(k)]);
      const __nv_bfloat16 h = __float2bfloat16_rn(v);
      unsigned short bits;
      memcpy(&bits, &h, 2);
      const int off = (nn / 8) * 1024 + (k / 8) * 128 + (nn % 8) * 16 + (k % 8) * 2;
      out[off / 2] = bits;
    }
  }
}

}  // namespace sv
